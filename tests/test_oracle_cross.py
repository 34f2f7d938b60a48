"""Pins of the oracle's full auxiliary state (aux model 1, Sec. IV-A Eq. (12)):
per contact four cross-complementarity states integrating
(phi_n, lambda^c, gamma, rho^c) and one path-penalty state, with contact
inputs (phi_t, phi_n, gamma).

Nothing here re-types the oracle's right-hand side:
* the phi_n and gamma states integrate inputs that are affine in tau under
  the first-order hold, so RK4 gives their exact integral s (u_L + u_R) / 2;
* with gamma = 0, lambda^c is the tangential velocity of the contact point, so
  its state's increment converges (fourth order) to the contact point's x
  displacement over the interval, measured from the poses by rotation
  matrices;
* rho^c vanishes exactly on the friction-cone boundary |phi_t| = mu |phi_n|
  and its state is then 0; with constant inputs it is s rho^c;
* feasible inputs (phi_n, gamma > 0 inside the cone, contact point above
  ground) leave the path-penalty state and its Jacobian rows exactly 0;
* the IND Jacobian matches central differences of the nonlinear flow map.
"""
import numpy as np
import pytest

import oracle
from paper_2604_09993_gb300 import synth


def _robot(name="hopper", seed=3):
    rng = np.random.default_rng(seed)
    return synth.with_cross_states(getattr(synth, name)(rng))


def _rot(th):
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]])


def _contact_x(R, x, i):
    b = R.contact_body[i]
    return x[3 * b] + (_rot(x[3 * b + 2]) @ R.contact_rho[i])[0]


def _interval(R, rng, nsub=4, s=0.1, feasible=False):
    nb, nj, nc = R.nb, R.nj, R.nc
    x0 = np.zeros(R.nxt)
    x0[: 6 * nb] = rng.uniform(-0.3, 0.3, 6 * nb)
    uL = rng.standard_normal(R.nu)
    uR = rng.standard_normal(R.nu)
    if feasible:
        for i in range(nc):
            c0 = 3 * nj + 3 * i
            for u in (uL, uR):
                u[c0 + 1] = rng.uniform(1.0, 2.0)                        # phi_n > 0
                u[c0] = rng.uniform(-0.3, 0.3) * R.contact_mu[i] * u[c0 + 1]  # inside the cone
                u[c0 + 2] = rng.uniform(0.1, 0.5)                        # gamma > 0
            x0[3 * R.contact_body[i] + 1] += 3.0                         # far above the ground
    return x0, uL, uR, s, nsub


def test_dimensions():
    R = _robot("cheetah7")
    m = oracle.OracleModel(R.as_dict())
    assert (m.nxt, m.nu) == (6 * R.nb + 5 * R.nc, 3 * R.nj + 3 * R.nc) == (R.nxt, R.nu)


@pytest.mark.parametrize("name", ["hopper", "biped"])
def test_phi_n_and_gamma_states_integrate_exactly(name):
    R = _robot(name)
    rng = np.random.default_rng(1)
    x0, uL, uR, s, nsub = _interval(R, rng, nsub=3, s=0.13)
    x1 = oracle.flow(R.as_dict(), nsub, x0, uL, uR, s)
    nx, nj = 6 * R.nb, R.nj
    for i in range(R.nc):
        c0 = 3 * nj + 3 * i
        assert abs(x1[nx + 4 * i] - s * (uL[c0 + 1] + uR[c0 + 1]) / 2) <= 1e-15
        assert abs(x1[nx + 4 * i + 2] - s * (uL[c0 + 2] + uR[c0 + 2]) / 2) <= 1e-15


def test_lambda_c_state_converges_to_contact_displacement():
    """gamma = 0: d y_lambda / dtau = s t^T J_c v = d(contact x)/dtau."""
    R = _robot("hopper")
    rng = np.random.default_rng(2)
    x0, uL, uR, s, _ = _interval(R, rng, s=0.2)
    c0 = 3 * R.nj
    uL[c0 + 2] = uR[c0 + 2] = 0.0
    nx = 6 * R.nb
    errs = []
    for nsub in (4, 8, 16, 32, 64):
        x1 = oracle.flow(R.as_dict(), nsub, x0, uL, uR, s)
        disp = _contact_x(R, x1, 0) - _contact_x(R, x0, 0)
        errs.append(abs(x1[nx + 1] - disp))
    assert errs[-1] <= 1e-9
    ratios = [errs[k] / errs[k + 1] for k in range(len(errs) - 1) if errs[k + 1] > 1e-14]
    assert len(ratios) == 4 and all(14.0 < r < 18.0 for r in ratios), (errs, ratios)


def test_contact_force_moves_a_free_link():
    """One link with one contact, no joints: the contact-frame force (phi_t,
    phi_n) is the world force, so the velocity changes by s (average force)/m
    (plus gravity); linear in tau under the first-order hold."""
    R = {"mass": np.array([2.0]), "inertia": np.array([0.3]),
         "joint_parent": np.zeros(0, dtype=np.int32), "joint_child": np.zeros(0, dtype=np.int32),
         "joint_rho_parent": np.zeros((0, 2)), "joint_rho_child": np.zeros((0, 2)),
         "contact_body": np.array([0], dtype=np.int32), "contact_rho": np.array([[0.1, -0.4]]),
         "contact_mu": np.array([0.7]), "gravity": 9.81, "aux_model": 1}
    x0 = np.zeros(6 + 5)
    x0[:6] = [0.3, 0.5, 0.7, -0.2, -1.1, 0.0]
    uL = np.array([0.8, 2.0, 0.1])
    uR = np.array([-0.4, 3.0, 0.2])
    s = 0.15
    x1 = oracle.flow(R, 5, x0, uL, uR, s)
    assert abs(x1[3] - (x0[3] + s * (uL[0] + uR[0]) / 2 / 2.0)) <= 1e-14
    assert abs(x1[4] - (x0[4] + s * ((uL[1] + uR[1]) / 2 / 2.0 - 9.81))) <= 1e-14


def test_rho_c_state_on_and_inside_the_cone():
    R = _robot("hopper")
    R.contact_mu[:] = 0.6
    rng = np.random.default_rng(3)
    x0, uL, uR, s, nsub = _interval(R, rng, nsub=2, s=0.1)
    c0, nx, mu = 3 * R.nj, 6 * R.nb, R.contact_mu[0]
    # on the boundary, constant in tau: rho^c = 0 exactly
    for u in (uL, uR):
        u[c0 + 1] = 1.3
        u[c0] = -mu * 1.3
    x1 = oracle.flow(R.as_dict(), nsub, x0, uL, uR, s)
    assert x1[nx + 3] == 0.0
    # constant inputs strictly inside: s rho^c with rho^c = |mu phi_n|~ - |phi_t|~ > 0
    uR[c0] = uL[c0] = 0.2
    x1 = oracle.flow(R.as_dict(), nsub, x0, uL, uR, s)
    assert x1[nx + 3] > 0.0
    x1b = oracle.flow(R.as_dict(), 2 * nsub, x0, uL, uR, s)
    assert abs(x1[nx + 3] - x1b[nx + 3]) <= 1e-16  # integrand constant in tau


def test_feasible_inputs_leave_the_path_penalty_exactly_zero():
    R = _robot("biped")
    rng = np.random.default_rng(4)
    x0, uL, uR, s, nsub = _interval(R, rng, nsub=3, s=0.1, feasible=True)
    x1, A, Bm, Bp, S = oracle.interval(R.as_dict(), nsub, x0, uL, uR, s)
    pen = slice(6 * R.nb + 4 * R.nc, R.nxt)
    assert np.all(x1[pen] == 0.0)
    assert not np.any(A[pen, : 6 * R.nb]) and not np.any(Bm[pen]) and not np.any(Bp[pen])
    assert not np.any(S[pen])


def test_cross_ind_matches_central_differences():
    R = _robot("hopper")
    rng = np.random.default_rng(5)
    x0, uL, uR, s, nsub = _interval(R, rng, nsub=2, s=0.12)
    x1, A, Bm, Bp, S = oracle.interval(R.as_dict(), nsub, x0, uL, uR, s)
    f = lambda x, a, b, ss: oracle.flow(R.as_dict(), nsub, x, a, b, ss)  # noqa: E731
    h = 1e-6
    for c in range(R.nxt):
        e = np.zeros(R.nxt)
        e[c] = h
        fd = (f(x0 + e, uL, uR, s) - f(x0 - e, uL, uR, s)) / (2 * h)
        assert np.max(np.abs(fd - A[:, c])) <= 1e-6 * max(1.0, np.max(np.abs(A))), c
    for q in range(R.nu):
        e = np.zeros(R.nu)
        e[q] = h
        fdm = (f(x0, uL + e, uR, s) - f(x0, uL - e, uR, s)) / (2 * h)
        fdp = (f(x0, uL, uR + e, s) - f(x0, uL, uR - e, s)) / (2 * h)
        assert np.max(np.abs(fdm - Bm[:, q])) <= 1e-6 * max(1.0, np.max(np.abs(Bm))), q
        assert np.max(np.abs(fdp - Bp[:, q])) <= 1e-6 * max(1.0, np.max(np.abs(Bp))), q
    fds = (f(x0, uL, uR, s + h) - f(x0, uL, uR, s - h)) / (2 * h)
    assert np.max(np.abs(fds - S)) <= 1e-6 * max(1.0, np.max(np.abs(S)))


def test_cross_discretize_penalty_is_the_path_state_increment():
    R = _robot("hopper")
    rng = np.random.default_rng(6)
    p = synth.draw_instance(R, rng, 7, 3, q_noise=0.05, u_dist="normal", s_range=(0.05, 0.15))
    out = oracle.discretize(R.as_dict(), p.X, p.U, p.s, p.n_sub)
    assert out["penalty"].shape == (7, R.nc)
    pen = 6 * R.nb + 4 * R.nc
    assert np.allclose(out["penalty"][:, 0], out["defect"][:, pen] + p.X[1:, pen] - p.X[:-1, pen],
                       rtol=0, atol=1e-14)
