"""Pins for the oracle's paper-faithful dynamics (no GPU):

* joint reaction forces eliminated at the acceleration level (Sec. II-A,
  Eq. (3)): the constraint acceleration vanishes (checked by a numerical second
  derivative of the joint gaps from forward kinematics alone), the reaction
  forces lie in the range of grad C^T (checked against the input-force model
  with zero joint forces, projected on a numerically differentiated null space
  of grad C), momentum and energy are conserved where physics says so;
* the sinusoidal contact surface (Sec. VI-B): the approximate signed distance
  agrees with the exact distance to the curve up to O(h^c^2), the contact frame
  is the curve's unit normal and tangent, flat ground is reproduced exactly;
* the Runge-Kutta-Fehlberg 4(5) scheme (Sec. VI): order conditions of its
  tableau, its stability polynomial on a linear system, fifth-order convergence
  on the nonlinear robot;
* the IND blocks of all of it against central finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_09993_gb300 import synth


def _robot(name="biped", seed=0, **kw):
    rng = np.random.default_rng(seed)
    return synth.with_paper_dynamics(getattr(synth, name)(rng), **kw)


def _gaps(R, q):
    """Joint gaps C_j(q) = p_c + R(theta_c) rho_c - p_p - R(theta_p) rho_p, [nj, 2]."""
    q = q.reshape(-1, 3)
    out = []
    for j in range(R.nj):
        p, c = R.joint_parent[j], R.joint_child[j]
        rot = lambda th: np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])  # noqa: E731
        out.append(q[c, :2] + rot(q[c, 2]) @ R.joint_rho_child[j] - q[p, :2] - rot(q[p, 2]) @ R.joint_rho_parent[j])
    return np.array(out).reshape(-1)


def _random_state(R, rng, scale=0.3):
    X = rng.uniform(-scale, scale, R.nxt)
    X[2:3 * R.nb:3] = rng.uniform(-1.0, 1.0, R.nb)        # angles
    X[3 * R.nb + 2:6 * R.nb:3] = rng.uniform(-2.0, 2.0, R.nb)  # angular rates
    return X


# ---------------------------------------------------------------------------
# Eq. (3): acceleration-level elimination of the joint reaction forces
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7"])
def test_constraint_acceleration_vanishes(name):
    """d^2/dt^2 C(q(t)) = 0 along q(t) = q + t v + t^2/2 v' for the returned v'."""
    R = _robot(name, seed=1, scheme=0)
    rng = np.random.default_rng(2)
    for _ in range(3):
        x = _random_state(R, rng)
        u = rng.standard_normal(R.nu)
        vd = oracle.rhs(R.as_dict(), x, u)[3 * R.nb:6 * R.nb]
        q, v = x[:3 * R.nb], x[3 * R.nb:6 * R.nb]
        eps = 1e-4
        curve = lambda t: q + t * v + 0.5 * t * t * vd  # noqa: E731
        c2 = (_gaps(R, curve(eps)) - 2 * _gaps(R, curve(0.0)) + _gaps(R, curve(-eps))) / eps**2
        assert np.max(np.abs(c2)) < 1e-6 * max(1.0, np.max(np.abs(vd))), c2


@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7"])
def test_reaction_forces_in_range_of_constraint_gradient(name):
    """M v' - F lies in range(grad C^T): it is orthogonal to every velocity
    direction the joints admit (virtual power), F from the input-force model
    with zero joint forces; grad C from finite differences of the joint gaps."""
    R = _robot(name, seed=3, scheme=0, terrain=synth.TERRAIN_SINE)
    Rin = synth.with_paper_dynamics(R, joint_forces=0, scheme=0)
    rng = np.random.default_rng(4)
    nq = 3 * R.nb
    M = np.repeat(R.mass, 3).astype(float)
    M[2::3] = R.inertia
    for _ in range(3):
        x = _random_state(R, rng)
        u = rng.standard_normal(R.nu)
        uin = np.concatenate([u[:R.nj], np.zeros(2 * R.nj), u[R.nj:]])
        vd = oracle.rhs(R.as_dict(), x, u)[nq:2 * nq]
        a_free = oracle.rhs(Rin.as_dict(), x, uin)[nq:2 * nq]
        resid = M * (vd - a_free)
        q = x[:nq]
        G = np.zeros((2 * R.nj, nq))
        for a in range(nq):
            e = np.zeros(nq)
            e[a] = 1e-6
            G[:, a] = (_gaps(R, q + e) - _gaps(R, q - e)) / 2e-6
        _, sv, Vt = np.linalg.svd(G)
        null = Vt[np.sum(sv > 1e-8):]
        assert null.shape[0] == nq - 2 * R.nj
        proj = null @ resid
        assert np.max(np.abs(proj)) < 1e-7 * max(1.0, np.max(np.abs(resid))), proj
        # and the reaction forces are not zero (the elimination does something)
        assert np.max(np.abs(resid)) > 1e-3


def _consistent_state(R, rng):
    rel = rng.uniform(-0.6, 0.6, R.nj)
    rates = rng.uniform(-2.0, 2.0, R.nj)
    q, v = synth.fk(R, (0.1, 1.0), rng.uniform(-0.3, 0.3), rel, torso_v=(0.4, -0.2),
                    torso_omega=0.7, rel_rates=rates)
    x = np.zeros(R.nxt)
    x[:3 * R.nb] = q.reshape(-1)
    x[3 * R.nb:6 * R.nb] = v.reshape(-1)
    return x


def _energy(R, x):
    nb = R.nb
    q = x[:3 * nb].reshape(nb, 3)
    v = x[3 * nb:6 * nb].reshape(nb, 3)
    return float(np.sum(0.5 * R.mass * (v[:, 0] ** 2 + v[:, 1] ** 2) + 0.5 * R.inertia * v[:, 2] ** 2
                        + R.mass * R.gravity * q[:, 1]))


@pytest.mark.parametrize("scheme,ratio", [(0, 16.0), (1, 32.0)])
def test_energy_and_constraints_drift_at_the_scheme_order(scheme, ratio):
    """Unforced chain under gravity: the eliminated reaction forces do no work,
    so energy and the joint gaps drift only by the integration error, which
    shrinks by 2^order per halving of the step."""
    R = _robot("cheetah7", seed=5, scheme=scheme)
    x0 = _consistent_state(R, np.random.default_rng(6))
    assert np.max(np.abs(_gaps(R, x0[:3 * R.nb]))) < 1e-12
    u = np.zeros(R.nu)
    E0 = _energy(R, x0)
    dE, dC = [], []
    for n in (8, 16, 32):
        x1 = oracle.flow(R.as_dict(), n, x0, u, u, 0.6)
        dE.append(abs(_energy(R, x1) - E0))
        dC.append(np.max(np.abs(_gaps(R, x1[:3 * R.nb]))))
    for errs in (dE, dC):
        r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
        assert 0.6 * ratio < r1 < 1.6 * ratio and 0.6 * ratio < r2 < 1.6 * ratio, (errs, r1, r2)


def test_momentum_without_gravity():
    """g = 0, no contact forces, random joint torques: linear momentum is
    conserved to round-off (a linear invariant RK keeps exactly), angular
    momentum about the origin to the integration error."""
    R = synth.with_paper_dynamics(_robot("biped", seed=7), scheme=1)
    R.gravity = 0.0
    rng = np.random.default_rng(8)
    x0 = _consistent_state(R, rng)
    uL = np.concatenate([rng.standard_normal(R.nj), np.zeros(3 * R.nc)])
    uR = np.concatenate([rng.standard_normal(R.nj), np.zeros(3 * R.nc)])
    nb = R.nb

    def momenta(x):
        q = x[:3 * nb].reshape(nb, 3)
        v = x[3 * nb:6 * nb].reshape(nb, 3)
        P = (R.mass[:, None] * v[:, :2]).sum(0)
        L = float(np.sum(R.inertia * v[:, 2] + R.mass * (q[:, 0] * v[:, 1] - q[:, 1] * v[:, 0])))
        return P, L

    P0, L0 = momenta(x0)
    errs = []
    for n in (8, 16):
        x1 = oracle.flow(R.as_dict(), n, x0, uL, uR, 0.5)
        P1, L1 = momenta(x1)
        assert np.max(np.abs(P1 - P0)) < 1e-12
        errs.append(abs(L1 - L0))
    assert errs[1] < errs[0] / 10.0 and errs[1] < 1e-5, errs
    # the torques did change the motion
    assert np.max(np.abs(x1[3 * nb:6 * nb] - x0[3 * nb:6 * nb])) > 1e-2


# ---------------------------------------------------------------------------
# Sec. VI-B: sinusoidal contact surface
# ---------------------------------------------------------------------------
def _single_body(terrain, aux=0, mass=2.0, inertia=0.3, rho=(0.1, -0.2)):
    return {"mass": np.array([mass]), "inertia": np.array([inertia]),
            "joint_parent": np.zeros(0, np.int32), "joint_child": np.zeros(0, np.int32),
            "joint_rho_parent": np.zeros((0, 2)), "joint_rho_child": np.zeros((0, 2)),
            "contact_body": np.array([0], np.int32), "contact_rho": np.array([rho], float),
            "contact_mu": np.array([1.0]), "gravity": 0.0, "aux_model": aux, "terrain": terrain}


def _place(R, theta, point):
    """Body pose (p_x, p_y, theta) that puts the contact point at `point`."""
    c, s = math.cos(theta), math.sin(theta)
    r = np.array([c * R["contact_rho"][0][0] - s * R["contact_rho"][0][1],
                  s * R["contact_rho"][0][0] + c * R["contact_rho"][0][1]])
    return np.array([point[0] - r[0], point[1] - r[1], theta])


def _curve_frame(a, k, x):
    d = a * k * math.cos(k * x)  # slope of y = a sin(k x)
    w = 1.0 / math.sqrt(1.0 + d * d)
    return np.array([w, d * w]), np.array([-d * w, w])  # unit tangent (+x), unit normal (up)


def _exact_distance(a, k, p):
    xs = np.linspace(p[0] - 1.0, p[0] + 1.0, 200001)
    d2 = (xs - p[0]) ** 2 + (a * np.sin(k * xs) - p[1]) ** 2
    x = xs[np.argmin(d2)]
    for _ in range(30):  # Newton on the stationarity of the squared distance
        f = a * math.sin(k * x) - p[1]
        g = (x - p[0]) + f * a * k * math.cos(k * x)
        h = 1.0 + (a * k * math.cos(k * x)) ** 2 - f * a * k * k * math.sin(k * x)
        x -= g / h
    dist = math.hypot(x - p[0], a * math.sin(k * x) - p[1])
    return math.copysign(dist, p[1] - a * math.sin(k * p[0]))


def _node_phi(R, x):
    z = np.zeros(6 + 1)
    z[:3] = x
    th = oracle.node_value(R, z, z, np.array([0.0, 0.0]), np.array([0.0]), 1e-3, np.array([0.0]))[1]
    return -th[5]


def test_signed_distance_is_second_order_accurate():
    a, k = synth.TERRAIN_SINE
    R = _single_body((a, k))
    rng = np.random.default_rng(9)
    for x in rng.uniform(-1.0, 1.0, 6):
        _, n = _curve_frame(a, k, x)
        on = np.array([x, a * math.sin(k * x)])
        assert abs(_node_phi(R, _place(R, 0.3, on))) < 1e-15
        for eps in (1e-2, -1e-2, 1e-3, -1e-3):
            p = on + eps * n  # exact distance eps
            phi = _node_phi(R, _place(R, 0.3, p))
            d = _exact_distance(a, k, p)
            assert abs(d - eps) < 1e-9
            assert abs(phi - d) <= 3.0 * eps * eps, (x, eps, phi, d)


def test_flat_ground_reproduces_the_flat_model():
    R = _robot("biped", seed=10, scheme=0)
    Rt = synth.with_paper_dynamics(R, terrain=(0.0, 3.0))
    rng = np.random.default_rng(11)
    x, u = _random_state(R, rng), rng.standard_normal(R.nu)
    assert np.array_equal(oracle.rhs(R.as_dict(), x, u), oracle.rhs(Rt.as_dict(), x, u))


@pytest.mark.parametrize("aux", [0, 1])
def test_contact_force_acts_along_the_curve_frame(aux):
    """Unit normal input -> force along the curve's unit normal; unit tangential
    input -> force along its unit tangent; also off the surface (the frame of
    the level set through the point, which is the vertical translate of the curve)."""
    a, k = synth.TERRAIN_SINE
    m = 2.0
    R = _single_body((a, k), aux=aux, mass=m)
    rng = np.random.default_rng(12)
    for x in rng.uniform(-1.0, 1.0, 4):
        t, n = _curve_frame(a, k, x)
        for off in (0.0, 0.07):
            pose = _place(R, -0.4, (x, a * math.sin(k * x) + off))
            st = np.concatenate([pose, np.zeros(3), np.zeros(5 if aux else 1)])
            # aux 0 inputs (lambda_n, lambda_t+, lambda_t-); aux 1 (phi_t, phi_n, gamma)
            un = np.array([1.0, 0.0, 0.0]) if aux == 0 else np.array([0.0, 1.0, 0.0])
            ut = np.array([0.0, 1.0, 0.0]) if aux == 0 else np.array([1.0, 0.0, 0.0])
            np.testing.assert_allclose(m * oracle.rhs(R, st, un)[3:5], n, atol=1e-14)
            np.testing.assert_allclose(m * oracle.rhs(R, st, ut)[3:5], t, atol=1e-14)


def test_tangential_velocity_along_the_curve():
    """Eq. (12) lambda^c = t^T J_c v (gamma = 0): the contact point's velocity along the curve tangent."""
    a, k = synth.TERRAIN_SINE
    R = _single_body((a, k), aux=1)
    x = 0.37
    t, _ = _curve_frame(a, k, x)
    pose = _place(R, 0.2, (x, a * math.sin(k * x)))
    v = np.array([0.8, -0.3, 0.0])
    st = np.concatenate([pose, v, np.zeros(5)])
    out = oracle.rhs(R, st, np.zeros(3))
    assert abs(out[6 + 1] - t @ v[:2]) < 1e-14


def test_impact_impulse_in_the_curve_frame():
    """Node constraints on the sinusoidal surface: the impulse (Phi_t, Phi_n)
    enters the impact map as t Phi_t + n Phi_n (single free link, v+ = v-)."""
    a, k = synth.TERRAIN_SINE
    R = _single_body((a, k))
    x = -0.61
    t, n = _curve_frame(a, k, x)
    pose = _place(R, 0.5, (x, a * math.sin(k * x)))
    z = np.concatenate([pose, [0.3, 0.1, 0.2], [0.0]])
    g, _ = oracle.node_value(R, z, z, np.array([0.7, 1.3]), np.array([0.0]), 1e-3, np.array([0.0]))
    np.testing.assert_allclose(-g[3:5], 0.7 * t + 1.3 * n, atol=1e-14)


# ---------------------------------------------------------------------------
# Sec. VI: Runge-Kutta-Fehlberg 4(5)
# ---------------------------------------------------------------------------
def _order_conditions(b, A, c):
    """Butcher's order conditions up to order 5 (one per rooted tree)."""
    Ac = A @ c
    return [
        (b.sum(), 1.0),
        (b @ c, 1 / 2),
        (b @ c**2, 1 / 3), (b @ Ac, 1 / 6),
        (b @ c**3, 1 / 4), (b @ (c * Ac), 1 / 8), (b @ (A @ c**2), 1 / 12), (b @ (A @ Ac), 1 / 24),
        (b @ c**4, 1 / 5), (b @ (c**2 * Ac), 1 / 10), (b @ Ac**2, 1 / 20), (b @ (c * (A @ c**2)), 1 / 15),
        (b @ (A @ c**3), 1 / 20), (b @ (c * (A @ Ac)), 1 / 30), (b @ (A @ (c * Ac)), 1 / 40),
        (b @ (A @ (A @ c**2)), 1 / 60), (b @ (A @ (A @ Ac)), 1 / 120),
    ]


@pytest.mark.parametrize("scheme,order", [(0, 4), (1, 5)])
def test_tableau_order_conditions(scheme, order):
    s, c, A, b = oracle.tableau(scheme)
    c, A, b = c[:s], A[:s, :s], b[:s]
    assert np.all(np.triu(A) == 0.0)  # explicit
    np.testing.assert_allclose(A.sum(1), c, atol=1e-15)
    n_conds = {4: 8, 5: 17}[order]
    conds = _order_conditions(b, A, c)
    for got, want in conds[:n_conds]:
        assert abs(got - want) < 1e-14, (got, want)
    if order == 4:  # classical RK4 is exactly fourth order
        assert any(abs(g - w) > 1e-6 for g, w in conds[8:])


@pytest.mark.parametrize("scheme", [0, 1])
def test_stability_polynomial_on_a_linear_system(scheme):
    """For x' = s Ac x the step map is R(h s Ac) with R(z) = 1 + sum_k b^T A^(k-1) 1 z^k."""
    st, c, A, b = oracle.tableau(scheme)
    A, b = A[:st, :st], b[:st]
    rng = np.random.default_rng(13)
    n = 5
    Ac = rng.standard_normal((n, n))
    Bc = rng.standard_normal((n, 2))
    nsub, s = 3, 0.7
    x0, uL, uR = rng.standard_normal(n), rng.standard_normal(2), rng.standard_normal(2)
    _, Aout, _, _, _ = oracle.linear_interval(Ac, Bc, nsub, x0, uL, uR, s, scheme=scheme)
    Z = (s / nsub) * Ac
    Rz = np.eye(n)
    Zk = np.eye(n)
    coef = np.ones(st)
    for k in range(1, st + 1):
        Zk = Zk @ Z
        gamma = b @ np.linalg.matrix_power(A, k - 1) @ np.ones(st)
        Rz = Rz + gamma * Zk
        coef[k - 1] = gamma
    np.testing.assert_allclose(Aout, np.linalg.matrix_power(Rz, nsub), rtol=1e-12, atol=1e-13)
    assert np.allclose(coef[:4], [1, 1 / 2, 1 / 6, 1 / 24])


def test_rkf45_converges_at_fifth_order_on_the_robot():
    R = _robot("hopper", seed=14, scheme=1, terrain=synth.TERRAIN_SINE)
    rng = np.random.default_rng(15)
    x0 = _consistent_state(R, rng)
    uL, uR = rng.standard_normal(R.nu), rng.standard_normal(R.nu)
    ref = oracle.flow(R.as_dict(), 512, x0, uL, uR, 0.5)
    e = [np.max(np.abs(oracle.flow(R.as_dict(), n, x0, uL, uR, 0.5) - ref)) for n in (8, 16, 32)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 20.0 < r1 < 50.0 and 20.0 < r2 < 50.0, (e, r1, r2)
    # RK4 on the same problem converges to the same flow
    R4 = synth.with_paper_dynamics(R, scheme=0)
    e4 = np.max(np.abs(oracle.flow(R4.as_dict(), 128, x0, uL, uR, 0.5) - ref))
    assert e4 < 1e-7


# ---------------------------------------------------------------------------
# IND blocks against central finite differences
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,aux", [("hopper", 0), ("biped", 1)])
def test_ind_blocks_match_finite_differences(name, aux):
    R = _robot(name, seed=16, scheme=1, terrain=synth.TERRAIN_SINE)
    if aux:
        R = synth.with_cross_states(R)
    d = R.as_dict()
    rng = np.random.default_rng(17)
    x0 = _consistent_state(R, rng)
    x0[1:3 * R.nb:3] -= 0.95  # feet near the surface
    uL, uR = rng.standard_normal(R.nu), rng.standard_normal(R.nu)
    s, nsub = 0.12, 3
    _, A, Bm, Bp, S = oracle.interval(d, nsub, x0, uL, uR, s)
    F = lambda x, a, c, ss: oracle.flow(d, nsub, x, a, c, ss)  # noqa: E731
    h = 1e-6

    def fd(fun, v):
        J = np.zeros((R.nxt, v.size))
        for i in range(v.size):
            e = np.zeros(v.size)
            e[i] = h
            J[:, i] = (fun(v + e) - fun(v - e)) / (2 * h)
        return J

    for got, want in ((A, fd(lambda v: F(v, uL, uR, s), x0)),
                      (Bm, fd(lambda v: F(x0, v, uR, s), uL)),
                      (Bp, fd(lambda v: F(x0, uL, v, s), uR)),
                      (S[:, None], fd(lambda v: F(x0, uL, uR, v[0]), np.array([s])))):
        assert np.max(np.abs(got - want)) <= 2e-6 * max(1.0, np.max(np.abs(want)))
