"""Pins of the oracle's robot model and its discretization (no GPU).

Each check is fixed by mechanics or by the method's definition, not by the
oracle's own formulas:

* balance laws of Eq. (1) at any joint-consistent pose (anchors coincide and
  anchor velocities agree): joint reaction forces and joint torques are
  internal, so total momentum, angular momentum and energy change only through
  gravity, contact forces and joint-torque power;
* closed-form trajectories that RK4 integrates exactly (polynomial in tau);
* the CTCS penalty (Eq. (12)) is exactly zero on feasible inputs and equals
  s h(d) for a body resting at penetration depth d;
* IND against central finite differences of the nonlinear flow map;
* the split identity: one interval with 2n substeps equals two half intervals
  (dilation s/2 each, FOH midpoint control) composed by the chain rule;
* s = 0 gives A = I, B- = B+ = 0 exactly.
"""
import numpy as np
import pytest

from paper_2604_09993_gb300 import synth

G = synth.GRAVITY


def _rot(th):
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]])


def _robot(name, seed=3):
    return synth.ROBOTS[name](np.random.default_rng(seed))


def _consistent_state(robot, rng):
    rel = rng.uniform(-0.6, 0.6, robot.nj)
    rates = rng.uniform(-2.0, 2.0, robot.nj)
    q, v = synth.fk(robot, rng.uniform(-1, 1, 2), rng.uniform(-0.5, 0.5), rel,
                    torso_v=rng.uniform(-1, 1, 2), torso_omega=rng.uniform(-2, 2), rel_rates=rates)
    x = np.zeros(robot.nxt)
    x[: 3 * robot.nb] = q.reshape(-1)
    x[3 * robot.nb: 6 * robot.nb] = v.reshape(-1)
    return q, v, x


@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7"])
def test_balance_laws(oracle_mod, name):
    robot = _robot(name)
    rng = np.random.default_rng(17)
    nb, nj = robot.nb, robot.nj
    m, I = robot.mass, robot.inertia
    for _ in range(5):
        q, v, x = _consistent_state(robot, rng)
        u = rng.standard_normal(robot.nu)
        f = oracle_mod.rhs(robot.as_dict(), x, u)
        acc = f[3 * nb: 6 * nb].reshape(nb, 3)
        # contact forces and points, computed here from the input convention
        Fc, Pc, Vc = [], [], []
        for i, b in enumerate(robot.contact_body):
            ln, ltp, ltm = u[3 * nj + 3 * i: 3 * nj + 3 * i + 3]
            r = _rot(q[b, 2]) @ robot.contact_rho[i]
            Fc.append(np.array([ltp - ltm, ln]))
            Pc.append(q[b, :2] + r)
            Vc.append(v[b, :2] + v[b, 2] * np.array([-r[1], r[0]]))
        Fg = np.stack([np.zeros(nb), -m * G], axis=1)
        # linear momentum
        dP = (m[:, None] * acc[:, :2]).sum(0)
        assert np.allclose(dP, sum(Fc) + Fg.sum(0), rtol=1e-12, atol=1e-10)
        # angular momentum about the origin
        cr = lambda a, b: a[0] * b[1] - a[1] * b[0]  # noqa: E731
        dL = sum(m[b] * cr(q[b, :2], acc[b, :2]) + I[b] * acc[b, 2] for b in range(nb))
        ext = sum(cr(Pc[i], Fc[i]) for i in range(len(Fc))) + sum(cr(q[b, :2], Fg[b]) for b in range(nb))
        assert abs(dL - ext) < 1e-10 * max(1.0, abs(ext))
        # power
        dE = sum(m[b] * v[b, :2] @ acc[b, :2] + I[b] * v[b, 2] * acc[b, 2] + m[b] * G * v[b, 1]
                 for b in range(nb))
        tau_power = sum(u[j] * (v[robot.joint_child[j], 2] - v[robot.joint_parent[j], 2]) for j in range(nj))
        ext_p = sum(Fc[i] @ Vc[i] for i in range(len(Fc))) + tau_power
        assert abs(dE - ext_p) < 1e-10 * max(1.0, abs(ext_p))


def _two_link():
    return {
        "mass": np.array([2.0, 1.5]), "inertia": np.array([0.3, 0.2]),
        "joint_parent": np.array([0]), "joint_child": np.array([1]),
        "joint_rho_parent": np.array([[0.0, -0.2]]), "joint_rho_child": np.array([[0.0, 0.15]]),
        "contact_body": np.zeros(0, dtype=np.int32), "contact_rho": np.zeros((0, 2)),
        "contact_mu": np.zeros(0), "gravity": G,
    }


@pytest.mark.parametrize("n_sub", [1, 5])
def test_free_flight_with_foh_torque_is_exact(oracle_mod, n_sub):
    """Only a joint torque acts: theta'' = +-tau(t)/I, p'' = (0, -g), all polynomial in tau."""
    R = _two_link()
    x0 = np.array([0.1, 1.0, 0.2, -0.3, 0.4, -0.5, 0.7, -0.2, 1.1, 0.3, 0.5, -0.8])
    uL = np.array([0.9, 0.0, 0.0])
    uR = np.array([-0.4, 0.0, 0.0])
    s = 0.8
    x1 = oracle_mod.flow(R, n_sub, x0, uL, uR, s)
    m, I = R["mass"], R["inertia"]
    for b, sign in ((0, -1.0), (1, 1.0)):
        px, py, th = x0[3 * b: 3 * b + 3]
        vx, vy, om = x0[6 + 3 * b: 6 + 3 * b + 3]
        a_L, a_R = sign * uL[0] / I[b], sign * uR[0] / I[b]
        exp_th = th + s * om + s * s * (a_L / 3.0 + a_R / 6.0)
        exp_om = om + s * (a_L + a_R) / 2.0
        exp_py = py + s * vy - 0.5 * G * s * s
        exp_vy = vy - G * s
        exp_px = px + s * vx
        got = x1[[3 * b, 3 * b + 1, 3 * b + 2, 6 + 3 * b, 6 + 3 * b + 1, 6 + 3 * b + 2]]
        assert np.allclose(got, [exp_px, exp_py, exp_th, vx, exp_vy, exp_om], rtol=0, atol=1e-13)


def _one_foot(L=0.4, m=2.0):
    return {
        "mass": np.array([m]), "inertia": np.array([m * L * L / 12.0]),
        "joint_parent": np.zeros(0, dtype=np.int32), "joint_child": np.zeros(0, dtype=np.int32),
        "joint_rho_parent": np.zeros((0, 2)), "joint_rho_child": np.zeros((0, 2)),
        "contact_body": np.array([0]), "contact_rho": np.array([[0.0, -L / 2.0]]),
        "contact_mu": np.array([1.0]), "gravity": G,
    }


@pytest.mark.parametrize("d", [0.0, 1e-3, 0.05, 0.7])
def test_resting_penetration_penalty(oracle_mod, d):
    """lambda_n = m g under the centre: the body stays put at depth d and
    y(1) - y(0) = s (sqrt(1 + d^2) - 1)."""
    L, m = 0.4, 2.0
    R = _one_foot(L, m)
    x0 = np.array([0.3, L / 2.0 - d, 0.0, 0.0, 0.0, 0.0, 0.25])
    u = np.array([m * G, 0.0, 0.0])
    s = 0.11
    x1 = oracle_mod.flow(R, 4, x0, u, u, s)
    assert np.allclose(x1[:6], x0[:6], rtol=0, atol=1e-15)
    assert abs((x1[6] - x0[6]) - s * (np.sqrt(1.0 + d * d) - 1.0)) < 1e-16


def test_constant_force_violation_penalty(oracle_mod):
    """lambda_n = -a (pulling) well above ground: g = (a, 0, 0, -phi<0, mu a):
    Omega = h(a) + h(mu a), constant in time (free fall does not reach ground)."""
    R = _one_foot()
    a = 0.8
    x0 = np.array([0.0, 5.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    u = np.array([-a, 0.0, 0.0])
    s = 0.07
    x1 = oracle_mod.flow(R, 3, x0, u, u, s)
    h = lambda z: np.sqrt(1.0 + z * z) - 1.0  # noqa: E731
    assert abs(x1[6] - s * (h(a) + h(1.0 * a))) < 1e-15


@pytest.mark.parametrize("name", ["hopper", "cheetah7"])
def test_energy_conserved_without_inputs(oracle_mod, name):
    """u = 0: every link flies ballistically (no joint or contact force), which
    RK4 integrates exactly, so E = sum(m v^2/2 + I w^2/2 + m g p_y) is kept."""
    robot = _robot(name)
    rng = np.random.default_rng(2)
    nb = robot.nb
    m, I = robot.mass, robot.inertia

    def energy(x):
        v = x[3 * nb: 6 * nb].reshape(nb, 3)
        py = x[: 3 * nb].reshape(nb, 3)[:, 1]
        return (0.5 * m * (v[:, 0] ** 2 + v[:, 1] ** 2) + 0.5 * I * v[:, 2] ** 2 + m * G * py).sum()

    for _ in range(3):
        _, _, x0 = _consistent_state(robot, rng)
        u = np.zeros(robot.nu)
        x1 = oracle_mod.flow(robot.as_dict(), 7, x0, u, u, 0.3)
        assert abs(energy(x1) - energy(x0)) < 1e-12 * max(1.0, abs(energy(x0)))


def test_feasible_inputs_give_zero_penalty(oracle_mod):
    robot = _robot("cheetah7")
    rng = np.random.default_rng(4)
    p = synth.draw_instance(robot, rng, 4, 5, q_noise=0.02, u_dist="normal", s_range=(0.04, 0.06))
    X = p.X.copy()
    X[:, 1: 3 * robot.nb: 3] += 0.6           # lift every link well above the ground
    X[:, 3 * robot.nb: 6 * robot.nb] = 0.0
    U = p.U.copy()
    for i in range(robot.nc):
        base = 3 * robot.nj + 3 * i
        U[:, base] = rng.uniform(1.0, 2.0, p.N + 1)          # lambda_n >= 0
        U[:, base + 1] = rng.uniform(0.0, 0.4, p.N + 1)      # lambda_t+ >= 0
        U[:, base + 2] = rng.uniform(0.0, 0.4, p.N + 1)      # sum <= mu lambda_n
    o = oracle_mod.discretize(robot.as_dict(), X, U, p.s, p.n_sub)
    ny = slice(robot.nx, robot.nxt)
    assert np.all(o["penalty"] == 0.0)
    assert np.all(o["Bm"][:, ny, :] == 0.0) and np.all(o["Bp"][:, ny, :] == 0.0)
    assert np.all(o["S"][:, ny] == 0.0)
    A_y = o["A"][:, ny, :].copy()
    for i in range(robot.nc):
        assert np.all(A_y[:, i, robot.nx + i] == 1.0)
        A_y[:, i, robot.nx + i] = 0.0
    assert np.all(A_y == 0.0)


def test_zero_dilation(oracle_mod):
    robot = _robot("hopper")
    rng = np.random.default_rng(8)
    p = synth.draw_instance(robot, rng, 2, 3, q_noise=0.05, u_dist="uniform", s_range=(0.1, 0.1))
    k = 0
    x1, A, Bm, Bp, S = oracle_mod.interval(robot.as_dict(), p.n_sub, p.X[k], p.U[k], p.U[k + 1], 0.0)
    assert np.array_equal(x1, p.X[k])
    assert np.array_equal(A, np.eye(robot.nxt))
    assert np.all(Bm == 0.0) and np.all(Bp == 0.0)
    # x rows: f is affine in u, so Simpson's rule gives f(x_k, (u_L + u_R)/2)
    f_mid = oracle_mod.rhs(robot.as_dict(), p.X[k], 0.5 * (p.U[k] + p.U[k + 1]))
    assert np.allclose(S[: robot.nx], f_mid[: robot.nx], rtol=1e-13, atol=1e-13)


def _fd_blocks(oracle_mod, R, n_sub, x0, uL, uR, s, e=1e-6):
    n, m = len(x0), len(uL)
    f = lambda a, b, c, d: oracle_mod.flow(R, n_sub, a, b, c, d)  # noqa: E731
    cols = []
    for c in range(n):
        dx = np.zeros(n); dx[c] = e
        cols.append((f(x0 + dx, uL, uR, s) - f(x0 - dx, uL, uR, s)) / (2 * e))
    for c in range(m):
        du = np.zeros(m); du[c] = e
        cols.append((f(x0, uL + du, uR, s) - f(x0, uL - du, uR, s)) / (2 * e))
    for c in range(m):
        du = np.zeros(m); du[c] = e
        cols.append((f(x0, uL, uR + du, s) - f(x0, uL, uR - du, s)) / (2 * e))
    cols.append((f(x0, uL, uR, s + e) - f(x0, uL, uR, s - e)) / (2 * e))
    J = np.stack(cols, axis=1)
    return J[:, :n], J[:, n:n + m], J[:, n + m:n + 2 * m], J[:, -1]


@pytest.mark.parametrize("name,n_sub", [("hopper", 1), ("hopper", 4), ("biped", 2), ("cheetah7", 3)])
def test_ind_matches_central_differences(oracle_mod, name, n_sub):
    robot = _robot(name, seed=6)
    rng = np.random.default_rng(21)
    p = synth.draw_instance(robot, rng, 2, n_sub, q_noise=0.05, u_dist="normal", s_range=(0.1, 0.2))
    R = robot.as_dict()
    for k in range(p.N):
        x1, A, Bm, Bp, S = oracle_mod.interval(R, n_sub, p.X[k], p.U[k], p.U[k + 1], p.s[k])
        assert np.allclose(x1, oracle_mod.flow(R, n_sub, p.X[k], p.U[k], p.U[k + 1], p.s[k]),
                           rtol=0, atol=1e-14)
        fA, fBm, fBp, fS = _fd_blocks(oracle_mod, R, n_sub, p.X[k], p.U[k], p.U[k + 1], p.s[k])
        for g, r, nm in ((A, fA, "A"), (Bm, fBm, "Bm"), (Bp, fBp, "Bp"), (S, fS, "S")):
            err = np.abs(g - r).max() / max(1.0, np.abs(r).max())
            assert err < 1e-6, (nm, err)


@pytest.mark.parametrize("name", ["hopper", "cheetah7"])
def test_split_interval_chain_rule(oracle_mod, name):
    robot = _robot(name, seed=12)
    R = robot.as_dict()
    rng = np.random.default_rng(31)
    p = synth.draw_instance(robot, rng, 1, 6, q_noise=0.05, u_dist="normal", s_range=(0.08, 0.12))
    x0, uL, uR, s = p.X[0], p.U[0], p.U[1], p.s[0]
    n = 3
    um = 0.5 * (uL + uR)
    x1, A, Bm, Bp, S = oracle_mod.interval(R, 2 * n, x0, uL, uR, s)
    xa, A1, Bm1, Bp1, S1 = oracle_mod.interval(R, n, x0, uL, um, 0.5 * s)
    xb, A2, Bm2, Bp2, S2 = oracle_mod.interval(R, n, xa, um, uR, 0.5 * s)
    tol = 1e-12
    sc = lambda a: max(1.0, np.abs(a).max())  # noqa: E731
    assert np.abs(xb - x1).max() < tol * sc(x1)
    assert np.abs(A2 @ A1 - A).max() < tol * sc(A)
    assert np.abs(A2 @ (Bm1 + 0.5 * Bp1) + 0.5 * Bm2 - Bm).max() < tol * sc(Bm)
    assert np.abs(0.5 * A2 @ Bp1 + 0.5 * Bm2 + Bp2 - Bp).max() < tol * sc(Bp)
    assert np.abs(0.5 * (A2 @ S1 + S2) - S).max() < tol * sc(S)


def test_discretize_defect_and_layouts(oracle_mod):
    """defect_k = F~(x~_k, U_k, s_k) - x~_{k+1} (Eq. (17b)); both control layouts agree."""
    p = synth.hopper_fp64()
    R = p.robot.as_dict()
    nx = p.robot.nx
    p.X[:, nx:] = np.random.default_rng(1).uniform(0.0, 1.0, (p.N + 1, p.robot.nc))  # y_k != 0
    o = oracle_mod.discretize(R, p.X, p.U, p.s, p.n_sub)
    oi = oracle_mod.discretize(R, p.X, p.U_interval(), p.s, p.n_sub, layout="interval")
    for key in o:
        assert np.array_equal(o[key], oi[key]), key
    for k in range(p.N):
        x1 = oracle_mod.flow(R, p.n_sub, p.X[k], p.U[k], p.U[k + 1], p.s[k])
        assert np.allclose(o["defect"][k], x1 - p.X[k + 1], rtol=0, atol=1e-15)
        assert np.allclose(o["penalty"][k], x1[nx:] - p.X[k, nx:], rtol=0, atol=1e-15)
