"""Pins of the oracle's canonical SOCP of the SCP subproblem (oracle/socp.py).

Nothing here re-types the assembly; each check goes back to the nonlinear
functions or to the definitions of the objective and the sets:
* at the iterate, A zhat - b and the Theta/Psi rows of G zhat - h equal the
  row scales times the nonlinear constraint values (the flow map minus the
  next pre-impact state, the impact map, Theta, Psi, the boundary gaps),
  evaluated from the plain-FP64 functions with the variables unscaled;
* away from the iterate they agree to second order (error ratio 4 per halving);
* the input rows and friction cones accept a feasible control and reject
  exactly the row a violated bound belongs to; a Q^2 block holds iff
  |phi_t| <= mu phi_n;
* after normalization every row's largest problem-variable entry is 1;
* objective differences equal the proximal term, the torque cost integrated
  by Simpson's rule (exact for the quadratic FOH integrand) and the slack
  penalty, computed from their definitions.
"""
import numpy as np
import pytest

import oracle
from oracle import socp
from paper_2604_09993_gb300 import synth

NSUB, DELTA, EPS = 4, 0.05, 1e-4


def _case(name="hopper", cross=False, layout="node", N=3, seed=0, scaled=True):
    rng = np.random.default_rng(seed)
    Rb = getattr(synth, name)(rng)
    R = (synth.with_cross_states(Rb) if cross else Rb).as_dict()
    m = oracle.OracleModel(R)
    nxt, nu, nb, nj, nc = m.nxt, m.nu, m.nb, m.nj, m.nc
    Xp = np.zeros((N + 1, nxt))
    Xp[:, : 6 * nb] = rng.uniform(-0.3, 0.3, (N + 1, 6 * nb))
    Xp[:, 6 * nb:] = rng.uniform(-0.5, 0.5, (N + 1, nxt - 6 * nb))
    Xm = Xp + 0.05 * rng.standard_normal(Xp.shape)
    U = rng.standard_normal((N + 1, nu) if layout == "node" else (N, 2, nu))
    s = rng.uniform(0.05, 0.15, N)
    Phi = rng.standard_normal((N + 1, 2 * nc))
    Gam = rng.uniform(0.1, 1.0, (N + 1, nc))
    e = rng.uniform(0, 1, nc)
    prm = {"w_px": 3.0, "w_ep": 50.0, "w_torque": 0.7, "s_min": 0.02, "s_max": 0.3,
           "torque_max": rng.uniform(2, 4, nj), "x_init": rng.uniform(-0.2, 0.2, 6 * nb),
           "x_final": rng.uniform(-0.2, 0.2, 6 * nb)}
    if scaled:
        prm.update(scale_x=rng.uniform(0.5, 2, nxt), offset_x=rng.uniform(-0.1, 0.1, nxt),
                   scale_u=rng.uniform(0.5, 2, nu), offset_u=rng.uniform(-0.1, 0.1, nu),
                   scale_s=0.1, offset_s=0.05, scale_phi=rng.uniform(0.5, 2, 2 * nc),
                   offset_phi=rng.uniform(-0.1, 0.1, 2 * nc), scale_gam=rng.uniform(0.5, 2, nc),
                   offset_gam=rng.uniform(-0.1, 0.1, nc))
    out = socp.assemble(R, N, layout, prm, Xp, Xm, U, s, Phi, Gam, NSUB, DELTA, EPS, e)
    return R, out, e, prm


def _unpack(L, z):
    N = L.N
    Xp = np.array([z[L.col["xp", k]] for k in range(N + 1)])
    Xm = np.array([z[L.col["xm", k]] for k in range(N + 1)])
    Phi = np.array([z[L.col["phi", k]] for k in range(N + 1)])
    Gam = np.array([z[L.col["gam", k]] for k in range(N + 1)])
    s = np.array([z[L.col["s", k]][0] for k in range(N)])
    uL = [z[L.uL(k)] for k in range(N)]
    uR = [z[L.uR(k)] for k in range(N)]
    return Xp, Xm, Phi, Gam, s, uL, uR


def _nonlinear(R, L, z, e, prm):
    """Equality residuals, Theta and Psi at z, in the assembly's row order."""
    Xp, Xm, Phi, Gam, s, uL, uR = _unpack(L, z)
    eq, th = [], []
    for k in range(L.N + 1):
        g, t = oracle.node_value(R, Xp[k], Xm[k], Phi[k], Gam[k], DELTA, e)
        eq.append(g)
        th.append(t)
        if k < L.N:
            eq.append(oracle.flow(R, NSUB, Xp[k], uL[k], uR[k], s[k]) - Xm[k + 1])
    eq.append(Xm[0, :L.nx] - prm["x_init"])
    eq.append(Xp[L.N, :L.nx] - prm["x_final"])
    psi = oracle.psi(R, Xp, Xm, DELTA, EPS)["psi"] if L.nc else np.zeros((L.N, 0))
    return np.concatenate(eq), th, psi


def _theta_psi_rows(L):
    """Row indices (in G) of the Theta rows of each node and Psi rows of each interval."""
    th, ps = [], []
    r = 0
    nlin = 2 * L.nj + (1 if L.aux else 4) * L.nc
    for k in range(L.N + 1):
        th.append(np.arange(r, r + 8 * L.nc))
        r += 16 * L.nc + 2 * L.nxt + (nlin if L.node else 0)
        if k < L.N:
            ps.append(np.arange(r, r + L.npsi))
            r += 2 * L.npsi + 2 * L.nxt + 2 + (0 if L.node else 2 * nlin)
    return th, ps


def _zhat(out, z):
    zh = np.zeros_like(z)
    L = out["layout"]
    zh[L.is_problem] = ((z - out["o"]) / out["D"])[L.is_problem]
    return zh


@pytest.mark.parametrize("name,cross,layout", [("hopper", False, "node"), ("hopper", True, "interval"),
                                               ("biped", False, "interval"), ("biped", True, "node")])
def test_residuals_at_and_near_the_iterate(name, cross, layout):
    R, out, e, prm = _case(name, cross, layout)
    L = out["layout"]
    th_rows, ps_rows = _theta_psi_rows(L)

    def gap(z):
        zh = _zhat(out, z)
        eq, th, psi = _nonlinear(R, L, z, e, prm)
        ge = out["A"] @ zh - out["b"] - out["rho_A"] * eq
        gz = out["G"] @ zh - out["h"]
        gt = [gz[rows] - out["rho_G"][rows] * th[k] for k, rows in enumerate(th_rows)]
        gp = [gz[rows] - out["rho_G"][rows] * psi[k] for k, rows in enumerate(ps_rows)]
        return np.abs(np.concatenate([ge] + gt + gp)).max()

    z0 = out["zbar"]
    assert gap(z0) <= 1e-11
    rng = np.random.default_rng(9)
    d = np.where(L.is_problem, rng.standard_normal(L.n_var), 0.0)
    g1, g2 = gap(z0 + 1e-3 * d), gap(z0 + 5e-4 * d)
    assert g1 > 1e-9
    assert 3.0 < g1 / g2 < 5.0


@pytest.mark.parametrize("cross,layout", [(False, "node"), (True, "node"), (True, "interval")])
def test_input_rows_and_friction_cones(cross, layout):
    R, out, e, prm = _case("biped", cross, layout)
    L = out["layout"]
    lin_rows = np.array([np.all(out["G"][r, ~L.is_problem] == 0) and np.any(out["G"][r] != 0)
                         for r in range(out["n_nonneg"])])
    z = out["zbar"].copy()
    for _, _, ucols in L.controls():
        z[ucols[:L.nj]] = 0.5 * prm["torque_max"]
        for i in range(L.nc):
            a, b, c = L.contact_inputs(ucols, i)
            if cross:   # phi_t, phi_n, gamma inside the cone
                z[a], z[b], z[c] = 0.3 * L.mu[i], 1.0, 0.2
            else:       # lambda_n, lambda_t+, lambda_t-
                z[a], z[b], z[c] = 1.0, 0.2 * L.mu[i], 0.1 * L.mu[i]
    for k in range(L.N):
        z[L.col["s", k]] = 0.5 * (prm["s_min"] + prm["s_max"])
    slack = out["h"] - out["G"] @ _zhat(out, z)
    assert np.all(slack[: out["n_nonneg"]][lin_rows] >= -1e-12)
    for q in range(out["n_soc"]):
        s0, s1 = slack[out["n_nonneg"] + 2 * q: out["n_nonneg"] + 2 * q + 2]
        assert s0 >= abs(s1)
    # one torque beyond its bound: exactly one input row turns negative
    _, _, ucols = L.controls()[1]
    z2 = z.copy()
    z2[ucols[0]] = -1.5 * prm["torque_max"][0]
    sl2 = (out["h"] - out["G"] @ _zhat(out, z2))[: out["n_nonneg"]][lin_rows]
    assert (sl2 < -1e-12).sum() == 1
    if cross:   # a tangential force outside the cone leaves its Q^2 block
        i = 0
        a, b, _ = L.contact_inputs(ucols, i)
        z3 = z.copy()
        z3[a] = 1.2 * L.mu[i] * z3[b]
        sl3 = out["h"] - out["G"] @ _zhat(out, z3)
        blocks = [sl3[out["n_nonneg"] + 2 * q: out["n_nonneg"] + 2 * q + 2] for q in range(out["n_soc"])]
        assert sum(bl[0] < abs(bl[1]) for bl in blocks) == 1


@pytest.mark.parametrize("cross", [False, True])
def test_rows_normalized(cross):
    R, out, e, prm = _case("hopper", cross, "node")
    L = out["layout"]
    for M, rho in ((out["A"], out["rho_A"]), (out["G"][: out["n_nonneg"]], out["rho_G"][: out["n_nonneg"]])):
        mx = np.abs(M[:, L.is_problem]).max(axis=1)
        has = mx > 0
        np.testing.assert_allclose(mx[has], 1.0, rtol=1e-14)
        np.testing.assert_array_equal(rho[~has], 1.0)
    for q in range(out["n_soc"]):
        blk = out["G"][out["n_nonneg"] + 2 * q: out["n_nonneg"] + 2 * q + 2][:, L.is_problem]
        assert np.abs(blk).max() == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("layout", ["node", "interval"])
def test_objective_definition(layout):
    R, out, e, prm = _case("biped", True, layout)
    L = out["layout"]
    rng = np.random.default_rng(4)

    def f_hat(z):
        zh = _zhat(out, z)
        zh[~L.is_problem] = z[~L.is_problem]
        return 0.5 * zh @ out["P"] @ zh + out["c"] @ zh

    def f_def(z):
        p = L.is_problem
        val = 0.5 * prm["w_px"] * np.sum((z[p] - out["zbar"][p]) ** 2)
        for k in range(L.N):
            a, b = z[L.uL(k)[:L.nj]], z[L.uR(k)[:L.nj]]
            sq = lambda t: np.sum(((1 - t) * a + t * b) ** 2)  # noqa: E731
            val += prm["w_torque"] * (sq(0.0) + 4 * sq(0.5) + sq(1.0)) / 6
        return val + prm["w_ep"] * np.sum(z[~p])

    z1 = out["zbar"] + rng.standard_normal(L.n_var)
    z2 = out["zbar"] + rng.standard_normal(L.n_var)
    z1[~L.is_problem] = np.abs(z1[~L.is_problem])
    z2[~L.is_problem] = np.abs(z2[~L.is_problem])
    assert f_hat(z1) - f_hat(z2) == pytest.approx(f_def(z1) - f_def(z2), rel=1e-11)


@pytest.mark.parametrize("cross,layout", [(False, "interval"), (True, "node")])
def test_slacks_absorb_the_violation(cross, layout):
    """At the iterate, nu+ - nu- = the nonlinear residual closes every equality
    row, and t = max(Theta, 0), max(Psi, 0) leaves min(value, 0) in its row."""
    R, out, e, prm = _case("hopper", cross, layout)
    L = out["layout"]
    z = out["zbar"].copy()
    Xp, Xm, Phi, Gam, s, uL, uR = _unpack(L, z)
    for k in range(L.N + 1):
        g, th = oracle.node_value(R, Xp[k], Xm[k], Phi[k], Gam[k], DELTA, e)
        z[L.col["nuGp", k]] = np.maximum(g, 0)
        z[L.col["nuGm", k]] = np.maximum(-g, 0)
        z[L.col["tth", k]] = np.maximum(th, 0)
        if k < L.N:
            r = oracle.flow(R, NSUB, Xp[k], uL[k], uR[k], s[k]) - Xm[k + 1]
            z[L.col["nuFp", k]] = np.maximum(r, 0)
            z[L.col["nuFm", k]] = np.maximum(-r, 0)
    psi = oracle.psi(R, Xp, Xm, DELTA, EPS)["psi"]
    for k in range(L.N):
        z[L.col["tpsi", k]] = np.maximum(psi[k], 0)
    zh = _zhat(out, z)
    zh[~L.is_problem] = z[~L.is_problem]
    eq = out["A"] @ zh - out["b"]
    nb_rows = len(eq) - 2 * L.nx
    assert np.abs(eq[:nb_rows]).max() <= 1e-11
    th_rows, ps_rows = _theta_psi_rows(L)
    gz = out["G"] @ zh - out["h"]
    for k, rows in enumerate(th_rows):
        _, th = oracle.node_value(R, Xp[k], Xm[k], Phi[k], Gam[k], DELTA, e)
        np.testing.assert_allclose(gz[rows], out["rho_G"][rows] * np.minimum(th, 0), atol=1e-11)
    for k, rows in enumerate(ps_rows):
        np.testing.assert_allclose(gz[rows], out["rho_G"][rows] * np.minimum(psi[k], 0), atol=1e-11)
