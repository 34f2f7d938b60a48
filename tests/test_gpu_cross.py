"""GPU parity of the full Eq. (12) auxiliary state (CISCVX_AUX_CROSS) against
the FP64 oracle through the C ABI: single-instance and batched linearization,
both precisions and both control layouts, mixed batches of the two auxiliary
models, feasible inputs, the reverse-mode adjoint VJP (against the oracle's
Phi-contracted gradient and against central differences), and the affine term
z formed from the dense and from the compact outputs.
Tolerances as for the default model (FP64 1e-10; FP32-Phi blocks 1e-4,
defect and penalty 1e-10)."""
import numpy as np
import pytest

from _util import TOL_FP32_PHI, TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu

PHI = ("A", "Bm", "Bp", "S")
STATE = ("defect", "penalty")


@pytest.fixture(scope="module")
def env():
    import torch
    import oracle
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return torch, oracle, api


def _check(got, ref, precision):
    tol = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for k in PHI:
        assert block_err(got[k], ref[k]) <= tol, (k, block_err(got[k], ref[k]))
    for k in STATE:
        assert block_err(got[k], ref[k]) <= TOL_FP64, (k, block_err(got[k], ref[k]))


def _problem(name, seed, N, n_sub, feasible=False):
    rng = np.random.default_rng(seed)
    R = synth.with_cross_states(getattr(synth, name)(rng))
    p = synth.draw_instance(R, rng, N, n_sub, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15))
    if feasible:
        U = p.U.copy()
        for i in range(R.nc):
            c0 = 3 * R.nj + 3 * i
            U[:, c0 + 1] = rng.uniform(1.0, 2.0, p.N + 1)
            U[:, c0] = rng.uniform(-0.3, 0.3, p.N + 1) * R.contact_mu[i] * U[:, c0 + 1]
            U[:, c0 + 2] = rng.uniform(0.1, 0.5, p.N + 1)
        X = p.X.copy()
        X[:, 1:3 * R.nb:3] += 3.0  # every link far above the ground
        p = synth.Problem(R, p.N, p.n_sub, X, U, p.s, None, None)
    return p


def _single(env, p, precision, layout="node"):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    assert (m.ny, m.nc) == (5 * p.robot.nc, p.robot.nc)
    U = p.U if layout == "node" else p.U_interval()
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.discretize(m, t(p.X), t(U), t(p.s), p.n_sub, precision, layout)
    api.sync_status(m)
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    ref = oracle.discretize(p.robot.as_dict(), p.X, U, p.s, p.n_sub, layout=layout)
    return got, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("name,N,n_sub", [("hopper", 10, 4), ("biped", 45, 3), ("cheetah7", 50, 10)])
def test_cross_single_matches_oracle(env, precision, name, N, n_sub):
    got, ref = _single(env, _problem(name, 11, N, n_sub), precision)
    _check(got, ref, precision)


def test_cross_interval_layout(env):
    p = _problem("biped", 12, 37, 5)
    got, ref = _single(env, p, "fp64", layout="interval")
    _check(got, ref, "fp64")


def test_cross_feasible_inputs_leave_penalty_zero(env):
    p = _problem("cheetah7", 13, 33, 4, feasible=True)
    got, ref = _single(env, p, "fp64")
    _check(got, ref, "fp64")
    assert np.all(got["penalty"] == 0.0)
    pen = slice(6 * p.robot.nb + 4 * p.robot.nc, p.robot.nxt)
    assert not np.any(got["Bm"][:, pen]) and not np.any(got["S"][:, pen])


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_cross_batch_mixed_models(env, precision):
    """A batch holding both auxiliary models (and a robot without contacts)."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(14)
    robots = [synth.hopper(rng), synth.with_cross_states(synth.biped(rng)),
              synth.with_cross_states(synth.cheetah7(rng)), synth.cheetah7(rng)]
    probs, midx = [], []
    for _ in range(14):
        mi = int(rng.integers(0, len(robots)))
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 50)), int(rng.choice([1, 3])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15)))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs], precision=precision)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(plan.pack([p.X for p in probs], "X"))
    U = t(plan.pack([p.U for p in probs], "U"))
    s = t(plan.pack([p.s for p in probs], "s"))
    out = plan.discretize(X, U, s)
    plan.sync_status()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    for i, p in enumerate(probs):
        R = p.robot
        N, nxt, nu, nc = p.N, R.nxt, R.nu, R.nc
        got = {"A": plan.unpack(host["A"], "A", i, (N, nxt, nxt)),
               "Bm": plan.unpack(host["Bm"], "B", i, (N, nxt, nu)),
               "Bp": plan.unpack(host["Bp"], "B", i, (N, nxt, nu)),
               "S": plan.unpack(host["S"], "S", i, (N, nxt)),
               "defect": plan.unpack(host["defect"], "defect", i, (N, nxt)),
               "penalty": plan.unpack(host["penalty"], "penalty", i, (N, nc))}
        ref = oracle.discretize(R.as_dict(), p.X, p.U, p.s, p.n_sub)
        _check(got, ref, precision)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("layout", ["node", "interval"])
def test_cross_affine_term_with_compact_outputs(env, precision, tol, layout):
    """z with compact outputs (a post-pass over the structural nonzeros by
    rows) equals z from the oracle's blocks, and the compact values equal the
    dense outputs at the pattern's positions."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("biped", 15, 41, 3)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    U = p.U if layout == "node" else p.U_interval()
    got = api.discretize_compact(m, t(p.X), t(U), t(p.s), p.n_sub, precision, layout, want_z=True)
    dense = api.discretize(m, t(p.X), t(U), t(p.s), p.n_sub, precision, layout, want_z=True)
    api.sync_status(m)
    ref = oracle.discretize(p.robot.as_dict(), p.X, U, p.s, p.n_sub, layout=layout)
    uL = U[:-1] if layout == "node" else U[:, 0]
    uR = U[1:] if layout == "node" else U[:, 1]
    z = ref["defect"] + p.X[1:] - np.einsum("kij,kj->ki", ref["A"], p.X[:-1]) \
        - np.einsum("kij,kj->ki", ref["Bm"], uL) - np.einsum("kij,kj->ki", ref["Bp"], uR) \
        - ref["S"] * p.s[:, None]
    zg = got["z"].cpu().numpy()
    for k in range(p.N):
        assert block_err(zg[k], z[k]) <= tol, k
    # same blocks in both formats, hence the same z up to the summation order
    assert block_err(zg, dense["z"].cpu().numpy()) <= 1e-12
    ar, ac, br, bc = m.pattern()
    Ad = dense["A"].double().cpu().numpy()
    assert np.array_equal(got["A"].double().cpu().numpy(), Ad[:, ar, ac])


def test_cross_node_constraints(env):
    """The node kernel's auxiliary-state continuity rows cover all 5 n_c states."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(16)
    R = synth.with_cross_states(synth.cheetah7(rng)).as_dict()
    m = api.Model(R)
    n = 40
    Xm = rng.uniform(-1, 1, (n, m.nxt))
    Xp = Xm + 0.3 * rng.standard_normal((n, m.nxt))
    Phi = rng.standard_normal((n, 2 * m.nc))
    Gam = rng.uniform(0, 1, (n, m.nc))
    e = np.full(m.nc, 0.4)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.node_linearize(m, t(Xp), t(Xm), t(Phi), t(Gam), 1e-3, e)
    api.sync_status(m)
    ref = oracle.node(R, Xp, Xm, Phi, Gam, 1e-3, e)
    assert block_err(out["g"].cpu().numpy(), ref["g"]) <= TOL_FP64
    assert block_err(out["theta"].cpu().numpy().reshape(n, -1), ref["theta"]) <= TOL_FP64


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("layout", ["node", "interval"])
def test_cross_vjp_matches_oracle(env, precision, tol, layout):
    """The reverse-mode adjoint of this model against the oracle's
    Phi-contracted gradient; its scratch is the default model's (the per-link
    partial sums), one size whatever n_sub and the precision."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("biped", 17, 75, 3)
    rng = np.random.default_rng(18)
    m = api.Model(p.robot)
    w = rng.standard_normal((p.N, m.nxt))
    rho = np.full((p.N, m.nc), 10.0)
    U = p.U if layout == "node" else p.U_interval()
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    lo, hi = api.discretize_workspace_size(m, p.N, p.n_sub, precision, api.OP_VJP, layout)
    assert lo == hi == api.workspace_size(m, api.OP_VJP, p.N, layout)
    ws = torch.empty(lo, dtype=torch.uint8, device=dev)
    gX, gU, gs, L = api.discretize_vjp(m, t(p.X), t(U), t(p.s), t(w), t(rho), p.n_sub, precision,
                                       layout, workspace=ws)
    api.sync_status(m)
    rX, rU, rs, rL = oracle.vjp(p.robot.as_dict(), p.X, U, p.s, w, rho, p.n_sub, layout=layout)
    for g, r, nm in ((gX, rX, "gX"), (gU, rU, "gU"), (gs, rs, "gs")):
        assert block_err(g.cpu().numpy(), r) <= tol, (nm, block_err(g.cpu().numpy(), r))
    assert abs(L.item() - rL) <= TOL_FP64 * max(1.0, abs(rL))


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("out_format", ["dense", "compact"])
def test_cross_fused_pass_in_mixed_batch(env, precision, tol, out_format):
    """ciscvx_batch_discretize_and_vjp on a batch mixing the Eq. (12) model with
    the default one: the fused pass (the Eq. (12) foot links record their
    checkpoints and quadratures, and the adjoint starts from them) against the
    two separate calls (to rounding) and the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(71)
    robots = [synth.with_cross_states(synth.biped(rng)), synth.hopper(rng),
              synth.with_cross_states(synth.cheetah7(rng))]
    probs, midx = [], []
    for i in range(8):
        mi = i % 3
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 50)), int(rng.choice([1, 3, 5])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15), with_cotangents=True))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision,
                         out_format=out_format)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, s = (t(plan.pack([getattr(q, k) for q in probs], k)) for k in ("X", "U", "s"))
    w = t(plan.pack([q.w for q in probs], "defect"))
    rho = t(plan.pack([q.rho for q in probs], "penalty"))
    ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=dev)
    plan.autotune_fused(X, U, s, w, rho, workspace=ws)
    out, g = plan.discretize_and_vjp(X, U, s, w, rho, workspace=ws)
    out = {k: v.clone() for k, v in out.items()}
    g = {k: v.clone() for k, v in g.items()}
    out2 = plan.discretize(X, U, s)
    g2 = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    f32 = precision == "fp32_phi"
    for k in out:
        e = block_err(out[k].double().cpu().numpy(), out2[k].double().cpu().numpy())
        assert e <= (1e-5 if f32 and k in PHI else 1e-13), (k, e)
    for k in ("gX", "gU", "gs", "L"):
        e = block_err(g[k].cpu().numpy(), g2[k].cpu().numpy())
        assert e <= (1e-5 if f32 else 1e-12), (k, e)
    host = {k: v.cpu().numpy() for k, v in g.items()}
    for i, q in enumerate(probs):
        rX, rU, rs, rL = oracle.vjp(q.robot.as_dict(), q.X, q.U, q.s, q.w, q.rho, q.n_sub)
        assert block_err(plan.unpack(host["gX"], "X", i, q.X.shape), rX) <= tol, i
        assert block_err(plan.unpack(host["gU"], "U", i, q.U.shape), rU) <= tol, i
        assert block_err(plan.unpack(host["gs"], "s", i, q.s.shape), rs) <= tol, i
        assert abs(host["L"][i] - rL) <= TOL_FP64 * max(1.0, abs(rL)), i


def test_cross_vjp_central_differences(env):
    """The adjoint's gradient of L = sum_k w_k . defect_k + rho_k . penalty_k
    against central differences (h = 1e-6) of the oracle's flow map, every
    entry of X, U and s, on a two-interval Eq. (12) biped."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("biped", 21, 2, 3)
    rng = np.random.default_rng(22)
    R = p.robot.as_dict()
    m = api.Model(p.robot)
    nxt, nc = m.nxt, m.nc
    w = rng.standard_normal((p.N, nxt))
    rho = np.full((p.N, nc), 10.0)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    got = api.discretize_vjp(m, t(p.X), t(p.U), t(p.s), t(w), t(rho), p.n_sub, "fp64")
    api.sync_status(m)
    got = [g.cpu().numpy() for g in got[:3]]
    pen = slice(nxt - nc, nxt)  # the path-penalty rows follow the four cross rows per contact

    def L(X, U, s):
        tot = 0.0
        for k in range(p.N):
            x1 = oracle.flow(R, p.n_sub, X[k], U[k], U[k + 1], s[k])
            tot += w[k] @ (x1 - X[k + 1]) + rho[k] @ (x1[pen] - X[k, pen])
        return tot

    e = 1e-6
    X, U, s = p.X.copy(), p.U.copy(), p.s.copy()
    for arr, g in ((X, got[0]), (U, got[1]), (s, got[2])):
        flat, gf = arr.reshape(-1), g.reshape(-1)
        for i in range(flat.size):
            v = flat[i]
            flat[i] = v + e; lp = L(X, U, s)
            flat[i] = v - e; lm = L(X, U, s)
            flat[i] = v
            fd = (lp - lm) / (2 * e)
            assert abs(fd - gf[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gf[i])


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
def test_cross_affine_term(env, precision, tol):
    """z_k = x~(1) - A x~_k - B- u_L - B+ u_R - S s_k, from the oracle's blocks."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("biped", 16, 37, 4)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    got = api.discretize(m, t(p.X), t(p.U), t(p.s), p.n_sub, precision, want_z=True)
    ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
    z = ref["defect"] + p.X[1:] - np.einsum("kij,kj->ki", ref["A"], p.X[:-1]) \
        - np.einsum("kij,kj->ki", ref["Bm"], p.U[:-1]) - np.einsum("kij,kj->ki", ref["Bp"], p.U[1:]) \
        - ref["S"] * p.s[:, None]
    zg = got["z"].cpu().numpy()
    for k in range(p.N):
        assert block_err(zg[k], z[k]) <= tol
