"""GPU parity of the compact outputs (ciscvx_discretize_compact and batch plans
with CISCVX_OUT_COMPACT) through the C ABI.

Compact A/B-/B+ hold the structural nonzeros in ciscvx_model_pattern's order.
They are checked two ways: scattered into dense blocks against the FP64 oracle
(same tolerances as the dense path), and against the dense path of the same
launch shape value by value.  The two kernels share their source but are
compiled separately, and the compiler may fuse a multiply and an add in one
and not in the other, so they agree to rounding (block-relative 1e-13 where
the values are FP64, 1e-5 for FP32 blocks), not necessarily bit for bit; the
dense path is exactly zero off the pattern.
"""
import numpy as np
import pytest

from _util import TOL_FP32_PHI, TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import oracle
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return torch, oracle, api


def _scatter(vals, rows, cols, shape):
    """Dense (N, *shape) blocks from compact (N, nnz) values."""
    out = np.zeros((vals.shape[0],) + shape)
    out[:, rows, cols] = vals
    return out


def _check_vs_oracle(got, ref, pat, nxt, nu, precision):
    ar, ac, br, bc = pat
    tol_phi = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    A = _scatter(got["A"], ar, ac, (nxt, nxt))
    Bm = _scatter(got["Bm"], br, bc, (nxt, nu))
    Bp = _scatter(got["Bp"], br, bc, (nxt, nu))
    for k, v in (("A", A), ("Bm", Bm), ("Bp", Bp), ("S", got["S"])):
        assert block_err(v, ref[k]) <= tol_phi, (k, block_err(v, ref[k]))
    for k in ("defect", "penalty"):
        assert block_err(got[k], ref[k]) <= TOL_FP64, k


def _close(a, b, what, fp32=False):
    """Compact vs dense values of the same launch: equal to rounding."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    assert block_err(a, b) <= (1e-5 if fp32 else 1e-13), (what, block_err(a, b))


def _single(env, p, precision, layout="node", want_z=False):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    U = p.U if layout == "node" else p.U_interval()
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, Ut, s = t(p.X), t(U), t(p.s)
    c = api.discretize_compact(m, X, Ut, s, p.n_sub, precision, layout, want_z=want_z)
    d = api.discretize(m, X, Ut, s, p.n_sub, precision, layout, want_z=want_z)
    api.sync_status(m)
    c = {k: v.cpu() for k, v in c.items()}
    d = {k: v.cpu() for k, v in d.items()}
    return m, U, c, d


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("case", ["hopper", "cheetah_n50", "biped_interval", "biped_cross",
                                  "cheetah7_cross_interval"])
def test_single_compact_vs_oracle_and_dense(env, precision, case):
    torch, oracle, api = env
    layout = "node"
    if case == "hopper":
        p = synth.hopper_fp64()
    elif case == "cheetah_n50":
        p = synth.cheetah_n50(seed=1)
    elif case.endswith("_cross") or case.endswith("_cross_interval"):
        # the Eq. (12) auxiliary state (four cross-complementarity rows per contact)
        rng = np.random.default_rng(10)
        robot = synth.with_cross_states(getattr(synth, case.split("_")[0])(rng))
        p = synth.draw_instance(robot, rng, 41, 3, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15))
        layout = "interval" if case.endswith("_interval") else "node"
    else:
        rng = np.random.default_rng(8)
        robot = synth.biped(rng)
        p = synth.draw_instance(robot, rng, 45, 3, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15))
        layout = "interval"
    m, U, c, d = _single(env, p, precision, layout)
    ar, ac, br, bc = m.pattern()
    assert c["A"].shape == (p.N, m.nnz_a) and c["Bm"].shape == (p.N, m.nnz_b)
    # equal to the dense path at the pattern, and the dense path is zero elsewhere
    f32 = precision == "fp32_phi"
    _close(c["A"], d["A"][:, ar, ac], "A", f32)
    _close(c["Bm"], d["Bm"][:, br, bc], "Bm", f32)
    _close(c["Bp"], d["Bp"][:, br, bc], "Bp", f32)
    _close(c["S"], d["S"], "S", f32)
    for k in ("defect", "penalty"):
        _close(c[k], d[k], k)
    maskA = torch.ones(d["A"].shape[1:], dtype=torch.bool)
    maskA[ar, ac] = False
    maskB = torch.ones(d["Bm"].shape[1:], dtype=torch.bool)
    maskB[br, bc] = False
    assert torch.all(d["A"][:, maskA] == 0) and torch.all(d["Bm"][:, maskB] == 0)
    assert torch.all(d["Bp"][:, maskB] == 0)
    ref = oracle.discretize(p.robot.as_dict(), p.X, U, p.s, p.n_sub, layout=layout)
    got = {k: v.double().numpy() for k, v in c.items()}
    _check_vs_oracle(got, ref, (ar, ac, br, bc), m.nxt, m.nu, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_compact_affine_term(env, precision):
    """z from the compact call matches z from the dense call."""
    torch, oracle, api = env
    p = synth.cheetah_n50(seed=2, N=37, n_sub=4)
    m, U, c, d = _single(env, p, precision, want_z=True)
    _close(c["z"], d["z"], "z", precision == "fp32_phi")
    if precision == "fp64":
        ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
        x1 = ref["defect"] + p.X[1:]
        z = x1 - np.einsum("kij,kj->ki", ref["A"], p.X[:-1]) - np.einsum("kij,kj->ki", ref["Bm"], p.U[:-1]) \
            - np.einsum("kij,kj->ki", ref["Bp"], p.U[1:]) - ref["S"] * p.s[:, None]
        assert block_err(c["z"].numpy(), z) <= 1e-10


@pytest.mark.parametrize("which", ["no_contact", "lone_link"])
def test_compact_edge_models(env, which):
    """n_c = 0 and n_u = 0 (nnz_B = 0: Bm/Bp may be null)."""
    from test_gpu_discretize import _edge_robots
    torch, oracle, api = env
    R = _edge_robots()[which]
    m = api.Model(R)
    rng = np.random.default_rng(4)
    N, n_sub = 33, 2
    X = rng.uniform(-0.5, 0.5, (N + 1, m.nxt))
    U = rng.standard_normal((N + 1, m.nu))
    s = rng.uniform(0.05, 0.15, N)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    c = api.discretize_compact(m, t(X), t(U), t(s), n_sub, "fp64")
    api.sync_status(m)
    got = {k: v.cpu().numpy() for k, v in c.items()}
    ref = oracle.discretize(R, X, U, s, n_sub)
    _check_vs_oracle(got, ref, m.pattern(), m.nxt, m.nu, "fp64")
    if which == "lone_link":
        assert m.nnz_b == 0


def test_compact_argument_errors(env):
    torch, oracle, api = env
    p = synth.hopper_fp64()
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    X, U, s = (torch.tensor(a, device=dev) for a in (p.X, p.U, p.s))
    out = {"A": torch.empty((p.N, m.nnz_a), dtype=torch.float64, device=dev),
           "Bm": torch.empty((p.N, m.nnz_b), dtype=torch.float64, device=dev),
           "Bp": torch.empty((p.N, m.nnz_b), dtype=torch.float64, device=dev),
           "S": torch.empty((p.N, m.nxt), dtype=torch.float64, device=dev),
           "defect": torch.empty((p.N, m.nxt), dtype=torch.float64, device=dev),
           "penalty": torch.empty((p.N, m.nc), dtype=torch.float64, device=dev)}
    lib = api.load()
    ptr = lambda t: t.data_ptr()  # noqa: E731
    st = lib.ciscvx_discretize_compact(m.handle, p.N, p.n_sub, 0, 0, ptr(X), ptr(U), ptr(s),
                                       ptr(out["A"]), None, ptr(out["Bp"]), ptr(out["S"]),
                                       ptr(out["defect"]), ptr(out["penalty"]), None, None, 0, None)
    assert st == api.EINVAL
    st = lib.ciscvx_discretize_compact(m.handle, p.N, p.n_sub, 3, 0, ptr(X), ptr(U), ptr(s),
                                       ptr(out["A"]), ptr(out["Bm"]), ptr(out["Bp"]), ptr(out["S"]),
                                       ptr(out["defect"]), ptr(out["penalty"]), None, None, 0, None)
    assert st == api.EUNSUPPORTED
    with pytest.raises(KeyError):
        api.BatchPlan([m], [0], [p.N], [p.n_sub], out_format="sparse")


def _mixed(seed=7, n=20):
    rng = np.random.default_rng(seed)
    robots = [synth.hopper(rng), synth.biped(rng), synth.cheetah7(rng)]
    probs, midx = [], []
    for _ in range(n):
        mi = int(rng.integers(0, 3))
        N = int(rng.integers(1, 60))
        ns = int(rng.choice([1, 2, 5]))
        probs.append(synth.draw_instance(robots[mi], rng, N, ns, q_noise=0.1, u_dist="normal",
                                         s_range=(0.05, 0.15)))
        midx.append(mi)
    return robots, probs, midx


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("tune", [None, {"warps_per_cta": 2, "ctas_per_sm": 0, "lpt_order": 0,
                                         "use_graph": 0, "occupancy": 1}])
def test_batch_compact_vs_dense_and_oracle(env, precision, tune):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _mixed()
    models = [api.Model(r) for r in robots]
    Ns, nss = [p.N for p in probs], [p.n_sub for p in probs]
    pc = api.BatchPlan(models, midx, Ns, nss, precision=precision, tune=tune, out_format="compact")
    pd = api.BatchPlan(models, midx, Ns, nss, precision=precision, tune=tune)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(pc.pack([p.X for p in probs], "X"))
    U = t(pc.pack([p.U for p in probs], "U"))
    s = t(pc.pack([p.s for p in probs], "s"))
    assert pc.sizes["A"] == sum(p.N * models[mi].nnz_a for p, mi in zip(probs, midx))
    assert pc.sizes["B"] == sum(p.N * models[mi].nnz_b for p, mi in zip(probs, midx))
    oc = pc.discretize(X, U, s)
    oc = pc.discretize(X, U, s, out=oc)
    od = pd.discretize(X, U, s)
    pc.sync_status()
    pd.sync_status()
    hc = {k: v.cpu() for k, v in oc.items()}
    hd = {k: v.cpu() for k, v in od.items()}
    f32 = precision == "fp32_phi"
    _close(hc["S"], hd["S"], "S", f32)
    for k in ("defect", "penalty"):
        _close(hc[k], hd[k], k)
    pats = [m.pattern() for m in models]
    for i, (p, mi) in enumerate(zip(probs, midx)):
        m = models[mi]
        ar, ac, br, bc = pats[mi]
        N, nxt, nu = p.N, m.nxt, m.nu
        cA = pc.unpack(hc["A"], "A", i, (N, m.nnz_a))
        cBm = pc.unpack(hc["Bm"], "B", i, (N, m.nnz_b))
        cBp = pc.unpack(hc["Bp"], "B", i, (N, m.nnz_b))
        dA = pd.unpack(hd["A"], "A", i, (N, nxt, nxt))
        dBm = pd.unpack(hd["Bm"], "B", i, (N, nxt, nu))
        dBp = pd.unpack(hd["Bp"], "B", i, (N, nxt, nu))
        _close(cA, dA[:, ar, ac], ("A", i), f32)
        _close(cBm, dBm[:, br, bc], ("Bm", i), f32)
        _close(cBp, dBp[:, br, bc], ("Bp", i), f32)
        ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
        f = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
        got = {"A": f(cA), "Bm": f(cBm), "Bp": f(cBp), "S": f(pc.unpack(hc["S"], "S", i, (N, nxt))),
               "defect": f(pc.unpack(hc["defect"], "defect", i, (N, nxt))),
               "penalty": f(pc.unpack(hc["penalty"], "penalty", i, (N, m.nc)))}
        _check_vs_oracle(got, ref, pats[mi], nxt, nu, precision)


def test_batch_compact_run_host_one_chunk_identical(env):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _mixed(seed=9, n=12)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision="fp32_phi", out_format="compact")
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(plan.pack([p.X for p in probs], "X"))
    U = t(plan.pack([p.U for p in probs], "U"))
    s = t(plan.pack([p.s for p in probs], "s"))
    ref = plan.discretize(X, U, s)
    torch.cuda.synchronize()
    pin = lambda a: a.cpu().pin_memory()  # noqa: E731
    host_in = {"X": pin(X), "U": pin(U), "s": pin(s)}
    host_out = {k: torch.full(v.shape, float("nan"), dtype=v.dtype).pin_memory() for k, v in ref.items()}
    dev_in = {k: torch.empty_like(v) for k, v in (("X", X), ("U", U), ("s", s))}
    dev_out = {k: torch.empty_like(v) for k, v in ref.items()}
    plan.run_host(host_in, host_out, dev_in, dev_out, n_chunks=1)
    torch.cuda.current_stream().synchronize()
    plan.sync_status()
    for k, v in ref.items():
        assert torch.equal(host_out[k], v.cpu()), k


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_batch_compact_both_aux_models(env, precision):
    """A compact batch mixing both auxiliary models: against the dense plan at
    the pattern and against the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(33)
    robots = [synth.hopper(rng), synth.with_cross_states(synth.biped(rng)),
              synth.with_cross_states(synth.cheetah7(rng))]
    probs, midx = [], []
    for i in range(10):
        mi = i % 3
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 50)), int(rng.choice([2, 4])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15)))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    Ns, nss = [p.N for p in probs], [p.n_sub for p in probs]
    pc = api.BatchPlan(models, midx, Ns, nss, precision=precision, out_format="compact")
    pd = api.BatchPlan(models, midx, Ns, nss, precision=precision)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(pc.pack([p.X for p in probs], "X"))
    U = t(pc.pack([p.U for p in probs], "U"))
    s = t(pc.pack([p.s for p in probs], "s"))
    hc = {k: v.cpu() for k, v in pc.discretize(X, U, s).items()}
    hd = {k: v.cpu() for k, v in pd.discretize(X, U, s).items()}
    pc.sync_status()
    pd.sync_status()
    f32 = precision == "fp32_phi"
    for i, (p, mi) in enumerate(zip(probs, midx)):
        m = models[mi]
        ar, ac, br, bc = m.pattern()
        N, nxt, nu = p.N, m.nxt, m.nu
        cA = pc.unpack(hc["A"], "A", i, (N, m.nnz_a))
        cBm = pc.unpack(hc["Bm"], "B", i, (N, m.nnz_b))
        cBp = pc.unpack(hc["Bp"], "B", i, (N, m.nnz_b))
        dA = pd.unpack(hd["A"], "A", i, (N, nxt, nxt))
        dBm = pd.unpack(hd["Bm"], "B", i, (N, nxt, nu))
        _close(cA, dA[:, ar, ac], ("A", i), f32)
        _close(cBm, dBm[:, br, bc], ("Bm", i), f32)
        ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
        f = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
        got = {"A": f(cA), "Bm": f(cBm), "Bp": f(cBp), "S": f(pc.unpack(hc["S"], "S", i, (N, nxt))),
               "defect": f(pc.unpack(hc["defect"], "defect", i, (N, nxt))),
               "penalty": f(pc.unpack(hc["penalty"], "penalty", i, (N, m.nc)))}
        _check_vs_oracle(got, ref, (ar, ac, br, bc), nxt, nu, precision)
