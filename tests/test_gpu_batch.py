"""GPU parity of the batched heterogeneous form (ciscvx_batch_*) against the oracle.

Small mixed batches are checked instance by instance in full under every launch
shape (persistent / one warp per item, cost / instance order, with and without
the CUDA graph) and after autotuning.  The full-size workloads — 1024 mixed
instances and the 4096 x 400 x 20 sweep — are checked on sampled instances and
intervals the oracle computes one by one.  Tolerances as in the single-instance
tests.
"""
import numpy as np
import pytest

from _util import TOL_FP32_PHI, TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu

TUNES = [
    None,
    {"warps_per_cta": 4, "ctas_per_sm": 0, "lpt_order": 1, "use_graph": 0, "occupancy": 0},
    {"warps_per_cta": 1, "ctas_per_sm": 8, "lpt_order": 0, "use_graph": 1, "occupancy": 0},
    {"warps_per_cta": 8, "ctas_per_sm": 1, "lpt_order": 1, "use_graph": 0, "occupancy": 0},
    {"warps_per_cta": 4, "ctas_per_sm": 3, "lpt_order": 1, "use_graph": 1, "occupancy": 1},
    {"warps_per_cta": 2, "ctas_per_sm": 0, "lpt_order": 1, "use_graph": 0, "occupancy": 2},
    {"warps_per_cta": 4, "ctas_per_sm": 3, "lpt_order": 2, "use_graph": 1, "occupancy": 1},
]

# The fused pass's autotuner candidates (warps per CTA, CTAs per SM, item
# order, graph, register-cap variant), as the library lists them: every
# launch shape the tuner can pick is run by the parity tests below, and the
# full-size test asserts that its pick is one of them.
FUSED_CANDIDATES = [
    (4, 2, 1, 0, 0, 0), (8, 1, 1, 0, 0, 0), (2, 4, 1, 0, 0, 0), (1, 8, 1, 0, 0, 0), (4, 0, 1, 0, 0, 0),
    (4, 2, 0, 0, 0, 0), (4, 3, 1, 0, 1, 0), (2, 6, 1, 0, 1, 0), (4, 4, 1, 0, 2, 0), (2, 8, 1, 0, 2, 0),
    (4, 0, 1, 0, 1, 0), (4, 0, 1, 0, 2, 0),
    # SM-partitioned foot-link / other-link queues
    (4, 3, 2, 0, 1, 0), (4, 2, 2, 0, 0, 0), (4, 4, 2, 0, 2, 0),
    # split form (linearization and adjoint of an item on two warps), small batches
    (1, 0, 1, 0, 0, 1), (2, 0, 1, 0, 0, 1), (4, 0, 1, 0, 0, 1),
]
_TUNE_KEYS = ("warps_per_cta", "ctas_per_sm", "lpt_order", "use_graph", "occupancy", "split")


def _tune_dict(c):
    return dict(zip(_TUNE_KEYS, c))


def _tune_tuple(t):
    return tuple(int(t.get(k, 0)) for k in _TUNE_KEYS)


# oracle results are independent of the launch shape: computed once per input set
_ORACLE_CACHE = {}


def _oracle_refs(oracle, key, probs, layout="node"):
    if (key, layout) not in _ORACLE_CACHE:
        refs = []
        for p in probs:
            Ui = p.U if layout == "node" else p.U_interval()
            R = p.robot.as_dict()
            refs.append((oracle.discretize(R, p.X, Ui, p.s, p.n_sub, layout=layout),
                         oracle.vjp(R, p.X, Ui, p.s, p.w, p.rho, p.n_sub, layout=layout)))
        _ORACLE_CACHE[(key, layout)] = refs
    return _ORACLE_CACHE[(key, layout)]


@pytest.fixture(scope="module")
def env():
    import torch
    import oracle
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return torch, oracle, api


def _small_mixed(seed=3, n=24):
    rng = np.random.default_rng(seed)
    robots = [synth.hopper(rng), synth.biped(rng), synth.cheetah7(rng)]
    styles = [dict(q_noise=0.05, u_dist="uniform"), dict(q_noise=0.1, u_dist="normal"),
              dict(q_noise=0.1, u_dist="normal")]
    probs, midx = [], []
    for i in range(n):
        m = int(rng.integers(0, 3))
        N = int(rng.integers(1, 71))
        ns = int(rng.choice([1, 3, 5]))
        probs.append(synth.draw_instance(robots[m], rng, N, ns, s_range=(0.05, 0.15),
                                         with_cotangents=True, **styles[m]))
        midx.append(m)
    return robots, probs, midx


def _packed(plan, probs, dev, torch, layout="node"):
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(plan.pack([p.X for p in probs], "X"))
    U = t(plan.pack([p.U if layout == "node" else p.U_interval() for p in probs], "U"))
    s = t(plan.pack([p.s for p in probs], "s"))
    w = t(plan.pack([p.w for p in probs], "defect"))
    rho = t(plan.pack([p.rho for p in probs], "penalty"))
    return X, U, s, w, rho


def _check_instance(plan, out, i, p, ref, precision):
    nxt, nu, nc, N = p.robot.nxt, p.robot.nu, p.robot.nc, p.N
    shapes = {"A": ("A", (N, nxt, nxt)), "Bm": ("B", (N, nxt, nu)), "Bp": ("B", (N, nxt, nu)),
              "S": ("S", (N, nxt)), "defect": ("defect", (N, nxt)), "penalty": ("penalty", (N, nc))}
    tol_phi = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for k, (okey, shape) in shapes.items():
        got = plan.unpack(out[k], okey, i, shape)
        tol = tol_phi if k in ("A", "Bm", "Bp", "S") else TOL_FP64
        e = block_err(got, ref[k])
        assert e <= tol, (i, k, e)


@pytest.mark.parametrize("tune", TUNES)
@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_small_mixed_batch_discretize(env, tune, precision):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _small_mixed()
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision=precision, tune=tune)
    X, U, s, _, _ = _packed(plan, probs, dev, torch)
    out = plan.discretize(X, U, s)
    out = plan.discretize(X, U, s, out=out)  # replay (graph path when enabled)
    plan.sync_status()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    for i, p in enumerate(probs):
        ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
        _check_instance(plan, host, i, p, ref, precision)


@pytest.mark.parametrize("layout", ["node", "interval"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_phi", 1e-4)])
def test_small_mixed_batch_vjp(env, layout, precision, tol):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _small_mixed(seed=5)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision=precision, layout=layout)
    X, U, s, w, rho = _packed(plan, probs, dev, torch, layout)
    g = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    gX, gU, gs, L = (g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L"))
    for i, p in enumerate(probs):
        Ui = p.U if layout == "node" else p.U_interval()
        rX, rU, rs, rL = oracle.vjp(p.robot.as_dict(), p.X, Ui, p.s, p.w, p.rho, p.n_sub, layout=layout)
        assert block_err(plan.unpack(gX, "X", i, rX.shape), rX) <= tol, i
        assert block_err(plan.unpack(gU, "U", i, rU.shape), rU) <= tol, i
        assert block_err(plan.unpack(gs, "s", i, rs.shape), rs) <= tol, i
        assert abs(L[i] - rL) <= tol * max(1.0, abs(rL)), i


def test_autotune_keeps_results(env):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _small_mixed(seed=8, n=40)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision="fp32_phi")
    X, U, s, _, _ = _packed(plan, probs, dev, torch)
    chosen = plan.autotune(X, U, s)
    assert chosen["warps_per_cta"] in (1, 2, 4, 8) and chosen["ctas_per_sm"] >= 0
    plan2 = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                          precision="fp32_phi")
    assert plan2.autotune(X, U, s) == chosen  # cached per process
    out = plan.discretize(X, U, s)
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    for i in (0, 7, 19, 39):
        p = probs[i]
        _check_instance(plan, host, i, p, oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub),
                        "fp32_phi")


def test_batch_errors(env):
    torch, oracle, api = env
    robots, probs, midx = _small_mixed(n=3)
    models = [api.Model(r) for r in robots]
    with pytest.raises(api.CiscvxError) as e:
        api.BatchPlan(models, [0, 5, 1], [2, 2, 2], [1, 1, 1])
    assert e.value.status == api.EINVAL
    with pytest.raises(api.CiscvxError) as e:
        api.BatchPlan(models, [0, 1, 2], [2, 0, 2], [1, 1, 1])
    assert e.value.status == api.EINVAL
    with pytest.raises(api.CiscvxError) as e:
        api.BatchPlan(models, [0, 1, 2], [2, 2, 2], [1, 1, 1], precision="bf16_tc")
    assert e.value.status == api.EUNSUPPORTED
    plan = api.BatchPlan(models, [0, 1, 2], [2, 2, 2], [1, 65, 1])
    dev = torch.device("cuda:0")
    z = torch.zeros(1024, dtype=torch.float64, device=dev)
    with pytest.raises(api.CiscvxError) as e:
        plan.discretize_vjp(z, z, z, z, z)
    assert e.value.status == api.EUNSUPPORTED


def test_mixed_1024_sampled(env):
    """1024 instances, hopper:biped:chain = 1:1:2, N ~ U{10..200}, n_sub in {4,8,16}, FP32 Phi."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    b = synth.mixed_batch(seed=0)
    probs = [b.instance(i) for i in range(len(b))]
    models = [api.Model(r) for r in b.robots]
    plan = api.BatchPlan(models, b.model_idx, b.Ns, b.n_subs, precision="fp32_phi")
    X, U, s, w, rho = _packed(plan, probs, dev, torch)
    plan.autotune(X, U, s)
    out = plan.discretize(X, U, s)
    g = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    gX, gU, gs, L = (g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L"))
    rng = np.random.default_rng(1)
    for i in sorted(rng.choice(len(b), 12, replace=False)):
        p = probs[i]
        R = p.robot.as_dict()
        _check_instance(plan, host, i, p, oracle.discretize(R, p.X, p.U, p.s, p.n_sub), "fp32_phi")
        rX, rU, rs, rL = oracle.vjp(R, p.X, p.U, p.s, p.w, p.rho, p.n_sub)
        assert block_err(plan.unpack(gX, "X", i, rX.shape), rX) <= 1e-4
        assert block_err(plan.unpack(gU, "U", i, rU.shape), rU) <= 1e-4
        assert block_err(plan.unpack(gs, "s", i, rs.shape), rs) <= 1e-4
        assert abs(L[i] - rL) <= 1e-4 * max(1.0, abs(rL))


@pytest.fixture(scope="module")
def sweep(env):
    """The 4096 x 400 x 20 sweep packed on the device, with the oracle's
    results for the sampled intervals (8 random instances plus the first and
    the last, 8 intervals each) and three instances' whole VJPs."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    b = synth.cheetah_sweep(seed=0)
    model = api.Model(b.robots[0])
    plan = api.BatchPlan([model], b.model_idx, b.Ns, b.n_subs, precision="fp32_phi")
    probs = [b.instance(i) for i in range(len(b))]
    X, U, s, w, rho = _packed(plan, probs, dev, torch)
    rng = np.random.default_rng(2)
    inst = sorted(rng.choice(len(b), 8, replace=False)) + [0, len(b) - 1]
    R = b.robots[0].as_dict()
    samples = []
    for i in inst:
        p = probs[i]
        for k in sorted(set(rng.choice(p.N, 6, replace=False).tolist() + [0, p.N - 1])):
            x1, A, Bm, Bp, S = oracle.interval(R, p.n_sub, p.X[k], p.U[k], p.U[k + 1], p.s[k])
            samples.append((i, k, A, Bm, Bp, S, x1 - p.X[k + 1]))
    vjps = {}
    for i in (0, 1234, 4095):
        p = probs[i]
        vjps[i] = oracle.vjp(R, p.X, p.U, p.s, p.w, p.rho, p.n_sub, threads=0)
    return dict(b=b, model=model, plan=plan, inputs=(X, U, s, w, rho), samples=samples, vjps=vjps)


def _check_sweep_samples(plan, out, sw):
    b = sw["b"]
    nxt, nu = b.robots[0].nxt, b.robots[0].nu
    for i, k, A, Bm, Bp, S, dref in sw["samples"]:
        o = plan.offsets[i]
        a0 = o["A"] + k * nxt * nxt
        b0 = o["B"] + k * nxt * nu
        v0 = o["S"] + k * nxt
        assert block_err(out["A"][a0:a0 + nxt * nxt].double().cpu().numpy(), A.ravel()) <= TOL_FP32_PHI
        assert block_err(out["Bm"][b0:b0 + nxt * nu].double().cpu().numpy(), Bm.ravel()) <= TOL_FP32_PHI
        assert block_err(out["Bp"][b0:b0 + nxt * nu].double().cpu().numpy(), Bp.ravel()) <= TOL_FP32_PHI
        assert block_err(out["S"][v0:v0 + nxt].double().cpu().numpy(), S) <= TOL_FP32_PHI
        d = out["defect"][v0:v0 + nxt].cpu().numpy()
        assert block_err(d, dref) <= TOL_FP64


def _check_sweep_vjps(plan, g, sw):
    gX, gU, gs, L = (g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L"))
    for i, (rX, rU, rs, rL) in sw["vjps"].items():
        assert block_err(plan.unpack(gX, "X", i, rX.shape), rX) <= 1e-4
        assert block_err(plan.unpack(gU, "U", i, rU.shape), rU) <= 1e-4
        assert block_err(plan.unpack(gs, "s", i, rs.shape), rs) <= 1e-4
        assert abs(L[i] - rL) <= 1e-4 * max(1.0, abs(rL))


def test_sweep_4096x400x20_sampled(env, sweep):
    """The 4096-instance sweep at full size (FP32 Phi), separate calls: sampled
    intervals checked one by one, three instances' VJPs checked whole; a graph
    replay reproduces the outputs bit for bit."""
    torch, oracle, api = env
    plan = sweep["plan"]
    X, U, s, w, rho = sweep["inputs"]
    nxt = sweep["b"].robots[0].nxt
    out = plan.discretize(X, U, s)
    torch.cuda.synchronize()
    _check_sweep_samples(plan, out, sweep)
    # replay reproduces bit for bit
    d0 = out["defect"].clone()
    a0 = out["A"][: 10 * nxt * nxt].clone()
    plan.discretize(X, U, s, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out["defect"], d0) and torch.equal(out["A"][: 10 * nxt * nxt], a0)
    del out
    g = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    _check_sweep_vjps(plan, g, sweep)
    del g
    torch.cuda.empty_cache()


@pytest.mark.parametrize("shape", ["autotune", (4, 2, 1, 0, 0), (4, 4, 1, 0, 2), (4, 3, 1, 0, 1), (4, 3, 2, 0, 1)],
                         ids=["autotuned", "occ0", "occ2", "occ1", "occ1-smqueues"])
def test_sweep_fused_pass_full_size_sampled(env, sweep, shape):
    """The fused pass (ciscvx_batch_discretize_and_vjp, the bench's step) on the
    full 4096 x 400 x 20 sweep under the autotuner's pick and under each
    register-cap variant: the same sampled intervals and instance VJPs against
    the oracle.  The autotuner's pick is one of the candidates the small-batch
    test runs one by one."""
    torch, oracle, api = env
    b = sweep["b"]
    X, U, s, w, rho = sweep["inputs"]
    if shape == "autotune":
        plan = sweep["plan"]
        ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=X.device)
        out = plan.alloc_outputs(X.device)
        pick = plan.autotune_fused(X, U, s, w, rho, workspace=ws, out=out)
        assert _tune_tuple(pick) in FUSED_CANDIDATES, pick
        assert _tune_tuple(plan.tune_fused()) == _tune_tuple(pick)
    else:
        plan = api.BatchPlan([sweep["model"]], b.model_idx, b.Ns, b.n_subs, precision="fp32_phi",
                             tune=_tune_dict(shape))
        assert plan.tune_fused()["occupancy"] == shape[4]
        ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=X.device)
        out = plan.alloc_outputs(X.device)
    out, g = plan.discretize_and_vjp(X, U, s, w, rho, workspace=ws, out=out)
    plan.sync_status()
    _check_sweep_samples(plan, out, sweep)
    _check_sweep_vjps(plan, g, sweep)
    del out, g, ws
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n_chunks", [1, 3, 24])
@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_run_host_pipelined_matches_device_path(env, n_chunks, precision):
    """ciscvx_batch_run_host on pinned host buffers gives the device path's outputs.

    Chunking regroups which intervals share a warp, and the warp votes on the
    Taylor tier of the angle chain, so the two agree to rounding (FP64 values
    within 1e-12 of each other, FP32 blocks within 1e-6), not bit for bit;
    with one chunk the decomposition is the same and they are identical."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _small_mixed(seed=11)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision=precision)
    X, U, s, w, rho = _packed(plan, probs, dev, torch)
    ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=dev)
    ref, gref = plan.discretize_and_vjp(X, U, s, w, rho, workspace=ws)  # the pass run_host runs per chunk
    torch.cuda.synchronize()
    pin = lambda t: t.cpu().pin_memory()  # noqa: E731
    host_in = {"X": pin(X), "U": pin(U), "s": pin(s)}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in ref.items()}
    host_vjp = {"w": pin(w), "rho": pin(rho)}
    host_vjp.update({k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in gref.items()})
    dev_in = {k: torch.empty_like(v) for k, v in (("X", X), ("U", U), ("s", s))}
    dev_out = {k: torch.empty_like(v) for k, v in ref.items()}
    dev_vjp = {"w": torch.empty_like(w), "rho": torch.empty_like(rho)}
    dev_vjp.update({k: torch.empty_like(v) for k, v in gref.items()})
    for _ in range(2):  # second call reuses the chunk tables
        for v in host_out.values():
            v.fill_(float("nan"))
        plan.run_host(host_in, host_out, dev_in, dev_out, n_chunks=n_chunks, host_vjp=host_vjp,
                      dev_vjp=dev_vjp, workspace=ws)
        torch.cuda.current_stream().synchronize()
        plan.sync_status()
        for k, v in list(ref.items()) + list(gref.items()):
            got = (host_out if k in host_out else host_vjp)[k]
            if n_chunks == 1:
                assert torch.equal(got, v.cpu()), k
            else:
                tol = 1e-6 if v.dtype == torch.float32 else 1e-12
                assert not torch.isnan(got).any(), k
                assert block_err(got.double().numpy(), v.double().cpu().numpy()) <= tol, k


def test_sweep_precision_report_16_instances(env, capsys):
    """Per-block maximum relative error of A_k, B-_k, B+_k, S_k (and defect,
    penalty) against the FP64 oracle on the first 16 instances of the sweep
    (400 intervals x 20 substeps each), every interval checked, for the FP64
    and the FP32-Phi paths.  Two measures per block: block-normwise
    max_k max|dX_k| / max|X_k|, and elementwise max |dX| / max(|X|, 1e-12 max|X_k|)."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    b = synth.cheetah_sweep(seed=0, n_inst=16)
    probs = [b.instance(i) for i in range(len(b))]
    model = api.Model(b.robots[0])
    R = b.robots[0].as_dict()
    refs = [oracle.discretize(R, p.X, p.U, p.s, p.n_sub, threads=0) for p in probs]
    report = {}
    for precision in ("fp64", "fp32_phi"):
        plan = api.BatchPlan([model], b.model_idx, b.Ns, b.n_subs, precision=precision)
        X, U, s, _, _ = _packed(plan, probs, dev, torch)
        out = {k: v.double().cpu().numpy() for k, v in plan.discretize(X, U, s).items()}
        rows = {}
        for key, okey in (("A", "A"), ("Bm", "B"), ("Bp", "B"), ("S", "S"), ("defect", "defect"),
                          ("penalty", "penalty")):
            bw, ew = 0.0, 0.0
            for i, p in enumerate(probs):
                ref = refs[i][key]
                got = plan.unpack(out[key], okey, i, ref.shape)
                for k in range(p.N):
                    r, g = ref[k], got[k]
                    sc = np.abs(r).max()
                    if sc == 0.0:
                        continue
                    d = np.abs(g - r)
                    bw = max(bw, d.max() / sc)
                    ew = max(ew, (d / np.maximum(np.abs(r), 1e-12 * sc)).max())
            rows[key] = (bw, ew)
        report[precision] = rows
    with capsys.disabled():
        print("\nper-block max relative error vs FP64 oracle, 16 x 400 x 20 sweep subset")
        for precision, rows in report.items():
            print(precision, " ".join(f"{k}: block {v[0]:.2e} elem {v[1]:.2e}" for k, v in rows.items()))
    for k, (bw, _) in report["fp64"].items():
        assert bw <= TOL_FP64, (k, bw)
    for k, (bw, _) in report["fp32_phi"].items():
        assert bw <= (TOL_FP32_PHI if k in ("A", "Bm", "Bp", "S") else TOL_FP64), (k, bw)


def _fused_check(env, precision, out_format, layout, tune):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _small_mixed(seed=13, n=18)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision=precision, layout=layout, out_format=out_format, tune=tune)
    if tune is not None:
        assert _tune_tuple(plan.tune_fused())[:3] == _tune_tuple(tune)[:3]
        assert plan.tune_fused()["occupancy"] == tune["occupancy"]
        assert plan.tune_fused()["split"] == tune.get("split", 0)
    X, U, s, w, rho = _packed(plan, probs, dev, torch, layout)
    out, g = plan.discretize_and_vjp(X, U, s, w, rho)
    sep = plan.discretize(X, U, s)
    gsep = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    f32 = precision == "fp32_phi"
    for k in ("A", "Bm", "Bp", "S"):
        e = block_err(out[k].double().cpu().numpy(), sep[k].double().cpu().numpy())
        assert e <= (1e-5 if f32 else 1e-13), (k, e)
    for k in ("defect", "penalty"):
        assert block_err(out[k].cpu().numpy(), sep[k].cpu().numpy()) <= 1e-13, k
    for k in ("gX", "gU", "gs", "L"):
        e = block_err(g[k].cpu().numpy(), gsep[k].cpu().numpy())
        assert e <= (1e-5 if f32 else 1e-12), (k, e)
    tol = 1e-4 if f32 else 1e-10
    refs = _oracle_refs(oracle, ("small_mixed", 13, 18), probs, layout)
    gX, gU, gs, L = (g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L"))
    for i, p in enumerate(probs):
        rX, rU, rs, rL = refs[i][1]
        assert block_err(plan.unpack(gX, "X", i, rX.shape), rX) <= tol, i
        assert block_err(plan.unpack(gU, "U", i, rU.shape), rU) <= tol, i
        assert block_err(plan.unpack(gs, "s", i, rs.shape), rs) <= tol, i
        assert abs(L[i] - rL) <= tol * max(1.0, abs(rL)), i
    if out_format == "dense":
        host = {k: v.double().cpu().numpy() for k, v in out.items()}
        for i, p in enumerate(probs):
            _check_instance(plan, host, i, p, refs[i][0], precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("out_format", ["dense", "compact"])
@pytest.mark.parametrize("layout", ["node", "interval"])
def test_fused_pass_matches_separate_calls_and_oracle(env, precision, out_format, layout):
    """ciscvx_batch_discretize_and_vjp: the linearization and the VJP from one
    pass equal the separate calls to rounding, and the oracle to the usual
    tolerances."""
    _fused_check(env, precision, out_format, layout, None)


@pytest.mark.parametrize("cand", FUSED_CANDIDATES, ids=lambda c: "w%d-c%d-l%d-g%d-occ%d-split%d" % c)
@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("out_format", ["dense", "compact"])
def test_fused_pass_every_tuner_candidate(env, cand, precision, out_format):
    """The fused pass under every launch shape its autotuner can pick, in
    particular each register-cap variant (occupancy 0: uncapped, 1: at most
    168 registers, 2: at most 128 registers, the one the tuner picks for the
    4096 x 400 x 20 sweep), against the separate calls and the oracle."""
    _fused_check(env, precision, out_format, "node", _tune_dict(cand))


def test_autotune_fused_keeps_results(env):
    """The fused pass's autotuner picks a valid launch shape and the results
    under it match the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _small_mixed(seed=21, n=16)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [p.N for p in probs], [p.n_sub for p in probs],
                         precision="fp32_phi")
    X, U, s, w, rho = _packed(plan, probs, dev, torch)
    t = plan.autotune_fused(X, U, s, w, rho)
    assert t == plan.tune_fused() and t["warps_per_cta"] in (1, 2, 4, 8)
    out, g = plan.discretize_and_vjp(X, U, s, w, rho)
    plan.sync_status()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    gX, gU, gs, L = (g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L"))
    for i, p in enumerate(probs):
        ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
        _check_instance(plan, host, i, p, ref, "fp32_phi")
        rX, rU, rs, rL = oracle.vjp(p.robot.as_dict(), p.X, p.U, p.s, p.w, p.rho, p.n_sub)
        assert block_err(plan.unpack(gX, "X", i, rX.shape), rX) <= 1e-4
        assert block_err(plan.unpack(gU, "U", i, rU.shape), rU) <= 1e-4
        assert abs(L[i] - rL) <= 1e-4 * max(1.0, abs(rL))


@pytest.mark.parametrize("robot,N,n_sub", [("hopper", 1, 4), ("hopper", 10, 4), ("cheetah7", 50, 10),
                                             ("cheetah7", 100, 10)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_single_instance_step_split_and_autotuned(env, robot, N, n_sub, precision):
    """The single-instance configurations (hopper N = 10 with 4 substeps, the
    7-link chain at N = 50 and 100 with 10 substeps, and N = 1) through a
    one-instance plan's discretize_and_vjp, as the bench times them: under
    each split-form launch shape, and under the fused autotuner's pick (which
    must come from the candidate list), against the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    make = synth.hopper_fp64 if robot == "hopper" else synth.cheetah_n50
    p = make(seed=5, N=N, n_sub=n_sub)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, sv, w, rho = t(p.X), t(p.U), t(p.s), t(p.w), t(p.rho)
    ref = oracle.discretize(p.robot.as_dict(), p.X, p.U, p.s, p.n_sub)
    rX, rU, rs, rL = oracle.vjp(p.robot.as_dict(), p.X, p.U, p.s, p.w, p.rho, p.n_sub)
    tol = TOL_FP32_PHI if precision == "fp32_phi" else TOL_FP64
    shapes = [c for c in FUSED_CANDIDATES if c[5] == 1] + ["autotune"]
    for shape in shapes:
        if shape == "autotune":
            plan = api.BatchPlan([m], [0], [N], [n_sub], precision=precision)
            ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=dev)
            pick = plan.autotune_fused(X, U, sv, w, rho, workspace=ws)
            assert _tune_tuple(pick) in FUSED_CANDIDATES, pick
        else:
            plan = api.BatchPlan([m], [0], [N], [n_sub], precision=precision, tune=_tune_dict(shape))
            assert plan.tune_fused()["split"] == 1
            ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=dev)
        out, g = plan.discretize_and_vjp(X, U, sv, w, rho, workspace=ws)
        plan.sync_status()
        host = {k: v.double().cpu().numpy() for k, v in out.items()}
        _check_instance(plan, host, 0, p, ref, precision)
        gX, gU, gs, L = (g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L"))
        assert block_err(plan.unpack(gX, "X", 0, rX.shape), rX) <= tol, shape
        assert block_err(plan.unpack(gU, "U", 0, rU.shape), rU) <= tol, shape
        assert block_err(plan.unpack(gs, "s", 0, rs.shape), rs) <= tol, shape
        assert abs(L[0] - rL) <= tol * max(1.0, abs(rL)), shape


_TUNE_SCRIPT = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_2604_09993_gb300 import api, synth
rng = np.random.default_rng(3)
R = synth.hopper(rng)
probs = [synth.draw_instance(R, rng, 20, 4, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15)) for _ in range(5)]
m = api.Model(R)
plan = api.BatchPlan([m], [0] * 5, [q.N for q in probs], [q.n_sub for q in probs], precision="fp32_phi")
t = lambda a: torch.tensor(a, device="cuda:0")
X, U, s = t(plan.pack([q.X for q in probs], "X")), t(plan.pack([q.U for q in probs], "U")), t(plan.pack([q.s for q in probs], "s"))
print(json.dumps(plan.autotune(X, U, s)))
"""


def test_tune_cache_file(env, tmp_path):
    """CISCVX_TUNE_CACHE: a process's autotune choice is written to the file,
    and the next process takes it from there instead of timing again (shown by
    planting a different valid choice in the file)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    envv = dict(os.environ, CISCVX_TUNE_CACHE=str(cache))
    script = _TUNE_SCRIPT.format(root=root)
    r1 = subprocess.run([sys.executable, "-c", script], env=envv, capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0, r1.stderr[-2000:]
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    key = lines[0].split("\t")[0]
    cache.write_text(f"{key}\t2 6 1 0 1\nnot a tune line\n")
    r2 = subprocess.run([sys.executable, "-c", script], env=envv, capture_output=True, text=True, timeout=300)
    assert r2.returncode == 0, r2.stderr[-2000:]
    t2 = json.loads(r2.stdout.strip().splitlines()[-1])
    assert (t2["warps_per_cta"], t2["ctas_per_sm"], t2["lpt_order"], t2["occupancy"]) == (2, 6, 1, 1)
    assert len(cache.read_text().splitlines()) == 2   # nothing re-timed, nothing appended
