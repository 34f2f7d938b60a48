"""GPU parity of the coupled-links path (joint reaction forces eliminated by
Eq. (3), the sinusoidal contact surface of Sec. VI-B, the RKF45 scheme)
against the FP64 oracle, through the C ABI.

Tolerances as for the per-link path: FP64 rel <= 1e-10 on every block
(block-normwise); FP32-Phi rel <= 1e-4 on A, B-, B+, S and rel <= 1e-10 on
defect and penalty; the reverse-mode adjoint VJP against the oracle's
Phi-contracted gradient at the same tolerances and against central
differences on a tiny case.  Sizes span several warps of
intervals, thread blocks of tangent columns and a ragged tail; a short
workspace forces several chunks.
"""
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


def _problem(name, seed, N, n_sub, cross=False, **kw):
    rng = np.random.default_rng(seed)
    R = synth.with_paper_dynamics(getattr(synth, name)(rng), **kw)
    if cross:
        R = synth.with_cross_states(R)
    return synth.draw_instance(R, rng, N, n_sub, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15))


def _run(env, p, precision, layout="node", workspace=None):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    assert m.coupled
    U = p.U if layout == "node" else p.U_interval()
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.discretize(m, t(p.X), t(U), t(p.s), p.n_sub, precision, layout, workspace=workspace)
    api.sync_status(m)
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    ref = oracle.discretize(p.robot.as_dict(), p.X, U, p.s, p.n_sub, layout=layout)
    return got, ref


def _check(got, ref, precision):
    tol = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for k in PHI:
        assert block_err(got[k], ref[k]) <= tol, (k, block_err(got[k], ref[k]))
    for k in STATE:
        assert block_err(got[k], ref[k]) <= TOL_FP64, (k, block_err(got[k], ref[k]))


PAPER = dict(joint_forces=1, scheme=1, terrain=synth.TERRAIN_SINE)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("name,N,n_sub", [("hopper", 10, 4), ("biped", 45, 3), ("cheetah7", 70, 5)])
def test_paper_dynamics_matches_oracle(env, precision, name, N, n_sub):
    got, ref = _run(env, _problem(name, 21, N, n_sub, **PAPER), precision)
    _check(got, ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("feature", [
    dict(joint_forces=1, scheme=0),                                  # Eq. (3) alone
    dict(joint_forces=0, scheme=0, terrain=synth.TERRAIN_SINE),      # surface alone
    dict(joint_forces=0, scheme=1),                                  # RKF45 alone
    dict(joint_forces=1, scheme=0, terrain=synth.TERRAIN_SINE),
], ids=["eliminated", "terrain", "rkf45", "eliminated+terrain"])
def test_each_feature_matches_oracle(env, precision, feature):
    got, ref = _run(env, _problem("cheetah7", 22, 37, 4, **feature), precision)
    _check(got, ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_full_eq12_state_with_paper_dynamics(env, precision):
    got, ref = _run(env, _problem("biped", 23, 40, 3, cross=True, **PAPER), precision)
    _check(got, ref, precision)


def test_interval_layout(env):
    got, ref = _run(env, _problem("biped", 24, 33, 3, **PAPER), "fp64", layout="interval")
    _check(got, ref, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_chunked_workspace_is_bitwise_equal(env, precision):
    """A workspace of the minimum size (32 intervals per chunk) gives the very
    same numbers as one chunk for all intervals."""
    torch, oracle, api = env
    p = _problem("cheetah7", 25, 101, 3, **PAPER)
    m = api.Model(p.robot)
    lo, hi = api.discretize_workspace_size(m, p.N, p.n_sub, precision)
    assert 0 < lo < hi
    dev = torch.device("cuda:0")
    small = torch.empty(lo, dtype=torch.uint8, device=dev)
    full = torch.empty(hi, dtype=torch.uint8, device=dev)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    a = api.discretize(m, t(p.X), t(p.U), t(p.s), p.n_sub, precision, workspace=small)
    b = api.discretize(m, t(p.X), t(p.U), t(p.s), p.n_sub, precision, workspace=full)
    api.sync_status(m)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_single_interval_and_no_contacts(env):
    """Degenerate sizes: N = 1, n_sub = 1; a robot without contacts (no y rows)."""
    p = _problem("hopper", 26, 1, 1, **PAPER)
    got, ref = _run(env, p, "fp64")
    _check(got, ref, "fp64")
    rng = np.random.default_rng(27)
    R = synth.with_paper_dynamics(synth.biped(rng), **PAPER)
    R = synth.Robot(**{**R.__dict__, "contact_body": np.zeros(0, np.int32),
                       "contact_rho": np.zeros((0, 2)), "contact_mu": np.zeros(0)})
    q = synth.draw_instance(R, rng, 5, 2, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15))
    got, ref = _run(env, q, "fp64")
    for k in ("A", "Bm", "Bp", "S", "defect"):
        assert block_err(got[k], ref[k]) <= TOL_FP64, k


def test_short_workspace_is_an_argument_error(env):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("hopper", 28, 10, 4, **PAPER)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, s = t(p.X), t(p.U), t(p.s)
    tiny = torch.empty(16, dtype=torch.uint8, device=dev)
    for call in (lambda: api.discretize(m, X, U, s, p.n_sub, "fp64", workspace=tiny),
                 lambda: api.discretize_compact(m, X, U, s, p.n_sub, "fp64", workspace=tiny)):
        with pytest.raises(api.CiscvxError) as err:
            call()
        assert err.value.status == api.EINVAL


COMPACT_CASES = [("hopper", 70, 3, dict(PAPER), False), ("cheetah7", 45, 2, dict(PAPER), True),
                 ("biped", 33, 2, dict(joint_forces=0, scheme=0, terrain=synth.TERRAIN_SINE), False),
                 ("biped", 40, 3, dict(joint_forces=1, scheme=0), True)]


def _compact_check(env, p, precision, layout):
    """Compact A, B-, B+ against the dense blocks of the same call: every
    pattern entry bit for bit, every entry off the pattern exactly zero; S,
    defect and penalty identical; z from the compact values against z from the
    dense ones (the same sums in another order)."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    U = p.U if layout == "node" else p.U_interval()
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, Ut, s = t(p.X), t(U), t(p.s)
    dense = api.discretize(m, X, Ut, s, p.n_sub, precision, layout, want_z=True)
    comp = api.discretize_compact(m, X, Ut, s, p.n_sub, precision, layout, want_z=True)
    api.sync_status(m)
    ar, ac, br, bc = (torch.tensor(a.astype(np.int64), device=dev) for a in m.pattern())
    nxt, nu = m.nxt, m.nu
    assert comp["A"].shape[1] == len(ar) < nxt * nxt and comp["Bm"].shape[1] == len(br) == nxt * nu
    assert torch.equal(comp["A"], dense["A"][:, ar, ac])
    for k in ("Bm", "Bp"):
        assert torch.equal(comp[k], dense[k][:, br, bc]), k
    off = torch.ones(nxt, nxt, dtype=torch.bool, device=dev)
    off[ar, ac] = False
    assert not torch.any(dense["A"][:, off] != 0)
    for k in ("S", "defect", "penalty"):
        assert torch.equal(comp[k], dense[k]), k
    assert block_err(comp["z"].cpu().numpy(), dense["z"].cpu().numpy()) <= 1e-12
    ref = oracle.discretize(p.robot.as_dict(), p.X, U, p.s, p.n_sub, layout=layout)
    got = {k: v.double().cpu().numpy() for k, v in dense.items()}
    _check(got, ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("case", range(len(COMPACT_CASES)))
def test_compact_outputs_match_dense_and_oracle(env, precision, case):
    name, N, n_sub, kw, cross = COMPACT_CASES[case]
    p = _problem(name, 40 + case, N, n_sub, cross=cross, **kw)
    _compact_check(env, p, precision, "node" if case % 2 == 0 else "interval")


def test_compact_outputs_specialized_and_generic_kernels(env, monkeypatch):
    """The generic coupled kernels (CISCVX_COUPLED_JIT=0) write the same
    compact layout as the run-time specialized ones."""
    p = _problem("biped", 52, 37, 2, cross=True, **PAPER)
    monkeypatch.setenv("CISCVX_COUPLED_JIT", "0")
    _compact_check(env, p, "fp32_phi", "node")
    monkeypatch.delenv("CISCVX_COUPLED_JIT")


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_batch_plan_compact_with_coupled_models(env, precision):
    """A compact batch plan mixing per-link and coupled models: every
    instance's compact values equal the single-instance compact call's (to
    rounding: intervals are grouped differently into warps, and the angle
    chain's Taylor tier is a warp vote), and the plan's graph replays them."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(53)
    robots = [synth.hopper(rng),
              synth.with_paper_dynamics(synth.biped(rng), **PAPER),
              synth.with_cross_states(synth.with_paper_dynamics(synth.cheetah7(rng), joint_forces=1, scheme=0))]
    probs, midx = [], []
    for i in range(9):
        mi = i % 3
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 50)), int(rng.choice([1, 3])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15)))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision,
                         out_format="compact")
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(plan.pack([q.X for q in probs], "X"))
    U = t(plan.pack([q.U for q in probs], "U"))
    sv = t(plan.pack([q.s for q in probs], "s"))
    out = plan.discretize(X, U, sv)
    plan.sync_status()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    tol = 1e-12 if precision == "fp64" else 1e-6
    for i, q in enumerate(probs):
        m = models[midx[i]]
        c = api.discretize_compact(m, t(q.X), t(q.U), t(q.s), q.n_sub, precision)
        api.sync_status(m)
        N, na, nb_ = q.N, m.nnz_a, m.nnz_b
        got = {"A": plan.unpack(host["A"], "A", i, (N, na)), "Bm": plan.unpack(host["Bm"], "B", i, (N, nb_)),
               "Bp": plan.unpack(host["Bp"], "B", i, (N, nb_)), "S": plan.unpack(host["S"], "S", i, (N, m.nxt)),
               "defect": plan.unpack(host["defect"], "defect", i, (N, m.nxt))}
        for k, v in got.items():
            assert block_err(v, c[k].double().cpu().numpy()) <= tol, (i, k)
    out2 = plan.discretize(X, U, sv)
    plan.sync_status()
    for k in out:
        assert torch.equal(out[k], out2[k]), k


def test_node_constraints_with_eliminated_joint_forces(env):
    """The impulse model does not depend on how the continuous-time reaction
    forces are treated: on flat ground the node kernel serves these models."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(29)
    R = synth.with_paper_dynamics(synth.cheetah7(rng), joint_forces=1, scheme=1).as_dict()
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


def test_sweep_size_sampled(env):
    """At the benchmark's size and launch configuration (7-link chain, paper
    dynamics, 65 536 intervals x 10 substeps in 2 GiB chunks, FP32-Phi): sampled
    intervals against the oracle, and every defect finite."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = synth.cheetah_paper_sweep(seed=0)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.discretize(m, t(p.X), t(p.U), t(p.s), p.n_sub, "fp32_phi")
    api.sync_status(m)
    assert torch.isfinite(out["defect"]).all()
    rng = np.random.default_rng(1)
    ks = np.unique(np.concatenate([[0, p.N - 1], rng.integers(0, p.N, 14)]))
    for k in ks:
        ref = oracle.discretize(p.robot.as_dict(), p.X[k:k + 2], p.U[k:k + 2], p.s[k:k + 1], p.n_sub)
        got = {kk: v[k:k + 1].double().cpu().numpy() for kk, v in out.items()}
        _check(got, ref, "fp32_phi")


def _vjp(env, p, precision, layout="node", workspace=None):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(30)
    m = api.Model(p.robot)
    w = rng.standard_normal((p.N, m.nxt))
    rho = np.full((p.N, m.nc), 10.0)
    U = p.U if layout == "node" else p.U_interval()
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    got = api.discretize_vjp(m, t(p.X), t(U), t(p.s), t(w), t(rho), p.n_sub, precision, layout,
                             workspace=workspace)
    api.sync_status(m)
    ref = oracle.vjp(p.robot.as_dict(), p.X, U, p.s, w, rho, p.n_sub, layout=layout)
    return got, ref


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("layout", ["node", "interval"])
def test_vjp_matches_oracle(env, precision, tol, layout):
    p = _problem("cheetah7", 31, 45, 3, **PAPER)
    (gX, gU, gs, L), (rX, rU, rs, rL) = _vjp(env, p, precision, layout)
    for g, r, nm in ((gX, rX, "gX"), (gU, rU, "gU"), (gs, rs, "gs")):
        assert block_err(g.cpu().numpy(), r) <= tol, (nm, block_err(g.cpu().numpy(), r))
    assert abs(L.item() - rL) <= TOL_FP64 * max(1.0, abs(rL))


FEATURES = [
    dict(joint_forces=1, scheme=0),                                  # Eq. (3) alone
    dict(joint_forces=0, scheme=0, terrain=synth.TERRAIN_SINE),      # surface alone
    dict(joint_forces=0, scheme=1),                                  # RKF45 alone
    dict(joint_forces=1, scheme=0, terrain=synth.TERRAIN_SINE),
]
FEATURE_IDS = ["eliminated", "terrain", "rkf45", "eliminated+terrain"]


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("feature", FEATURES, ids=FEATURE_IDS)
def test_vjp_each_feature_matches_oracle(env, precision, tol, feature):
    """The reverse-mode adjoint under each modelling option alone and combined."""
    p = _problem("cheetah7", 35, 37, 4, **feature)
    (gX, gU, gs, L), (rX, rU, rs, rL) = _vjp(env, p, precision)
    for g, r, nm in ((gX, rX, "gX"), (gU, rU, "gU"), (gs, rs, "gs")):
        assert block_err(g.cpu().numpy(), r) <= tol, (nm, block_err(g.cpu().numpy(), r))
    assert abs(L.item() - rL) <= TOL_FP64 * max(1.0, abs(rL))


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("name,N,n_sub,cross", [("hopper", 10, 4, False), ("biped", 40, 3, True),
                                                ("hopper", 1, 1, True)])
def test_vjp_robots_and_eq12_state(env, precision, tol, name, N, n_sub, cross):
    """Other robots, the full Eq. (12) auxiliary state with the paper's dynamics,
    and the degenerate N = 1, n_sub = 1."""
    p = _problem(name, 36, N, n_sub, cross=cross, **PAPER)
    for layout in ("node", "interval"):
        (gX, gU, gs, L), (rX, rU, rs, rL) = _vjp(env, p, precision, layout)
        for g, r, nm in ((gX, rX, "gX"), (gU, rU, "gU"), (gs, rs, "gs")):
            assert block_err(g.cpu().numpy(), r) <= tol, (layout, nm, block_err(g.cpu().numpy(), r))
        assert abs(L.item() - rL) <= TOL_FP64 * max(1.0, abs(rL))


def test_vjp_central_differences(env):
    """The adjoint's gradient against central differences (h = 1e-6) of
    L = sum w . defect + rho . penalty, evaluated with the FP64 linearization
    of the same path, on a tiny case (hopper, N = 2, 2 RKF45 substeps)."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("hopper", 37, 2, 2, **PAPER)
    m = api.Model(p.robot)
    rng = np.random.default_rng(38)
    w = rng.standard_normal((p.N, m.nxt))
    rho = np.full((p.N, m.nc), 10.0)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    gX, gU, gs, L = api.discretize_vjp(m, t(p.X), t(p.U), t(p.s), t(w), t(rho), p.n_sub, "fp64")
    gX, gU, gs = gX.cpu().numpy(), gU.cpu().numpy(), gs.cpu().numpy()

    def Lval(X, U, s):
        o = api.discretize(m, t(X), t(U), t(s), p.n_sub, "fp64")
        return float((o["defect"].cpu().numpy() * w).sum() + (o["penalty"].cpu().numpy() * rho).sum())

    assert abs(Lval(p.X, p.U, p.s) - L.item()) <= 1e-12 * max(1.0, abs(L.item()))
    h = 1e-6
    for arr, g in ((p.X, gX), (p.U, gU), (p.s, gs)):
        fd = np.zeros(arr.size)
        for i in range(arr.size):
            a, b = arr.copy().ravel(), arr.copy().ravel()
            a[i] += h
            b[i] -= h
            args_a = [a.reshape(arr.shape) if x is arr else x for x in (p.X, p.U, p.s)]
            args_b = [b.reshape(arr.shape) if x is arr else x for x in (p.X, p.U, p.s)]
            fd[i] = (Lval(*args_a) - Lval(*args_b)) / (2 * h)
        assert block_err(g.ravel(), fd) <= 1e-6, block_err(g.ravel(), fd)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_phi", 1e-5)])
@pytest.mark.parametrize("scheme", [0, 1])
def test_specialized_and_generic_adjoint_kernels_agree(env, precision, tol, scheme, monkeypatch):
    """The run-time specialized adjoint (default) and the generic one
    (CISCVX_COUPLED_JIT=0) give the same gradient; both meet the oracle."""
    p = _problem("cheetah7", 39, 41, 3, joint_forces=1, scheme=scheme, terrain=synth.TERRAIN_SINE)
    a, ref = _vjp(env, p, precision)
    monkeypatch.setenv("CISCVX_COUPLED_JIT", "0")
    b, _ = _vjp(env, p, precision)
    monkeypatch.delenv("CISCVX_COUPLED_JIT")
    otol = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for ga, gb, r in zip(a[:3], b[:3], ref[:3]):
        ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
        assert block_err(ga, r) <= otol and block_err(gb, r) <= otol
        assert block_err(ga, gb) <= tol, block_err(ga, gb)


def test_vjp_chunking_is_bitwise_equal(env):
    """A minimum workspace (chunks of 32 intervals, node-shared sums carried
    across chunk boundaries) gives the same gradient as one chunk."""
    torch, oracle, api = env
    p = _problem("biped", 32, 77, 2, **PAPER)
    m = api.Model(p.robot)
    lo, hi = api.discretize_workspace_size(m, p.N, p.n_sub, "fp64", api.OP_VJP)
    dev = torch.device("cuda:0")
    a = _vjp(env, p, "fp64", workspace=torch.empty(lo, dtype=torch.uint8, device=dev))[0]
    b = _vjp(env, p, "fp64", workspace=torch.empty(hi, dtype=torch.uint8, device=dev))[0]
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    assert a[3].item() != 0.0


def test_autograd_through_the_coupled_path(env):
    """torch.autograd through discretize_fn: backward is the contracted VJP."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("hopper", 33, 12, 3, **PAPER)
    m = api.Model(p.robot)
    X = torch.tensor(p.X, device=dev, requires_grad=True)
    U = torch.tensor(p.U, device=dev, requires_grad=True)
    s = torch.tensor(p.s, device=dev, requires_grad=True)
    d, pen = api.discretize_fn(m, X, U, s, p.n_sub, "fp64")
    w = torch.randn_like(d)
    (d * w).sum().add((pen * 10.0).sum()).backward()
    rho = np.full((p.N, m.nc), 10.0)
    rX, rU, rs, _ = oracle.vjp(p.robot.as_dict(), p.X, p.U, p.s, w.cpu().numpy(), rho, p.n_sub)
    assert block_err(X.grad.cpu().numpy(), rX) <= TOL_FP64
    assert block_err(U.grad.cpu().numpy(), rU) <= TOL_FP64
    assert block_err(s.grad.cpu().numpy(), rs) <= TOL_FP64


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_phi", 1e-5)])
@pytest.mark.parametrize("scheme", [0, 1])
def test_specialized_and_generic_tangent_kernels_agree(env, precision, tol, scheme, monkeypatch):
    """The run-time specialized kernels (default) and the generic ones
    (CISCVX_COUPLED_JIT=0) compute the same blocks; both meet the oracle.
    The specialized nominal kernel chains sin/cos by angle addition and uses
    other roundings, so the FP64 state agrees to 1e-12, not bitwise."""
    torch, oracle, api = env
    p = _problem("cheetah7", 34, 41, 3, joint_forces=1, scheme=scheme, terrain=synth.TERRAIN_SINE)
    got_jit, ref = _run(env, p, precision)
    monkeypatch.setenv("CISCVX_COUPLED_JIT", "0")
    got_gen, _ = _run(env, p, precision)
    monkeypatch.delenv("CISCVX_COUPLED_JIT")
    _check(got_jit, ref, precision)
    _check(got_gen, ref, precision)
    for k in PHI:
        assert block_err(got_jit[k], got_gen[k]) <= tol, k
    for k in STATE:
        assert block_err(got_jit[k], got_gen[k]) <= 1e-12, k


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_batch_plan_with_coupled_models(env, precision):
    """A batch plan mixing per-link models (default, Eq. (12)) with coupled ones
    (paper dynamics with RKF45, eliminated joints with RK4) and several n_sub:
    the per-link instances take the persistent kernel, the coupled ones are
    grouped by (model, n_sub) and take the coupled path; every instance meets
    the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(35)
    robots = [synth.hopper(rng),
              synth.with_paper_dynamics(synth.biped(rng), **PAPER),
              synth.with_paper_dynamics(synth.cheetah7(rng), joint_forces=1, scheme=0),
              synth.with_cross_states(synth.biped(rng))]
    probs, midx = [], []
    for _ in range(13):
        mi = int(rng.integers(0, len(robots)))
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 60)), int(rng.choice([1, 3])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15)))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(plan.pack([q.X for q in probs], "X"))
    U = t(plan.pack([q.U for q in probs], "U"))
    sv = t(plan.pack([q.s for q in probs], "s"))
    out = plan.discretize(X, U, sv)
    plan.sync_status()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    for i, q in enumerate(probs):
        R = q.robot
        N, nxt, nu, nc = q.N, R.nxt, R.nu, R.nc
        got = {"A": plan.unpack(host["A"], "A", i, (N, nxt, nxt)),
               "Bm": plan.unpack(host["Bm"], "B", i, (N, nxt, nu)),
               "Bp": plan.unpack(host["Bp"], "B", i, (N, nxt, nu)),
               "S": plan.unpack(host["S"], "S", i, (N, nxt)),
               "defect": plan.unpack(host["defect"], "defect", i, (N, nxt)),
               "penalty": plan.unpack(host["penalty"], "penalty", i, (N, nc))}
        ref = oracle.discretize(R.as_dict(), q.X, q.U, q.s, q.n_sub)
        _check(got, ref, precision)
    # graph replay gives the same numbers
    out2 = plan.discretize(X, U, sv)
    plan.sync_status()
    for k in out:
        assert torch.equal(out[k], out2[k]), k


@pytest.mark.parametrize("n_chunks", [1, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_host_executor_with_coupled_models(env, precision, n_chunks):
    """ciscvx_batch_run_host on a plan mixing per-link and coupled-link models
    (linearization, and linearization + VJP): every output equals the device
    path's to rounding (the executor regroups which intervals share a warp,
    and warps vote on the angle chain's Taylor tier), and the coupled VJPs
    meet the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(40)
    robots = [synth.cheetah7(rng), synth.with_paper_dynamics(synth.biped(rng), **PAPER)]
    probs, midx = [], []
    for i in range(7):
        mi = i % 2
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(5, 50)), 3, q_noise=0.1,
                                         u_dist="normal", s_range=(0.05, 0.15), with_cotangents=True))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X = t(plan.pack([q.X for q in probs], "X"))
    U = t(plan.pack([q.U for q in probs], "U"))
    sv = t(plan.pack([q.s for q in probs], "s"))
    w = t(plan.pack([q.w for q in probs], "defect"))
    rho = t(plan.pack([q.rho for q in probs], "penalty"))
    ws = torch.empty(plan.vjp_workspace_size(), dtype=torch.uint8, device=dev)
    ref = plan.discretize(X, U, sv)
    gref = plan.discretize_vjp(X, U, sv, w, rho, workspace=ws)
    torch.cuda.synchronize()
    pin = lambda a: a.cpu().pin_memory()  # noqa: E731
    host_in = {"X": pin(X), "U": pin(U), "s": pin(sv)}
    dev_in = {k: torch.empty_like(v) for k, v in (("X", X), ("U", U), ("s", sv))}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in ref.items()}
    dev_out = {k: torch.empty_like(v) for k, v in ref.items()}
    host_vjp = {"w": pin(w), "rho": pin(rho)}
    host_vjp.update({k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in gref.items()})
    dev_vjp = {"w": torch.empty_like(w), "rho": torch.empty_like(rho)}
    dev_vjp.update({k: torch.empty_like(v) for k, v in gref.items()})
    for with_vjp in (False, True):
        plan.run_host(host_in, host_out, dev_in, dev_out, n_chunks=n_chunks,
                      host_vjp=host_vjp if with_vjp else None, dev_vjp=dev_vjp if with_vjp else None,
                      workspace=ws)
        torch.cuda.current_stream().synchronize()
        plan.sync_status()
        for k, v in ref.items():
            tol = 1e-6 if v.dtype == torch.float32 else 1e-12
            assert block_err(host_out[k].double().numpy(), v.double().cpu().numpy()) <= tol, k
        if with_vjp:
            for k, v in gref.items():
                assert block_err(host_vjp[k].numpy(), v.cpu().numpy()) <= 1e-12, k
            tol = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
            gX = host_vjp["gX"].numpy()
            for i, q in enumerate(probs):
                if midx[i] != 1:
                    continue
                rX, rU, rs, rL = oracle.vjp(q.robot.as_dict(), q.X, q.U, q.s, q.w, q.rho, q.n_sub)
                assert block_err(plan.unpack(gX, "X", i, rX.shape), rX) <= tol, i


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("layout", ["node", "interval"])
def test_affine_term(env, precision, tol, layout):
    """z_k = x~(1) - A x~_k - B- u_L - B+ u_R - S s_k, from the oracle's blocks
    (coupled links: formed from the dense outputs after the coupled kernels)."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    p = _problem("hopper", 29, 45, 4, **PAPER)
    U = p.U
    if layout == "interval":
        U = np.stack([p.U[:-1], p.U[1:]], axis=1) + 0.1
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)  # noqa: E731
    got = api.discretize(m, t(p.X), t(U), t(p.s), p.n_sub, precision, layout, want_z=True)
    ref = oracle.discretize(p.robot.as_dict(), p.X, U, p.s, p.n_sub, layout)
    uL, uR = (p.U[:-1], p.U[1:]) if layout == "node" else (U[:, 0], U[:, 1])
    z = ref["defect"] + p.X[1:] - np.einsum("kij,kj->ki", ref["A"], p.X[:-1]) \
        - np.einsum("kij,kj->ki", ref["Bm"], uL) - np.einsum("kij,kj->ki", ref["Bp"], uR) \
        - ref["S"] * p.s[:, None]
    zg = got["z"].cpu().numpy()
    for k in range(p.N):
        assert block_err(zg[k], z[k]) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
@pytest.mark.parametrize("out_format", ["dense", "compact"])
def test_shared_nominal_pass_in_the_fused_entry_point(env, precision, tol, out_format):
    """ciscvx_batch_discretize_and_vjp on a plan of default and coupled models:
    the coupled instances take one nominal pass for the linearization and the
    VJP.  Against the two separate calls (to rounding: the separate
    linearization groups the coupled intervals into warps across instances,
    and the default-model instances take the fused per-link pass) and against
    the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(61)
    robots = [synth.hopper(rng), synth.with_paper_dynamics(synth.biped(rng), **PAPER),
              synth.with_paper_dynamics(synth.cheetah7(rng), joint_forces=1, scheme=0)]
    probs, midx = [], []
    for i in range(7):
        mi = i % 3
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 45)), int(rng.choice([1, 2])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15), with_cotangents=True))
        midx.append(mi)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision,
                         out_format=out_format)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, sv = (t(plan.pack([getattr(q, k) for q in probs], k)) for k in ("X", "U", "s"))
    w = t(plan.pack([q.w for q in probs], "defect"))
    rho = t(plan.pack([q.rho for q in probs], "penalty"))
    out, g = plan.discretize_and_vjp(X, U, sv, w, rho)
    out = {k: v.clone() for k, v in out.items()}
    g = {k: v.clone() for k, v in g.items()}
    out2 = plan.discretize(X, U, sv)
    g2 = plan.discretize_vjp(X, U, sv, w, rho)
    plan.sync_status()
    btol = 1e-13 if precision == "fp64" else 1e-6
    for k in out:
        assert block_err(out[k].double().cpu().numpy(), out2[k].double().cpu().numpy()) <= btol, k
    for k in ("gX", "gU", "gs", "L"):  # (the default-model instances: fused pass against the adjoint kernel)
        e = block_err(g[k].cpu().numpy(), g2[k].cpu().numpy())
        assert e <= (1e-12 if precision == "fp64" else 1e-5), (k, e)
    host = {k: v.cpu().numpy() for k, v in g.items()}
    for i, q in enumerate(probs):
        rX, rU, rs, rL = oracle.vjp(q.robot.as_dict(), q.X, q.U, q.s, q.w, q.rho, q.n_sub)
        assert block_err(plan.unpack(host["gX"], "X", i, q.X.shape), rX) <= tol, i
        assert block_err(plan.unpack(host["gU"], "U", i, q.U.shape), rU) <= tol, i
        assert block_err(plan.unpack(host["gs"], "s", i, q.s.shape), rs) <= tol, i
        assert abs(host["L"][i] - rL) <= TOL_FP64 * max(1.0, abs(rL)) + (0 if precision == "fp64" else tol), i
