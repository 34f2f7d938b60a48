"""Batched VJPs of plans that hold instances whose VJP is linearize-and-contract
(the Eq. (12) auxiliary state, coupled links) next to default-model instances
(the adjoint kernel).  Every instance's gX, gU, gs and L is compared with the
oracle's Phi-contracted gradient (FP64 1e-10, FP32-Phi 1e-4 for the
gradients; L in FP64), and the fused entry point gives the same numbers as
the two calls."""
import numpy as np
import pytest

from _util import TOL_FP32_PHI, TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu

PAPER = dict(joint_forces=1, scheme=1, terrain=synth.TERRAIN_SINE)


@pytest.fixture(scope="module")
def env():
    import torch
    import oracle
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return torch, oracle, api


def _batch(seed, n_inst):
    rng = np.random.default_rng(seed)
    robots = [synth.hopper(rng),
              synth.with_cross_states(synth.biped(rng)),
              synth.with_paper_dynamics(synth.hopper(rng), **PAPER),
              synth.with_cross_states(synth.with_paper_dynamics(synth.biped(rng), joint_forces=1, scheme=0))]
    probs, midx = [], []
    for i in range(n_inst):
        mi = i % len(robots) if i < len(robots) else int(rng.integers(0, len(robots)))
        probs.append(synth.draw_instance(robots[mi], rng, int(rng.integers(1, 40)), int(rng.choice([2, 3])),
                                         q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15),
                                         with_cotangents=True))
        midx.append(mi)
    return robots, probs, midx


def _packed(torch, plan, probs, dev):
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    return (t(plan.pack([q.X for q in probs], "X")), t(plan.pack([q.U for q in probs], "U")),
            t(plan.pack([q.s for q in probs], "s")), t(plan.pack([q.w for q in probs], "defect")),
            t(plan.pack([q.rho for q in probs], "penalty")))


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
def test_batch_vjp_with_contract_instances(env, precision, tol):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _batch(41, 11)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision)
    X, U, s, w, rho = _packed(torch, plan, probs, dev)
    g = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    host = {k: v.cpu().numpy() for k, v in g.items()}
    for i, q in enumerate(probs):
        R = q.robot
        rX, rU, rs, rL = oracle.vjp(R.as_dict(), q.X, q.U, q.s, q.w, q.rho, q.n_sub)
        gX = plan.unpack(host["gX"], "X", i, q.X.shape)
        gU = plan.unpack(host["gU"], "U", i, q.U.shape)
        gs = plan.unpack(host["gs"], "s", i, q.s.shape)
        for got, ref, nm in ((gX, rX, "gX"), (gU, rU, "gU"), (gs, rs, "gs")):
            assert block_err(got, ref) <= tol, (i, midx[i], nm, block_err(got, ref))
        assert abs(host["L"][i] - rL) <= (TOL_FP64 if precision == "fp64" else tol) * max(1.0, abs(rL)), i


def test_fused_entry_point_with_contract_instances(env):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _batch(42, 9)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision="fp64")
    X, U, s, w, rho = _packed(torch, plan, probs, dev)
    out, gout = plan.discretize_and_vjp(X, U, s, w, rho)
    out2 = plan.discretize(X, U, s)
    g2 = plan.discretize_vjp(X, U, s, w, rho)
    plan.sync_status()
    for k in ("A", "Bm", "Bp", "S", "defect", "penalty"):
        assert torch.equal(out[k], out2[k]), k
    for k in ("gX", "gU", "gs", "L"):
        assert torch.equal(gout[k], g2[k]), k


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
def test_batched_and_per_instance_contract_paths_agree(env, precision, tol):
    """A workspace of the full size takes the batched contract pass, one of the
    minimum size the per-instance one; both meet the oracle and agree."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _batch(43, 14)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision)
    lo, hi = plan.vjp_workspace_sizes()
    assert hi > lo
    X, U, s, w, rho = _packed(torch, plan, probs, dev)
    g_full = plan.discretize_vjp(X, U, s, w, rho, workspace=torch.empty(hi, dtype=torch.uint8, device=dev))
    g_min = plan.discretize_vjp(X, U, s, w, rho, workspace=torch.empty(lo, dtype=torch.uint8, device=dev))
    plan.sync_status()
    for k in ("gX", "gU", "gs", "L"):
        a, b = g_full[k].cpu().numpy(), g_min[k].cpu().numpy()
        assert block_err(a, b) <= (1e-12 if precision == "fp64" else 1e-5), (k, block_err(a, b))
    host = {k: v.cpu().numpy() for k, v in g_full.items()}
    for i, q in enumerate(probs):
        rX, rU, rs, rL = oracle.vjp(q.robot.as_dict(), q.X, q.U, q.s, q.w, q.rho, q.n_sub)
        assert block_err(plan.unpack(host["gX"], "X", i, q.X.shape), rX) <= tol, i
        assert block_err(plan.unpack(host["gU"], "U", i, q.U.shape), rU) <= tol, i
        assert block_err(plan.unpack(host["gs"], "s", i, q.s.shape), rs) <= tol, i
