"""Batched VJPs of plans that mix the default model, the Eq. (12) auxiliary
state (the per-link adjoint kernel with its CROSS foot links) and coupled
links (the coupled path's reverse-mode adjoint, one instance after another).
Every instance's gX, gU, gs and L is compared with the oracle's
Phi-contracted gradient (FP64 1e-10, FP32-Phi 1e-4 for the gradients; L in
FP64), the fused entry point gives the same numbers as the two calls, and the
pipelined host executor those of the device path."""
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
    # coupled instances: one nominal pass per instance feeds both outputs; the
    # separate linearization groups the coupled intervals of the plan into
    # warps differently (the angle chain's Taylor tier is a warp vote), so
    # the blocks agree to rounding; per-link instances (Eq. (12) ones
    # included) take the fused per-link pass
    for k in ("A", "Bm", "Bp", "S", "defect", "penalty"):
        assert block_err(out[k].cpu().numpy(), out2[k].cpu().numpy()) <= 1e-13, k
    for k in ("gX", "gU", "gs", "L"):  # (per-link instances: fused pass against the adjoint kernel)
        assert block_err(gout[k].cpu().numpy(), g2[k].cpu().numpy()) <= 1e-12, k


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_phi", TOL_FP32_PHI)])
def test_run_host_with_eq12_and_coupled_instances(env, precision, tol):
    """ciscvx_batch_run_host with the VJP on such a mixed batch (Eq. (12)
    instances: linearization then adjoint per chunk; coupled instances: their
    own path) equals the device path, and the oracle."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    robots, probs, midx = _batch(43, 14)
    models = [api.Model(r) for r in robots]
    plan = api.BatchPlan(models, midx, [q.N for q in probs], [q.n_sub for q in probs], precision=precision)
    lo, hi = plan.vjp_workspace_sizes()
    assert lo == hi  # no dense blocks: one scratch size
    X, U, s, w, rho = _packed(torch, plan, probs, dev)
    ws = torch.empty(lo, dtype=torch.uint8, device=dev)
    out_d, g_d = plan.discretize_and_vjp(X, U, s, w, rho, workspace=ws)
    plan.sync_status()
    out_d = {k: v.clone() for k, v in out_d.items()}
    g_d = {k: v.clone() for k, v in g_d.items()}
    pin = lambda v: v.cpu().pin_memory()  # noqa: E731
    host_in = {"X": pin(X), "U": pin(U), "s": pin(s)}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out_d.items()}
    hv = {"X": host_in["X"], "U": host_in["U"], "s": host_in["s"], "w": pin(w), "rho": pin(rho)}
    hv.update({k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in g_d.items()})
    dev_in = {k: torch.empty_like(v) for k, v in (("X", X), ("U", U), ("s", s))}
    dev_out = {k: torch.empty_like(v) for k, v in out_d.items()}
    dv = {"X": dev_in["X"], "U": dev_in["U"], "s": dev_in["s"], "w": torch.empty_like(w),
          "rho": torch.empty_like(rho)}
    dv.update({k: torch.empty_like(v) for k, v in g_d.items()})
    plan.run_host(host_in, host_out, dev_in, dev_out, n_chunks=3, host_vjp=hv, dev_vjp=dv, workspace=ws)
    torch.cuda.synchronize()
    plan.sync_status()
    for k in ("defect", "penalty"):
        assert block_err(host_out[k].numpy(), out_d[k].cpu().numpy()) <= 1e-13, k
    for k in ("A", "Bm", "Bp", "S"):
        assert block_err(host_out[k].double().numpy(), out_d[k].double().cpu().numpy()) <= 1e-6, k
    for k in ("gX", "gU", "gs", "L"):
        e = block_err(hv[k].numpy(), g_d[k].cpu().numpy())
        assert e <= (1e-12 if precision == "fp64" else 1e-5), (k, e)
    host = {k: hv[k].numpy() for k in ("gX", "gU", "gs", "L")}
    for i, q in enumerate(probs):
        rX, rU, rs, rL = oracle.vjp(q.robot.as_dict(), q.X, q.U, q.s, q.w, q.rho, q.n_sub)
        assert block_err(plan.unpack(host["gX"], "X", i, q.X.shape), rX) <= tol, i
        assert block_err(plan.unpack(host["gU"], "U", i, q.U.shape), rU) <= tol, i
        assert block_err(plan.unpack(host["gs"], "s", i, q.s.shape), rs) <= tol, i
