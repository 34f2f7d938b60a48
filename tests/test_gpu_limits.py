"""GPU parity at the library's model-size limit (through the C ABI).

The largest model ciscvx_model_create takes has CISCVX_MAX_BODIES = 32 links;
here a torso with legs of 15 and 16 links (n_x~ = 194, n_u = 99, two
contacts, six inputs on every link).  Its linearization, its VJP and the
fused linearization + VJP of a one-instance batch plan are checked against
the oracle over a ragged horizon (37 intervals: a full warp of intervals and
a tail of 5), in both precisions.  Tolerances as in the other parity tests.
"""
import numpy as np
import pytest

from _util import TOL_FP32_PHI, TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_BODIES = 32


@pytest.fixture(scope="module")
def env():
    import torch
    import oracle
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return torch, oracle, api


@pytest.fixture(scope="module")
def case(env):
    torch, oracle, api = env
    rng = np.random.default_rng(32)
    R = synth.chain32(rng)
    assert R.nb == MAX_BODIES
    p = synth.draw_instance(R, rng, 37, 3, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15),
                            with_cotangents=True)
    ref = oracle.discretize(R.as_dict(), p.X, p.U, p.s, p.n_sub)
    gref = oracle.vjp(R.as_dict(), p.X, p.U, p.s, p.w, p.rho, p.n_sub)
    return p, ref, gref


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_largest_model_discretize_and_vjp(env, case, precision):
    torch, oracle, api = env
    p, ref, gref = case
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    m = api.Model(p.robot)
    assert (m.nx + m.ny, m.nu) == (p.robot.nxt, p.robot.nu)
    out = api.discretize(m, t(p.X), t(p.U), t(p.s), p.n_sub, precision)
    gX, gU, gs, L = api.discretize_vjp(m, t(p.X), t(p.U), t(p.s), t(p.w), t(p.rho), p.n_sub, precision)
    api.sync_status(m)
    tol_phi = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for k in ("A", "Bm", "Bp", "S"):
        assert block_err(out[k].double().cpu().numpy(), ref[k]) <= tol_phi, k
    for k in ("defect", "penalty"):
        assert block_err(out[k].cpu().numpy(), ref[k]) <= TOL_FP64, k
    tol = 1e-10 if precision == "fp64" else 1e-4
    rX, rU, rs, rL = gref
    for g, r, nm in ((gX, rX, "gX"), (gU, rU, "gU"), (gs, rs, "gs")):
        assert block_err(g.cpu().numpy(), r) <= tol, nm
    assert abs(float(L) - rL) <= tol * max(1.0, abs(rL))


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_largest_model_fused_pass(env, case, precision):
    """The fused linearization + VJP (the bench's step) of a one-instance
    plan of the 32-link model, under the fused autotuner's pick."""
    torch, oracle, api = env
    p, ref, gref = case
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    plan = api.BatchPlan([m], [0], [p.N], [p.n_sub], precision=precision)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, s = t(plan.pack([p.X], "X")), t(plan.pack([p.U], "U")), t(plan.pack([p.s], "s"))
    w, rho = t(plan.pack([p.w], "defect")), t(plan.pack([p.rho], "penalty"))
    plan.autotune_fused(X, U, s, w, rho)
    out, g = plan.discretize_and_vjp(X, U, s, w, rho)
    plan.sync_status()
    tol_phi = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    okey = {"A": "A", "Bm": "B", "Bp": "B", "S": "S", "defect": "defect", "penalty": "penalty"}
    for k in ("A", "Bm", "Bp", "S", "defect", "penalty"):
        got = plan.unpack(host[k], okey[k], 0, ref[k].shape)
        assert block_err(got, ref[k]) <= (tol_phi if k in ("A", "Bm", "Bp", "S") else TOL_FP64), k
    tol = 1e-10 if precision == "fp64" else 1e-4
    rX, rU, rs, rL = gref
    gh = {k: g[k].cpu().numpy() for k in ("gX", "gU", "gs", "L")}
    assert block_err(plan.unpack(gh["gX"], "X", 0, rX.shape), rX) <= tol
    assert block_err(plan.unpack(gh["gU"], "U", 0, rU.shape), rU) <= tol
    assert block_err(plan.unpack(gh["gs"], "s", 0, rs.shape), rs) <= tol
    assert abs(gh["L"][0] - rL) <= tol * max(1.0, abs(rL))
