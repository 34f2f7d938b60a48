"""The allocation-free VJP entry point agrees with the workspace VJP (GPU).

ciscvx_discretize_vjp_static is for callers that cannot allocate device memory
when they call the library: a control loop with a real-time budget (cudaMalloc
can synchronize the device and has no latency bound), or a framework that owns
all device memory through its own pool.  It runs the same VJP with scratch
memory held inside the library.  Here it is called twice in a row, through
the C ABI and through the Python wrapper, and both results are checked against
ciscvx_discretize_vjp with a caller workspace, within the tolerances the parity
tests use: the default per-link model in FP64 and FP32-Phi, the Eq. (12)
auxiliary-state model (the per-link adjoint, whose scratch does not depend on
n_sub) and a model with coupled links (the reverse-mode adjoint of the
coupled path, chunked to what the static array holds).  It must pass alone in a
fresh process and after the other tests, so it builds and loads everything it
needs itself.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from _util import TOL_FP32_PHI, TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2604_09993_gb300 import api, build
    build.build()
    api.load()
    return torch, api


def _static_call(api, lib, m, N, n_sub, precision, X, U, s, w, rho):
    import torch
    gX, gU, gs = torch.empty_like(X), torch.empty_like(U), torch.empty_like(s)
    L = torch.empty((), dtype=torch.float64, device=X.device)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = lib.ciscvx_discretize_vjp_static(
        m.handle, N, n_sub, api.PRECISION[precision], api.LAYOUT["node"], p(X), p(U), p(s), p(w),
        p(rho), p(gX), p(gU), p(gs), p(L), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == api.OK, lib.ciscvx_last_error()
    return gX, gU, gs, L


def _problem(kind):
    if kind == "cheetah7":
        return synth.cheetah_adjoint(seed=0)
    rng = np.random.default_rng(7)
    if kind == "cheetah7-eq12":
        R = synth.with_cross_states(synth.cheetah7(rng))
        N, n_sub = 1000, 10
    else:  # paper dynamics: coupled links (Eq. (3)), RKF45, sinusoidal surface
        R = synth.with_paper_dynamics(synth.cheetah7(rng), terrain=synth.TERRAIN_SINE)
        N, n_sub = 700, 5
    return synth.draw_instance(R, rng, N, n_sub, q_noise=0.1, u_dist="normal", s_range=(0.01, 0.05),
                               with_cotangents=True)


CASES = [("cheetah7", "fp64"), ("cheetah7", "fp32_phi"), ("cheetah7-eq12", "fp32_phi"),
         ("cheetah7-paper", "fp64")]


@pytest.mark.parametrize("kind,precision", CASES)
def test_static_scratch_vjp_matches_workspace_vjp_twice(env, kind, precision):
    torch, api = env
    lib = api.load()
    dev = torch.device("cuda:0")
    p = _problem(kind)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, s, w, rho = t(p.X), t(p.U), t(p.s), t(p.w), t(p.rho)
    lo, hi = api.discretize_workspace_size(m, p.N, p.n_sub, precision, api.OP_VJP)
    assert lo <= api.STATIC_SCRATCH_BYTES
    if kind == "cheetah7-paper":  # chunked: more than one chunk of the static array
        assert hi > api.STATIC_SCRATCH_BYTES
    else:  # the per-link adjoint: one size
        assert lo == hi == api.workspace_size(m, api.OP_VJP, p.N)
    ref = api.discretize_vjp(m, X, U, s, w, rho, p.n_sub, precision)
    tol = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for _ in range(2):
        got = _static_call(api, lib, m, p.N, p.n_sub, precision, X, U, s, w, rho)
        torch.cuda.synchronize()
        for g, r, name in zip(got, ref, ("gX", "gU", "gs", "L")):
            err = block_err(g.cpu().numpy(), r.cpu().numpy())
            assert err <= tol, (name, err)
    # the Python wrapper, without L
    gX, gU, gs, L = api.discretize_vjp_static(m, X, U, s, w, rho, p.n_sub, precision, want_L=False)
    torch.cuda.synchronize()
    assert L is None
    for g, r, name in zip((gX, gU, gs), ref[:3], ("gX", "gU", "gs")):
        assert block_err(g.cpu().numpy(), r.cpu().numpy()) <= tol, name
    api.sync_status(m)


def test_static_scratch_rejects_requests_above_its_size(env):
    torch, api = env
    lib = api.load()
    p = synth.hopper_fp64(seed=0)
    m = api.Model(p.robot)
    per = api.workspace_size(m, api.OP_VJP, 1000) / 1000.0
    N = int(1.2 * api.STATIC_SCRATCH_BYTES / per)
    assert api.workspace_size(m, api.OP_VJP, N) > api.STATIC_SCRATCH_BYTES
    # The size check comes before any pointer is used, so empty buffers suffice.
    st = lib.ciscvx_discretize_vjp_static(m.handle, N, 4, 0, 0, *([ctypes.c_void_p(16)] * 9),
                                          None)
    assert st == api.EUNSUPPORTED
    assert b"static scratch" in lib.ciscvx_last_error()
