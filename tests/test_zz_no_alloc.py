"""The allocation-free VJP entry point agrees with the workspace VJP (GPU).

ciscvx_discretize_vjp_static is for callers that cannot allocate device memory
when they call the library (a control loop with a real-time budget, or a
framework that owns all device memory through its own pool).  It runs the same
VJP with scratch memory held inside the library.  Here it is called twice in a
row through the C ABI, and both results are checked against
ciscvx_discretize_vjp with a caller workspace, within the FP64 tolerance the
parity tests use.  It must pass alone in a fresh process and after the other
tests, so it builds and loads everything it needs itself.
"""
import ctypes

import numpy as np
import pytest

from _util import TOL_FP64, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2604_09993_gb300 import api, build
    build.build()
    api.load()
    return torch, api


def _static_call(api, lib, m, N, n_sub, X, U, s, w, rho):
    import torch
    gX, gU, gs = torch.empty_like(X), torch.empty_like(U), torch.empty_like(s)
    L = torch.empty((), dtype=torch.float64, device=X.device)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = lib.ciscvx_discretize_vjp_static(
        m.handle, N, n_sub, api.PRECISION["fp64"], api.LAYOUT["node"], p(X), p(U), p(s), p(w),
        p(rho), p(gX), p(gU), p(gs), p(L), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == api.OK, lib.ciscvx_last_error()
    return gX, gU, gs, L


def test_static_scratch_vjp_matches_workspace_vjp_twice(env):
    torch, api = env
    lib = api.load()
    dev = torch.device("cuda:0")
    p = synth.cheetah_adjoint(seed=0)
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    X, U, s, w, rho = t(p.X), t(p.U), t(p.s), t(p.w), t(p.rho)
    ref = api.discretize_vjp(m, X, U, s, w, rho, p.n_sub, "fp64")
    for _ in range(2):
        got = _static_call(api, lib, m, p.N, p.n_sub, X, U, s, w, rho)
        torch.cuda.synchronize()
        for g, r, name in zip(got, ref, ("gX", "gU", "gs", "L")):
            err = block_err(g.cpu().numpy(), r.cpu().numpy())
            assert err <= TOL_FP64, (name, err)
    api.sync_status(m)


def test_static_scratch_rejects_requests_above_its_size(env):
    torch, api = env
    lib = api.load()
    p = synth.hopper_fp64(seed=0)
    m = api.Model(p.robot)
    per = api.workspace_size(m, api.OP_VJP, 1000) / 1000.0
    N = int(1.2 * (16 * 1024 * 1024) / per)
    assert api.workspace_size(m, api.OP_VJP, N) > 16 * 1024 * 1024
    # The size check comes before any pointer is used, so empty buffers suffice.
    st = lib.ciscvx_discretize_vjp_static(m.handle, N, 4, 0, 0, *([ctypes.c_void_p(16)] * 9),
                                          None)
    assert st == api.EUNSUPPORTED
    assert b"static scratch" in lib.ciscvx_last_error()
