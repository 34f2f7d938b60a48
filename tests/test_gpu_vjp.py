"""GPU parity of ciscvx_discretize_vjp against the oracle's Phi-contracted
gradient and against central differences (through the C ABI).

Tolerances: FP64 adjoint rel <= 1e-10 (block-normwise per output); FP32
adjoint rel <= 1e-4; central differences (h = 1e-6) rel <= 1e-6.
"""
import numpy as np
import pytest

from _util import block_err
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


def _vjp(env, p, precision, layout="node", U=None):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    U = (p.U if layout == "node" else p.U_interval()) if U is None else U
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    gX, gU, gs, L = api.discretize_vjp(m, t(p.X), t(U), t(p.s), t(p.w), t(p.rho), p.n_sub,
                                       precision, layout)
    api.sync_status(m)
    got = (gX.cpu().numpy(), gU.cpu().numpy(), gs.cpu().numpy(), float(L))
    ref = oracle.vjp(p.robot.as_dict(), p.X, U, p.s, p.w, p.rho, p.n_sub, layout=layout)
    return got, ref


def _check(got, ref, tol):
    for g, r, nm in zip(got[:3], ref[:3], ("gX", "gU", "gs")):
        assert block_err(g, r) <= tol, (nm, block_err(g, r))
    assert abs(got[3] - ref[3]) <= tol * max(1.0, abs(ref[3]))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_phi", 1e-4)])
def test_hopper(env, precision, tol):
    got, ref = _vjp(env, synth.hopper_fp64(), precision)
    _check(got, ref, tol)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_phi", 1e-4)])
def test_cheetah_adjoint_n100(env, precision, tol):
    got, ref = _vjp(env, synth.cheetah_adjoint(), precision)
    _check(got, ref, tol)


def test_interval_layout_biped(env):
    rng = np.random.default_rng(8)
    robot = synth.biped(rng)
    p = synth.draw_instance(robot, rng, 45, 4, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15),
                            with_cotangents=True)
    U = p.U_interval() + 0.2 * rng.standard_normal((p.N, 2, robot.nu))
    got, ref = _vjp(env, p, "fp64", layout="interval", U=U)
    _check(got, ref, 1e-10)


@pytest.mark.parametrize("N,n_sub", [(1, 1), (2, 64), (40, 2)])
def test_edges(env, N, n_sub):
    p = synth.cheetah_n50(seed=9, N=N, n_sub=n_sub)
    got, ref = _vjp(env, p, "fp64")
    _check(got, ref, 1e-10)


def test_central_differences(env):
    torch, oracle, api = env
    p = synth.hopper_fp64(seed=1, N=2, n_sub=3)
    got, _ = _vjp(env, p, "fp64")
    R = p.robot.as_dict()
    nx = p.robot.nx

    def L(X, U, s):
        tot = 0.0
        for k in range(p.N):
            x1 = oracle.flow(R, p.n_sub, X[k], U[k], U[k + 1], s[k])
            tot += p.w[k] @ (x1 - X[k + 1]) + p.rho[k] @ (x1[nx:] - X[k, nx:])
        return tot

    e = 1e-6
    for arr, g in ((p.X, got[0]), (p.U, got[1]), (p.s, got[2])):
        flat, gf = arr.reshape(-1), g.reshape(-1)
        for i in range(flat.size):
            v = flat[i]
            flat[i] = v + e; lp = L(p.X, p.U, p.s)
            flat[i] = v - e; lm = L(p.X, p.U, p.s)
            flat[i] = v
            fd = (lp - lm) / (2 * e)
            assert abs(fd - gf[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gf[i])


def test_autograd_function(env):
    torch, oracle, api = env
    p = synth.cheetah_n50(seed=2, N=20, n_sub=5)
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    X = torch.tensor(p.X, device=dev, requires_grad=True)
    U = torch.tensor(p.U, device=dev, requires_grad=True)
    s = torch.tensor(p.s, device=dev, requires_grad=True)
    defect, penalty = api.discretize_fn(m, X, U, s, p.n_sub)
    L = (torch.tensor(p.w, device=dev) * defect).sum() + (torch.tensor(p.rho, device=dev) * penalty).sum()
    L.backward()
    rX, rU, rs, rL = oracle.vjp(p.robot.as_dict(), p.X, p.U, p.s, p.w, p.rho, p.n_sub)
    assert abs(L.item() - rL) <= 1e-10 * max(1.0, abs(rL))
    assert block_err(X.grad.cpu().numpy(), rX) <= 1e-10
    assert block_err(U.grad.cpu().numpy(), rU) <= 1e-10
    assert block_err(s.grad.cpu().numpy(), rs) <= 1e-10


def test_workspace_errors(env):
    torch, oracle, api = env
    p = synth.hopper_fp64()
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    small = torch.empty(8, dtype=torch.uint8, device=dev)
    import ctypes
    lib = api.load()
    gX, gU, gs = torch.empty_like(t(p.X)), torch.empty_like(t(p.U)), torch.empty_like(t(p.s))
    X, U, s, w, r = t(p.X), t(p.U), t(p.s), t(p.w), t(p.rho)
    st = lib.ciscvx_discretize_vjp(m.handle, p.N, p.n_sub, 0, 0, *(ctypes.c_void_p(a.data_ptr()) for a in (X, U, s, w, r, gX, gU, gs)),
                                   None, ctypes.c_void_p(small.data_ptr()), 8, None)
    assert st == api.EINVAL
    with pytest.raises(api.CiscvxError) as e:
        api.discretize_vjp(m, X, U, s, w, r, 65, "fp64")
    assert e.value.status == api.EUNSUPPORTED
