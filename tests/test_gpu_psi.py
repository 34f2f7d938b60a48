"""GPU parity of Psi^{delta,eps} (ciscvx_psi_linearize) against the oracle.

Psi and its Jacobian in y-_{k+1} are compared interval by interval with the
oracle's dual-number values at the FP64 tolerance, for the Eq. (12) auxiliary
state and for one penalty state per contact; the oracle's Jacobian in y+_k is
checked to be the negative of the GPU's block.  Interval counts span several
blocks with a ragged tail; the sweep size is checked on sampled intervals.
"""
import numpy as np
import pytest

from _util import TOL_FP64, block_err
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


def _robot(name, cross):
    rng = np.random.default_rng(41)
    R = getattr(synth, name)(rng)
    return (synth.with_cross_states(R) if cross else R).as_dict()


def _nodes(R, N, seed, nxt):
    rng = np.random.default_rng(seed)
    Xp = rng.uniform(-1, 1, (N + 1, nxt))
    Xm = Xp + 0.3 * rng.standard_normal((N + 1, nxt))
    return Xp, Xm


@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7"])
@pytest.mark.parametrize("cross", [False, True])
@pytest.mark.parametrize("N", [1, 37, 1000])
def test_psi_parity(env, name, cross, N):
    torch, oracle, api = env
    R = _robot(name, cross)
    m = api.Model(R)
    ny = m.ny
    Xp, Xm = _nodes(R, N, 7 + N, m.nxt)
    delta, eps = 0.05, 1e-4
    dev = torch.device("cuda:0")
    out = api.psi_linearize(m, torch.tensor(Xp, device=dev), torch.tensor(Xm, device=dev), delta, eps)
    api.sync_status(m)
    ref = oracle.psi(R, Xp, Xm, delta, eps)
    psi, dpsi = out["psi"].cpu().numpy(), out["dpsi"].cpu().numpy()
    assert psi.shape == ref["psi"].shape == (N, api.psi_rows(m))
    assert dpsi.shape == (N, psi.shape[1], ny)
    for k in range(N):
        assert block_err(psi[k], ref["psi"][k]) <= TOL_FP64
        assert block_err(dpsi[k], ref["J"][k][:, ny:]) <= TOL_FP64
        assert block_err(-dpsi[k], ref["J"][k][:, :ny]) <= TOL_FP64


def test_psi_without_jacobian_and_at_sweep_size(env):
    """4096 x 400 intervals of the 7-link chain with the Eq. (12) state, sampled."""
    torch, oracle, api = env
    R = _robot("cheetah7", True)
    m = api.Model(R)
    N = 4096 * 400
    dev = torch.device("cuda:0")
    g = torch.Generator(device=dev).manual_seed(5)
    Xp = torch.rand((N + 1, m.nxt), device=dev, dtype=torch.float64, generator=g) * 2 - 1
    Xm = torch.rand((N + 1, m.nxt), device=dev, dtype=torch.float64, generator=g) * 2 - 1
    full = api.psi_linearize(m, Xp, Xm, 0.01, 1e-4)
    only = api.psi_linearize(m, Xp, Xm, 0.01, 1e-4, jacobian=False)
    api.sync_status(m)
    assert torch.equal(full["psi"], only["psi"])
    rng = np.random.default_rng(0)
    ks = np.concatenate([[0, N - 1], rng.integers(0, N, 64)])
    for k in ks:
        xp = Xp[k:k + 2].cpu().numpy()
        xm = Xm[k:k + 2].cpu().numpy()
        ref = oracle.psi(R, xp, xm, 0.01, 1e-4)
        assert block_err(full["psi"][k].cpu().numpy(), ref["psi"][0]) <= TOL_FP64
        assert block_err(full["dpsi"][k].cpu().numpy(), ref["J"][0][:, m.ny:]) <= TOL_FP64


def test_psi_edge_cases(env):
    torch, oracle, api = env
    from test_gpu_discretize import _edge_robots
    dev = torch.device("cuda:0")
    m0 = api.Model(_edge_robots()["no_contact"])
    assert api.psi_rows(m0) == 0
    X = torch.zeros((5, m0.nxt), dtype=torch.float64, device=dev)
    out = api.psi_linearize(m0, X, X, 0.1, 1e-4)
    assert out["psi"].shape == (4, 0)
    R = _robot("hopper", True)
    m = api.Model(R)
    X = torch.zeros((3, m.nxt), dtype=torch.float64, device=dev)
    lib = api.load()
    p = api._ptr(X)
    psi = torch.empty((2, api.psi_rows(m)), dtype=torch.float64, device=dev)
    for N, delta, eps in ((0, 0.1, 1e-4), (2, 0.0, 1e-4), (2, float("nan"), 1e-4), (2, 0.1, -1.0),
                          (2, 0.1, float("inf"))):
        assert lib.ciscvx_psi_linearize(m.handle, N, p, p, delta, eps, api._ptr(psi), None,
                                        api._stream()) == api.EINVAL
    assert lib.ciscvx_psi_linearize(m.handle, 2, None, p, 0.1, 1e-4, api._ptr(psi), None,
                                    api._stream()) == api.EINVAL
    # zero increments: FB rows are -sqrt(delta), path rows -eps
    out = api.psi_linearize(m, X, X, 0.25, 1e-3)
    np.testing.assert_array_equal(out["psi"].cpu().numpy()[:, :2 * m.nc], -0.5)
    np.testing.assert_array_equal(out["psi"].cpu().numpy()[:, 2 * m.nc:], -1e-3)


def _every_link_in_contact(cross):
    """7-link chain with one contact at the distal end of every link (n_c = 7)."""
    import dataclasses
    R = synth.cheetah7(np.random.default_rng(43))
    nb = R.nb
    half = 0.5 * np.asarray(R.length)
    R = dataclasses.replace(R, contact_body=np.arange(nb, dtype=np.int32),
                            contact_rho=np.stack([np.zeros(nb), -half], axis=1),
                            contact_mu=np.full(nb, synth.MU))
    return (synth.with_cross_states(R) if cross else R).as_dict()


@pytest.mark.parametrize("cross", [False, True])
def test_psi_many_contacts_and_unaligned_jacobian(env, cross):
    """n_c = 7: an odd contact count, blocks of 36 intervals with a ragged last
    block whose Jacobian slice has an odd length; then the same call with dpsi
    one double past a 16-byte boundary (element-wise stores), bit-identical."""
    torch, oracle, api = env
    R = _every_link_in_contact(cross)
    m = api.Model(R)
    assert m.nc == 7
    N = 101
    Xp, Xm = _nodes(R, N, 99, m.nxt)
    dev = torch.device("cuda:0")
    tXp, tXm = torch.tensor(Xp, device=dev), torch.tensor(Xm, device=dev)
    out = api.psi_linearize(m, tXp, tXm, 0.05, 1e-4)
    api.sync_status(m)
    ref = oracle.psi(R, Xp, Xm, 0.05, 1e-4)
    psi, dpsi = out["psi"].cpu().numpy(), out["dpsi"].cpu().numpy()
    ny = m.ny
    for k in range(N):
        assert block_err(psi[k], ref["psi"][k]) <= TOL_FP64
        assert block_err(dpsi[k], ref["J"][k][:, ny:]) <= TOL_FP64
    npsi = api.psi_rows(m)
    buf = torch.full((N * npsi * ny + 1,), float("nan"), dtype=torch.float64, device=dev)
    off = buf[1:]
    assert off.data_ptr() % 16 == 8
    psi2 = torch.empty_like(out["psi"])
    lib = api.load()
    assert lib.ciscvx_psi_linearize(m.handle, N, api._ptr(tXp), api._ptr(tXm), 0.05, 1e-4,
                                    api._ptr(psi2), api._ptr(off), api._stream()) == 0
    api.sync_status(m)
    assert torch.equal(psi2, out["psi"])
    assert torch.equal(off.view(N, npsi, ny), out["dpsi"])
    assert torch.isnan(buf[0])
