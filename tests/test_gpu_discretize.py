"""GPU parity of ciscvx_discretize against the FP64 oracle (through the C ABI).

Tolerances: FP64 path rel <= 1e-10 on every block (block-normwise); FP32-Phi
path rel <= 1e-4 on A, B-, B+, S and rel <= 1e-10 on defect and penalty (the
state stays FP64).  Sizes span several warps of 32 intervals and a ragged
tail.
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


def _run(env, p, precision, layout="node", want_z=False, X=None, U=None, s=None):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    X = p.X if X is None else X
    U = (p.U if layout == "node" else p.U_interval()) if U is None else U
    s = p.s if s is None else s
    m = api.Model(p.robot)
    out = api.discretize(m, torch.tensor(X, device=dev), torch.tensor(U, device=dev),
                         torch.tensor(s, device=dev), p.n_sub, precision, layout, want_z=want_z)
    api.sync_status(m)
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    ref = oracle.discretize(p.robot.as_dict(), X, U, s, p.n_sub, layout=layout)
    return got, ref


def _check(got, ref, precision):
    tol_phi = TOL_FP64 if precision == "fp64" else TOL_FP32_PHI
    for k in PHI:
        assert block_err(got[k], ref[k]) <= tol_phi, (k, block_err(got[k], ref[k]))
    for k in STATE:
        assert block_err(got[k], ref[k]) <= TOL_FP64, (k, block_err(got[k], ref[k]))


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_hopper_n10(env, precision):
    got, ref = _run(env, synth.hopper_fp64(), precision)
    _check(got, ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_cheetah_n50(env, precision):
    got, ref = _run(env, synth.cheetah_n50(), precision)
    _check(got, ref, precision)


def test_cheetah_per_interval_elementwise(env):
    """Per interval and element: |d| <= 1e-10 * max(|block|) of that interval."""
    got, ref = _run(env, synth.cheetah_n50(seed=3), "fp64")
    for k in PHI:
        for i in range(ref[k].shape[0]):
            assert block_err(got[k][i], ref[k][i]) <= TOL_FP64, (k, i)


@pytest.mark.parametrize("layout", ["node", "interval"])
def test_biped_ragged_layouts(env, layout):
    rng = np.random.default_rng(5)
    robot = synth.biped(rng)
    p = synth.draw_instance(robot, rng, 37, 6, q_noise=0.1, u_dist="normal", s_range=(0.05, 0.15))
    U = p.U_interval() if layout == "interval" else p.U
    if layout == "interval":   # FOH that jumps at the nodes
        U = U + 0.3 * rng.standard_normal(U.shape)
    got, ref = _run(env, p, "fp64", layout=layout, U=U)
    _check(got, ref, "fp64")


def test_affine_term(env):
    p = synth.hopper_fp64(seed=2)
    got, ref = _run(env, p, "fp64", want_z=True)
    x1 = ref["defect"] + p.X[1:]
    z = x1 - np.einsum("kij,kj->ki", ref["A"], p.X[:-1]) - np.einsum("kij,kj->ki", ref["Bm"], p.U[:-1]) \
        - np.einsum("kij,kj->ki", ref["Bp"], p.U[1:]) - ref["S"] * p.s[:, None]
    assert block_err(got["z"], z) <= 1e-10


@pytest.mark.parametrize("N,n_sub", [(1, 1), (1, 7), (33, 1), (64, 3)])
def test_small_and_tile_edges(env, N, n_sub):
    p = synth.cheetah_n50(seed=4, N=N, n_sub=n_sub)
    got, ref = _run(env, p, "fp64")
    _check(got, ref, "fp64")


def test_zero_dilation(env):
    p = synth.hopper_fp64(seed=6)
    s = np.zeros_like(p.s)
    got, ref = _run(env, p, "fp64", s=s)
    _check(got, ref, "fp64")
    assert np.array_equal(got["A"], np.broadcast_to(np.eye(p.robot.nxt), got["A"].shape))
    assert np.all(got["Bm"] == 0) and np.all(got["Bp"] == 0)


def test_feasible_inputs_penalty_exactly_zero(env):
    rng = np.random.default_rng(4)
    robot = synth.cheetah7(rng)
    p = synth.draw_instance(robot, rng, 40, 5, q_noise=0.02, u_dist="normal", s_range=(0.04, 0.06))
    X = p.X.copy()
    X[:, 1: 3 * robot.nb: 3] += 0.6
    X[:, 3 * robot.nb: 6 * robot.nb] = 0.0
    U = p.U.copy()
    for i in range(robot.nc):
        base = 3 * robot.nj + 3 * i
        U[:, base] = rng.uniform(1.0, 2.0, p.N + 1)
        U[:, base + 1] = rng.uniform(0.0, 0.4, p.N + 1)
        U[:, base + 2] = rng.uniform(0.0, 0.4, p.N + 1)
    got, ref = _run(env, p, "fp64", X=X, U=U)
    _check(got, ref, "fp64")
    assert np.all(got["penalty"] == 0.0)
    ny = slice(robot.nx, robot.nxt)
    assert np.all(got["Bm"][:, ny] == 0.0) and np.all(got["S"][:, ny] == 0.0)


def test_nonfinite_input_sets_status(env):
    torch, oracle, api = env
    p = synth.hopper_fp64()
    X = p.X.copy()
    X[3, 2] = np.nan
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    api.discretize(m, torch.tensor(X, device=dev), torch.tensor(p.U, device=dev),
                   torch.tensor(p.s, device=dev), p.n_sub, "fp64")
    with pytest.raises(api.CiscvxError) as e:
        api.sync_status(m)
    assert e.value.status == api.ENONFINITE
    api.sync_status(m)  # cleared by the read


def test_argument_errors(env):
    torch, oracle, api = env
    p = synth.hopper_fp64()
    dev = torch.device("cuda:0")
    m = api.Model(p.robot)
    X, U, s = (torch.tensor(a, device=dev) for a in (p.X, p.U, p.s))
    with pytest.raises(api.CiscvxError) as e:
        api.discretize(m, X, U, s, 0, "fp64")
    assert e.value.status == api.EINVAL
    for prec in ("tf32_tc", "bf16_tc"):
        with pytest.raises(api.CiscvxError) as e:
            api.discretize(m, X, U, s, 4, prec)
        assert e.value.status == api.EUNSUPPORTED


def _edge_robots():
    rng = np.random.default_rng(12)
    h = synth.hopper(rng).as_dict()
    no_contact = dict(h, contact_body=np.zeros(0, dtype=np.int32), contact_rho=np.zeros((0, 2)),
                      contact_mu=np.zeros(0))
    lone = {"mass": np.array([1.7]), "inertia": np.array([0.05]),
            "joint_parent": np.zeros(0, dtype=np.int32), "joint_child": np.zeros(0, dtype=np.int32),
            "joint_rho_parent": np.zeros((0, 2)), "joint_rho_child": np.zeros((0, 2)),
            "contact_body": np.zeros(0, dtype=np.int32), "contact_rho": np.zeros((0, 2)),
            "contact_mu": np.zeros(0), "gravity": synth.GRAVITY}
    return {"no_contact": no_contact, "lone_link": lone}


@pytest.mark.parametrize("which", ["no_contact", "lone_link"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
def test_models_without_contacts_or_inputs(env, which, precision):
    """n_c = 0 (no penalty state) and n_u = 0 (no inputs at all, empty B blocks)."""
    torch, oracle, api = env
    R = _edge_robots()[which]
    nb, nj = len(R["mass"]), len(R["joint_parent"])
    nxt, nu = 6 * nb, 3 * nj
    rng = np.random.default_rng(3)
    N, n_sub = 37, 4
    X = rng.uniform(-0.5, 0.5, (N + 1, nxt))
    U = rng.standard_normal((N + 1, nu))
    s = rng.uniform(0.05, 0.15, N)
    dev = torch.device("cuda:0")
    m = api.Model(R)
    assert (m.nx, m.ny, m.nu) == (nxt, 0, nu)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.discretize(m, t(X), t(U), t(s), n_sub, precision)
    api.sync_status(m)
    got = {k: v.double().cpu().numpy() for k, v in out.items()}
    ref = oracle.discretize(R, X, U, s, n_sub)
    _check(got, ref, precision)
    w = rng.standard_normal((N, nxt))
    gX, gU, gs, L = api.discretize_vjp(m, t(X), t(U), t(s), t(w), None, n_sub, precision)
    rX, rU, rs, rL = oracle.vjp(R, X, U, s, w, np.zeros((N, 0)), n_sub)
    tol = 1e-10 if precision == "fp64" else 1e-4
    assert block_err(gX.cpu().numpy(), rX) <= tol
    assert block_err(gU.cpu().numpy(), rU) <= tol
    assert block_err(gs.cpu().numpy(), rs) <= tol
    assert abs(float(L) - rL) <= tol * max(1.0, abs(rL))
