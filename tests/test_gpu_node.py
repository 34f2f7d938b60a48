"""GPU parity of the node constraints (ciscvx_node_linearize) against the oracle.

Every output block is compared node by node with the oracle's dual-number
Jacobians at the FP64 tolerance (block-normwise relative 1e-10): the residual
G~, d(v rows)/dv-, d(v rows)/dtheta-, d(v rows)/dPhi, d(v rows)/dp_x-,
Theta^delta and each contact's local Theta Jacobian, on flat ground and on
the sinusoidal surface of Sec. VI-B.  Node counts span several warps with a ragged
tail.
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


def _robot(name):
    rng = np.random.default_rng(31)
    if name in ("hopper", "biped", "cheetah7"):
        return getattr(synth, name)(rng).as_dict()
    if name.endswith("_cross"):  # the Eq. (12) auxiliary state (n_y = 5 n_c)
        return synth.with_cross_states(getattr(synth, name[:-6])(rng)).as_dict()
    if name.endswith("_sine"):  # the sinusoidal contact surface of Sec. VI-B
        R = getattr(synth, name[:-5])(rng)
        return synth.with_paper_dynamics(R, joint_forces=0, scheme=0, terrain=synth.TERRAIN_SINE).as_dict()
    from test_gpu_discretize import _edge_robots
    return _edge_robots()[name]


def _nxt(R):
    nb, nc = len(R["mass"]), len(R["contact_body"])
    return 6 * nb + (5 if R.get("aux_model", 0) else 1) * nc


def _inputs(R, n, seed):
    rng = np.random.default_rng(seed)
    nb, nc = len(R["mass"]), len(R["contact_body"])
    nxt = _nxt(R)
    Xm = rng.uniform(-1, 1, (n, nxt))
    Xp = Xm + 0.5 * rng.standard_normal((n, nxt))
    Phi = rng.standard_normal((n, 2 * nc))
    Gam = rng.uniform(0, 1.5, (n, nc))
    e = rng.uniform(0, 1, nc)
    return Xp, Xm, Phi, Gam, e


def _local_cols(R, nxt):
    """Oracle columns of (p_x-, p_y-, theta-, v_x+, v_y+, omega+, v_x-, v_y-, omega-, Phi_t, Phi_n, Gamma)."""
    nb, nc = len(R["mass"]), len(R["contact_body"])
    nq = 3 * nb
    out = []
    for i, b in enumerate(R["contact_body"]):
        out.append([nxt + 3 * b, nxt + 3 * b + 1, nxt + 3 * b + 2, nq + 3 * b, nq + 3 * b + 1,
                    nq + 3 * b + 2, nxt + nq + 3 * b, nxt + nq + 3 * b + 1, nxt + nq + 3 * b + 2,
                    2 * nxt + 2 * i, 2 * nxt + 2 * i + 1, 2 * nxt + 2 * nc + i])
    return out


def _node_errors(got, ref, R):
    nb, nc = len(R["mass"]), len(R["contact_body"])
    nq, nxt = 3 * nb, _nxt(R)
    V = slice(nq, 2 * nq)
    J = ref["Jg"]
    blocks = {
        "g": (got["g"], ref["g"]),
        "Gvm": (got["Gvm"], J[:, V, nxt + nq:nxt + 2 * nq]),
        "Gth": (got["Gth"], J[:, V, nxt + 2:nxt + nq:3]),
    }
    if nc:
        blocks["Gphi"] = (got["Gphi"], J[:, V, 2 * nxt:2 * nxt + 2 * nc])
        px = [nxt + 3 * b for b in R["contact_body"]]
        blocks["Gpx"] = (got["Gpx"], J[:, V][:, :, px])
        blocks["theta"] = (got["theta"], ref["theta"].reshape(-1, nc, 8))
        cols = _local_cols(R, nxt)
        dref = np.stack([ref["Jth"][:, 8 * i:8 * i + 8][:, :, cols[i]] for i in range(nc)], axis=1)
        blocks["dtheta"] = (got["dtheta"], dref)
    errs = {}
    for k, (a, b) in blocks.items():
        errs[k] = max(block_err(a[t], b[t]) for t in range(a.shape[0]))
    return errs


def _run(env, R, n, seed, delta=1e-3, jacobians=True):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    Xp, Xm, Phi, Gam, e = _inputs(R, n, seed)
    m = api.Model(R)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.node_linearize(m, t(Xp), t(Xm), t(Phi), t(Gam), delta, e, jacobians=jacobians)
    api.sync_status(m)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.node(R, Xp, Xm, Phi, Gam, delta, e)
    return got, ref


@pytest.mark.parametrize("name,n", [("hopper", 45), ("biped", 70), ("cheetah7", 101),
                                    ("no_contact", 33), ("lone_link", 5), ("hopper_sine", 40),
                                    ("biped_sine", 66), ("cheetah7_sine", 99), ("hopper_cross", 37),
                                    ("cheetah7_cross", 64)])
def test_node_linearize_matches_oracle(env, name, n):
    R = _robot(name)
    got, ref = _run(env, R, n, seed=n)
    errs = _node_errors(got, ref, R)
    for k, v in errs.items():
        assert v <= TOL_FP64, (name, k, v)


def test_node_linearize_residual_only(env):
    """Jacobian outputs are optional; the residuals do not change without them."""
    R = _robot("cheetah7")
    full, ref = _run(env, R, 40, seed=2)
    part, _ = _run(env, R, 40, seed=2, jacobians=False)
    assert np.array_equal(full["g"], part["g"]) and np.array_equal(full["theta"], part["theta"])


def test_node_linearize_single_node_and_small_delta(env):
    R = _robot("hopper")
    got, ref = _run(env, R, 1, seed=9, delta=1e-9)
    for k, v in _node_errors(got, ref, R).items():
        assert v <= TOL_FP64, (k, v)


def test_node_linearize_errors(env):
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    R = _robot("hopper")
    m = api.Model(R)
    Xp, Xm, Phi, Gam, e = (torch.tensor(a, device=dev) if isinstance(a, np.ndarray) and a.ndim == 2 else a
                           for a in _inputs(R, 8, 0))
    for delta in (0.0, -1.0, float("nan")):
        with pytest.raises(api.CiscvxError) as ex:
            api.node_linearize(m, Xp, Xm, Phi, Gam, delta, e)
        assert ex.value.status == api.EINVAL
    with pytest.raises(api.CiscvxError) as ex:
        api.node_linearize(m, Xp, Xm, Phi, Gam, 1e-3, [-0.5])
    assert ex.value.status == api.EINVAL
    # a link that is the child of two joints (a closed chain) is outside the forest requirement
    loop = dict(R, joint_parent=np.array([0, 1, 0], dtype=np.int32),
                joint_child=np.array([1, 2, 2], dtype=np.int32),
                joint_rho_parent=np.zeros((3, 2)), joint_rho_child=np.zeros((3, 2)))
    ml = api.Model(loop)
    n = 4
    Xl = torch.zeros((n, ml.nxt), dtype=torch.float64, device=dev)
    with pytest.raises(api.CiscvxError) as ex:
        api.node_linearize(ml, Xl, Xl, Phi[:n], Gam[:n], 1e-3, e)
    assert ex.value.status == api.EUNSUPPORTED
    # more joints than the node kernel supports
    nb = 14
    chain = {"mass": np.ones(nb), "inertia": np.full(nb, 0.1),
             "joint_parent": np.arange(nb - 1, dtype=np.int32), "joint_child": np.arange(1, nb, dtype=np.int32),
             "joint_rho_parent": np.tile([0.0, -0.1], (nb - 1, 1)), "joint_rho_child": np.tile([0.0, 0.1], (nb - 1, 1)),
             "contact_body": np.zeros(0, dtype=np.int32), "contact_rho": np.zeros((0, 2)),
             "contact_mu": np.zeros(0), "gravity": 9.81}
    mc = api.Model(chain)
    Xc = torch.zeros((n, mc.nxt), dtype=torch.float64, device=dev)
    with pytest.raises(api.CiscvxError) as ex:
        api.node_linearize(mc, Xc, Xc, None, None, 1e-3, [])
    assert ex.value.status == api.EUNSUPPORTED


def test_sweep_nodes_full_size_sampled(env):
    """Every node of the 4096 x 400 sweep (1 642 496 nodes) in one launch, as
    the bench times it; sampled nodes (first, last and 94 random) checked
    against the oracle block by block."""
    torch, oracle, api = env
    dev = torch.device("cuda:0")
    b = synth.cheetah_sweep(seed=0)
    R = b.robots[0].as_dict()
    m = api.Model(b.robots[0])
    Xm = np.concatenate([b.instance(i).X for i in range(len(b))])
    n = Xm.shape[0]
    assert n == 4096 * 401
    rng = np.random.default_rng(77)
    Xp = Xm + 0.1 * rng.standard_normal(Xm.shape)
    Phi = rng.standard_normal((n, 2 * m.nc))
    Gam = rng.uniform(0, 1.5, (n, m.nc))
    e = np.full(m.nc, 0.3)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    out = api.node_linearize(m, t(Xp), t(Xm), t(Phi), t(Gam), 1e-3, e)
    api.sync_status(m)
    sample = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 94, replace=False)]))
    idx = torch.tensor(sample, device=dev)
    got = {k: v[idx].cpu().numpy() for k, v in out.items()}
    ref = oracle.node(R, Xp[sample], Xm[sample], Phi[sample], Gam[sample], 1e-3, e)
    for k, v in _node_errors(got, ref, R).items():
        assert v <= TOL_FP64, (k, v)
