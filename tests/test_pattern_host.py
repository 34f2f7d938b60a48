"""Structural pattern of the compact outputs (ciscvx_model_pattern; host only,
no GPU) against the oracle's dense Jacobians.

The dynamics of Sec. II-A couple the links only through the joint forces,
which are inputs, so A_k is block diagonal per link plus the penalty row of
each contact, and an input enters only the rows of the links it acts on.  The
pattern must (1) contain every entry the oracle finds nonzero, (2) contain no
entry that stays zero on generic inputs (so the compact outputs are as small
as the structure allows), and (3) follow the order the header documents,
rebuilt here from the header's wording alone.
"""
import numpy as np
import pytest

from paper_2604_09993_gb300 import synth


@pytest.fixture(scope="module")
def env():
    import oracle
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return oracle, api


def _robots():
    from test_gpu_discretize import _edge_robots
    rng = np.random.default_rng(21)
    out = {"hopper": synth.hopper(rng), "biped": synth.biped(rng), "cheetah7": synth.cheetah7(rng)}
    out.update(_edge_robots())
    return out


def _as_dict(R):
    return R if isinstance(R, dict) else R.as_dict()


def _documented_order(R):
    """The compact order as the header states it."""
    nb = len(R["mass"])
    jp, jc = np.asarray(R["joint_parent"]), np.asarray(R["joint_child"])
    nj = len(jp)
    cb = list(np.asarray(R["contact_body"]))
    a, b = [], []
    for k in range(nb):
        px, py, th = 3 * k, 3 * k + 1, 3 * k + 2
        vx, vy, om = 3 * nb + 3 * k, 3 * nb + 3 * k + 1, 3 * nb + 3 * k + 2
        y = 6 * nb + cb.index(k) if k in cb else None
        a += [(px, px), (px, vx), (py, py), (py, vy), (th, th), (th, om), (vx, vx), (vy, vy),
              (om, th), (om, om)]
        if y is not None:
            a += [(y, py), (y, th), (y, vy), (y, om), (y, y)]
        inputs = []  # (column, has x force, has y force)
        for j in range(nj):
            if k in (jp[j], jc[j]):
                inputs += [(j, False, False), (nj + 2 * j, True, False), (nj + 2 * j + 1, False, True)]
        if y is not None:
            c0 = 3 * nj + 3 * cb.index(k)
            inputs += [(c0, False, True), (c0 + 1, True, False), (c0 + 2, True, False)]
        for q, fx, fy in inputs:
            rows = ([px] if fx else []) + ([py] if fy else []) + [th] + ([vx] if fx else []) + \
                   ([vy] if fy else []) + [om] + ([y] if y is not None else [])
            b += [(r, q) for r in rows]
    return a, b


@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7", "no_contact", "lone_link"])
def test_pattern_order_and_counts(env, name):
    oracle, api = env
    R = _as_dict(_robots()[name])
    ar, ac, br, bc = api.model_pattern(R)
    a, b = _documented_order(R)
    assert list(zip(ar.tolist(), ac.tolist())) == a
    assert list(zip(br.tolist(), bc.tolist())) == b
    assert len(set(a)) == len(a) and len(set(b)) == len(b)
    nb, nc = len(R["mass"]), len(R["contact_body"])
    assert len(a) == 10 * nb + 5 * nc


@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7", "no_contact", "lone_link"])
def test_pattern_matches_oracle_nonzeros(env, name):
    """Oracle nonzeros (union over intervals) == pattern, on inputs that make
    every penalty term active somewhere (feet below ground, negative forces)."""
    oracle, api = env
    R = _as_dict(_robots()[name])
    nb, nj, nc = len(R["mass"]), len(R["joint_parent"]), len(R["contact_body"])
    nxt, nu = 6 * nb + nc, 3 * nj + 3 * nc
    rng = np.random.default_rng(5)
    N, n_sub = 24, 3
    X = rng.uniform(-0.6, 0.6, (N + 1, nxt))
    X[:, 1:3 * nb:3] = rng.uniform(-0.4, 0.2, (N + 1, nb))  # p_y: contact points straddle y = 0
    U = rng.standard_normal((N + 1, nu))
    s = rng.uniform(0.05, 0.15, N)
    ref = oracle.discretize(R, X, U, s, n_sub)
    ar, ac, br, bc = api.model_pattern(R)
    pa = np.zeros((nxt, nxt), bool)
    pa[ar, ac] = True
    pb = np.zeros((nxt, nu), bool)
    pb[br, bc] = True
    nza = np.any(ref["A"] != 0.0, axis=0)
    nzb = np.any((ref["Bm"] != 0.0) | (ref["Bp"] != 0.0), axis=0)
    assert not np.any(nza & ~pa), np.argwhere(nza & ~pa)[:5]
    assert not np.any(nzb & ~pb), np.argwhere(nzb & ~pb)[:5]
    if name == "lone_link":
        # no input acts on the link: omega' = 0, so (om, th) is a pattern entry that stays 0
        assert np.argwhere(pa & ~nza).tolist() == [[5, 2]]
        pa[5, 2] = False
    assert not np.any(pa & ~nza), np.argwhere(pa & ~nza)[:5]
    assert not np.any(pb & ~nzb), np.argwhere(pb & ~nzb)[:5]
    # B- and B+ are each nonzero on the whole pattern too
    assert np.all(np.any(ref["Bm"] != 0.0, axis=0)[pb])
    assert np.all(np.any(ref["Bp"] != 0.0, axis=0)[pb])


def test_pattern_rejects_invalid_descriptions(env):
    oracle, api = env
    R = _as_dict(_robots()["hopper"])
    bad = dict(R, joint_parent=np.array([7, 1], dtype=np.int32))
    with pytest.raises(api.CiscvxError) as e:
        api.model_pattern(bad)
    assert e.value.status == api.EINVAL
    two = dict(R, contact_body=np.array([2, 2], dtype=np.int32), contact_rho=np.zeros((2, 2)),
               contact_mu=np.ones(2))
    with pytest.raises(api.CiscvxError) as e:
        api.model_pattern(two)
    assert e.value.status == api.EUNSUPPORTED
