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
    # the Eq. (12) auxiliary state: four cross-complementarity rows per contact
    for name in ("hopper", "biped", "cheetah7"):
        out[name + "_cross"] = synth.with_cross_states(out[name])
    return out


def _as_dict(R):
    return R if isinstance(R, dict) else R.as_dict()


def _documented_order(R):
    """The compact order as the header states it."""
    nb = len(R["mass"])
    jp, jc = np.asarray(R["joint_parent"]), np.asarray(R["joint_child"])
    nj = len(jp)
    cb = list(np.asarray(R["contact_body"]))
    nc = len(cb)
    cross = bool(R.get("aux_model", 0))
    a, b = [], []
    for k in range(nb):
        px, py, th = 3 * k, 3 * k + 1, 3 * k + 2
        vx, vy, om = 3 * nb + 3 * k, 3 * nb + 3 * k + 1, 3 * nb + 3 * k + 2
        foot = k in cb
        # the contact's path-penalty row comes after the 4 n_c cross rows in the Eq. (12) model
        y = 6 * nb + (4 * nc if cross else 0) + cb.index(k) if foot else None
        a += [(px, px), (px, vx), (py, py), (py, vy), (th, th), (th, om), (vx, vx), (vy, vy),
              (om, th), (om, om)]
        if foot:
            a += [(y, py), (y, th), (y, vy), (y, om), (y, y)]
        inputs = []  # (column, x force, y force, torque, enters lambda^c directly)
        for j in range(nj):
            if k in (jp[j], jc[j]):
                inputs += [(j, False, False, True, False), (nj + 2 * j, True, False, True, False),
                           (nj + 2 * j + 1, False, True, True, False)]
        if foot:
            c0 = 3 * nj + 3 * cb.index(k)
            if cross:   # phi_t (x force), phi_n (y force), gamma (no force)
                inputs += [(c0, True, False, True, True), (c0 + 1, False, True, True, False),
                           (c0 + 2, False, False, False, True)]
            else:       # lambda_n (y), lambda_t+ (x), lambda_t- (x)
                inputs += [(c0, False, True, True, False), (c0 + 1, True, False, True, False),
                           (c0 + 2, True, False, True, False)]
        for q, fx, fy, tq, _ in inputs:
            rows = ([px] if fx else []) + ([py] if fy else []) + ([th] if tq else []) + \
                   ([vx] if fx else []) + ([vy] if fy else []) + ([om] if tq else []) + \
                   ([y] if foot else [])
            b += [(r, q) for r in rows]
        if foot and cross:   # rows phi_n, lambda^c, gamma, rho^c of the contact
            r0 = 6 * nb + 4 * cb.index(k)
            a += [(r0, r0), (r0 + 1, r0 + 1), (r0 + 2, r0 + 2), (r0 + 3, r0 + 3),
                  (r0 + 1, vx), (r0 + 1, th), (r0 + 1, om)]
            b += [(r0 + 1, q) for q, fx, fy, tq, direct in inputs if fx or tq or direct]
            c0 = 3 * nj + 3 * cb.index(k)
            b += [(r0, c0 + 1), (r0 + 2, c0 + 2), (r0 + 3, c0), (r0 + 3, c0 + 1)]
    return a, b


NAMES = ["hopper", "biped", "cheetah7", "no_contact", "lone_link", "hopper_cross", "biped_cross",
         "cheetah7_cross"]


@pytest.mark.parametrize("name", NAMES)
def test_pattern_order_and_counts(env, name):
    oracle, api = env
    R = _as_dict(_robots()[name])
    ar, ac, br, bc = api.model_pattern(R)
    a, b = _documented_order(R)
    assert list(zip(ar.tolist(), ac.tolist())) == a
    assert list(zip(br.tolist(), bc.tolist())) == b
    assert len(set(a)) == len(a) and len(set(b)) == len(b)
    nb, nc = len(R["mass"]), len(R["contact_body"])
    assert len(a) == 10 * nb + (12 if R.get("aux_model", 0) else 5) * nc


@pytest.mark.parametrize("name", NAMES)
def test_pattern_matches_oracle_nonzeros(env, name):
    """Oracle nonzeros (union over intervals) == pattern, on inputs that make
    every penalty term active somewhere (feet below ground, negative forces)."""
    oracle, api = env
    R = _as_dict(_robots()[name])
    nb, nj, nc = len(R["mass"]), len(R["joint_parent"]), len(R["contact_body"])
    nxt, nu = 6 * nb + (5 if R.get("aux_model", 0) else 1) * nc, 3 * nj + 3 * nc
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


def _coupled_robots():
    rng = np.random.default_rng(23)
    hop, bip = synth.hopper(rng), synth.biped(rng)
    return {"hopper_paper": synth.with_paper_dynamics(hop, joint_forces=1, scheme=1,
                                                      terrain=synth.TERRAIN_SINE),
            "biped_paper_cross": synth.with_cross_states(synth.with_paper_dynamics(bip, joint_forces=1,
                                                                                   scheme=1)),
            "biped_sine": synth.with_paper_dynamics(bip, joint_forces=0, scheme=0,
                                                    terrain=synth.TERRAIN_SINE)}


def _coupled_documented_order(R):
    """The column-major order the header states for models with coupled links."""
    nb = len(R["mass"])
    nj, nc = len(R["joint_parent"]), len(R["contact_body"])
    cb = list(np.asarray(R["contact_body"]))
    cross = bool(R.get("aux_model", 0))
    nxt = 6 * nb + (5 if cross else 1) * nc
    nu = (1 if R.get("joint_forces", 0) else 3) * nj + 3 * nc
    a = []
    for c in range(nxt):
        if c >= 6 * nb:
            a.append((c, c))
            continue
        body = (c % (3 * nb)) // 3
        if body in cb or c % 3 == 2:
            a += [(r, c) for r in range(nxt)]
        elif c < 3 * nb:
            a.append((c, c))
        else:
            a += [(c - 3 * nb, c), (c, c)]
    b = [(r, q) for q in range(nu) for r in range(nxt)]
    return a, b, nxt, nu


@pytest.mark.parametrize("name", ["hopper_paper", "biped_paper_cross", "biped_sine"])
def test_coupled_pattern_order_and_oracle_nonzeros(env, name):
    """Models with coupled links: the pattern follows the documented
    column-major order and holds every entry the oracle finds nonzero; the
    entries off it (the closed-form columns' other rows) are exactly zero in
    the oracle's blocks."""
    oracle, api = env
    R = _as_dict(_coupled_robots()[name])
    ar, ac, br, bc = api.model_pattern(R)
    a, b, nxt, nu = _coupled_documented_order(R)
    assert list(zip(ar.tolist(), ac.tolist())) == a
    assert list(zip(br.tolist(), bc.tolist())) == b
    nb = len(R["mass"])
    rng = np.random.default_rng(6)
    N, n_sub = 5, 2
    X = rng.uniform(-0.6, 0.6, (N + 1, nxt))
    X[:, 1:3 * nb:3] = rng.uniform(-0.4, 0.2, (N + 1, nb))
    U = rng.standard_normal((N + 1, nu))
    s = rng.uniform(0.05, 0.15, N)
    ref = oracle.discretize(R, X, U, s, n_sub)
    pa = np.zeros((nxt, nxt), bool)
    pa[ar, ac] = True
    nza = np.any(ref["A"] != 0.0, axis=0)
    assert not np.any(nza & ~pa), np.argwhere(nza & ~pa)[:5]
    # the closed-form columns: A e_p = e_p, A e_v = e_v + s e_p, A e_y = e_y
    for c in range(nxt):
        if pa[:, c].sum() < nxt:
            rows = np.flatnonzero(pa[:, c])
            assert np.all(ref["A"][:, rows[-1], c] == 1.0)
            if len(rows) == 2:
                assert np.allclose(ref["A"][:, rows[0], c], s, rtol=0, atol=1e-15)
