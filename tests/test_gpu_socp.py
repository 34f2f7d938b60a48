"""GPU parity of the SOCP canonicalization (ciscvx_socp_*) against the oracle's
dense assembly of the same subproblem.

The GPU path linearizes on the GPU (ciscvx_discretize at X = Xp,
ciscvx_node_linearize, ciscvx_psi_linearize) and canonicalizes; the oracle
linearizes with its dual numbers and assembles densely from the definition.
A, b, G, h, P, c and the row scales are compared entry by entry
(block-normwise relative 1e-10 for FP64 inputs), for both auxiliary models,
both control layouts, the sinusoidal surface and the paper's dynamics, and
for several instances filled in one call.  The CSC structure is checked to be
well formed.
"""
import numpy as np
import pytest

from _util import TOL_FP64, TOL_FP32_PHI, block_err
from paper_2604_09993_gb300 import synth

pytestmark = pytest.mark.gpu

NSUB, DELTA, EPS = 4, 0.05, 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    import oracle
    from oracle import socp as osocp
    from paper_2604_09993_gb300 import api, build
    build.build()
    oracle.build()
    api.load()
    return torch, oracle, osocp, api


def _robot(name, variant):
    rng = np.random.default_rng(17)
    R = getattr(synth, name)(rng)
    if variant == "cross":
        R = synth.with_cross_states(R)
    elif variant == "sine":
        R = synth.with_paper_dynamics(R, joint_forces=0, scheme=0, terrain=synth.TERRAIN_SINE)
    elif variant == "paper":
        R = synth.with_cross_states(synth.with_paper_dynamics(R, terrain=synth.TERRAIN_SINE))
    return R.as_dict()


def _iterate(m, N, layout, rng):
    nxt, nu, nb, nc = m.nxt, m.nu, m.nb, m.nc
    Xp = np.zeros((N + 1, nxt))
    Xp[:, : 6 * nb] = rng.uniform(-0.3, 0.3, (N + 1, 6 * nb))
    Xp[:, 6 * nb:] = rng.uniform(-0.5, 0.5, (N + 1, nxt - 6 * nb))
    Xm = Xp + 0.05 * rng.standard_normal(Xp.shape)
    U = rng.standard_normal((N + 1, nu) if layout == "node" else (N, 2, nu))
    s = rng.uniform(0.05, 0.15, N)
    Phi = rng.standard_normal((N + 1, 2 * nc))
    Gam = rng.uniform(0.1, 1.0, (N + 1, nc))
    return Xp, Xm, U, s, Phi, Gam


def _params(m, rng, scaled=True):
    nb, nj, nc, nxt, nu = m.nb, m.nj, m.nc, m.nxt, m.nu
    prm = {"w_px": 3.0, "w_ep": 50.0, "w_torque": 0.7, "s_min": 0.02, "s_max": 0.3,
           "torque_max": rng.uniform(2, 4, nj), "x_init": rng.uniform(-0.2, 0.2, 6 * nb),
           "x_final": rng.uniform(-0.2, 0.2, 6 * nb)}
    if scaled:
        prm.update(scale_x=rng.uniform(0.5, 2, nxt), offset_x=rng.uniform(-0.1, 0.1, nxt),
                   scale_u=rng.uniform(0.5, 2, nu), offset_u=rng.uniform(-0.1, 0.1, nu),
                   scale_s=0.1, offset_s=0.05, scale_phi=rng.uniform(0.5, 2, 2 * nc),
                   offset_phi=rng.uniform(-0.1, 0.1, 2 * nc), scale_gam=rng.uniform(0.5, 2, nc),
                   offset_gam=rng.uniform(-0.1, 0.1, nc))
    return prm


def _socp(api, m, N, layout, prm):
    scaling = {k: (prm.get(f"scale_{k}"), prm.get(f"offset_{k}")) for k in ("x", "u", "phi", "gam")}
    scaling["s"] = (prm.get("scale_s", 0.0), prm.get("offset_s", 0.0))
    return api.Socp(m, N, layout, w_px=prm["w_px"], w_ep=prm["w_ep"], w_torque=prm["w_torque"],
                    s_min=prm["s_min"], s_max=prm["s_max"], torque_max=prm["torque_max"],
                    x_init=prm["x_init"], x_final=prm["x_final"], scaling=scaling)


def _linearize(torch, api, m, layout, its, precision):
    """GPU linearization of several iterates, concatenated per instance."""
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)  # noqa: E731
    cat = {}
    for Xp, Xm, U, s, Phi, Gam in its:
        d = api.discretize(m, t(Xp), t(U), t(s), NSUB, precision, layout)
        e = np.full(m.nc, 0.4)
        nd = api.node_linearize(m, t(Xp), t(Xm), t(Phi.reshape(-1, 2 * m.nc)), t(Gam.reshape(-1, m.nc)), DELTA, e)
        ps = api.psi_linearize(m, t(Xp), t(Xm), DELTA, EPS)
        parts = {"Xp": t(Xp), "Xm": t(Xm), "U": t(U), "s": t(s), "Phi": t(Phi), "Gam": t(Gam),
                 "A": d["A"], "Bm": d["Bm"], "Bp": d["Bp"], "S": d["S"], "defect": d["defect"],
                 "g": nd["g"], "Gvm": nd["Gvm"], "Gth": nd["Gth"], "Gphi": nd["Gphi"], "Gpx": nd["Gpx"],
                 "theta": nd["theta"], "dtheta": nd["dtheta"], "psi": ps["psi"], "dpsi": ps["dpsi"]}
        for k, v in parts.items():
            cat.setdefault(k, []).append(v.reshape(-1))
    return {k: torch.cat(v).contiguous() for k, v in cat.items()}


def _dense(colptr, rowind, vals, nrow, ncol):
    M = np.zeros((nrow, ncol))
    for c in range(ncol):
        for e in range(colptr[c], colptr[c + 1]):
            M[rowind[e], c] = vals[e]
    return M


def _check_structure(st, dims):
    for key, nnz, nrow in (("A", dims["nnz_A"], dims["n_eq"]), ("G", dims["nnz_G"], dims["n_ineq"]),
                           ("P", dims["nnz_P"], dims["n_var"])):
        cp, ri = st[f"{key}_colptr"], st[f"{key}_rowind"]
        assert cp[0] == 0 and cp[-1] == nnz and np.all(np.diff(cp) >= 0)
        for c in range(dims["n_var"]):
            rows = ri[cp[c]:cp[c + 1]]
            assert np.all(np.diff(rows) > 0) and (len(rows) == 0 or (rows[0] >= 0 and rows[-1] < nrow))
            if key == "P":
                assert len(rows) == 0 or rows[-1] <= c


CASES = [("hopper", "default", "node"), ("hopper", "cross", "interval"), ("biped", "default", "interval"),
         ("biped", "cross", "node"), ("cheetah7", "default", "node"), ("hopper", "sine", "node"),
         ("hopper", "paper", "interval")]


@pytest.mark.parametrize("name,variant,layout", CASES)
def test_socp_parity(env, name, variant, layout):
    torch, oracle, osocp, api = env
    R = _robot(name, variant)
    m = api.Model(R)
    rng = np.random.default_rng(5)
    N, n_inst = 3, 2
    prm = _params(m, rng)
    its = [_iterate(m, N, layout, rng) for _ in range(n_inst)]
    sp = _socp(api, m, N, layout, prm)
    dims = sp.dims
    st = sp.structure()
    _check_structure(st, dims)
    out = sp.fill(n_inst, _linearize(torch, api, m, layout, its, "fp64"))
    api.sync_status(m)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    for i, (Xp, Xm, U, s, Phi, Gam) in enumerate(its):
        ref = osocp.assemble(R, N, layout, prm, Xp, Xm, U, s, Phi, Gam, NSUB, DELTA, EPS, np.full(m.nc, 0.4))
        assert (dims["n_var"], dims["n_eq"], dims["n_ineq"]) == (len(ref["c"]), len(ref["b"]), len(ref["h"]))
        assert (dims["n_nonneg"], dims["n_soc"]) == (ref["n_nonneg"], ref["n_soc"])
        nv = dims["n_var"]
        A = _dense(st["A_colptr"], st["A_rowind"], out["A_values"][i], dims["n_eq"], nv)
        G = _dense(st["G_colptr"], st["G_rowind"], out["G_values"][i], dims["n_ineq"], nv)
        P = _dense(st["P_colptr"], st["P_rowind"], st["P_values"], nv, nv)
        P = P + np.triu(P, 1).T
        for got, want in ((A, ref["A"]), (out["b"][i], ref["b"]), (G, ref["G"]), (out["h"][i], ref["h"]),
                          (P, ref["P"]), (out["c"][i], ref["c"]), (out["rho_A"][i], ref["rho_A"]),
                          (out["rho_G"][i], ref["rho_G"])):
            assert block_err(got, want) <= TOL_FP64


def test_socp_fp32_phi_inputs(env):
    torch, oracle, osocp, api = env
    R = _robot("cheetah7", "default")
    m = api.Model(R)
    rng = np.random.default_rng(6)
    N = 4
    prm = _params(m, rng, scaled=False)
    it = _iterate(m, N, "node", rng)
    sp = _socp(api, m, N, "node", prm)
    st = sp.structure()
    out = sp.fill(1, _linearize(torch, api, m, "node", [it], "fp32_phi"), precision="fp32_phi")
    out = {k: v.cpu().numpy() for k, v in out.items()}
    ref = osocp.assemble(R, N, "node", prm, *it, NSUB, DELTA, EPS, np.full(m.nc, 0.4))
    d = sp.dims
    A = _dense(st["A_colptr"], st["A_rowind"], out["A_values"][0], d["n_eq"], d["n_var"])
    assert block_err(A, ref["A"]) <= TOL_FP32_PHI
    assert block_err(out["b"][0], ref["b"]) <= TOL_FP32_PHI
    G = _dense(st["G_colptr"], st["G_rowind"], out["G_values"][0], d["n_ineq"], d["n_var"])
    assert block_err(G, ref["G"]) <= TOL_FP64   # G takes no Phi block


def test_socp_arguments(env):
    torch, oracle, osocp, api = env
    R = _robot("hopper", "default")
    m = api.Model(R)
    rng = np.random.default_rng(1)
    prm = _params(m, rng)
    lib = api.load()
    for bad in ({"w_px": 0.0}, {"w_ep": -1.0}, {"s_min": 0.5, "s_max": 0.1},
                {"torque_max": np.zeros(m.nj)}, {"x_init": np.full(6 * m.nb, np.nan)}):
        with pytest.raises(Exception):
            _socp(api, m, 3, "node", dict(prm, **bad))
    with pytest.raises(Exception):
        _socp(api, m, 0, "node", prm)
    sp = _socp(api, m, 3, "node", prm)
    ins = api._SocpInputs()
    outs = api._SocpOutputs()
    import ctypes
    assert lib.ciscvx_socp_fill(sp._h, 1, ctypes.byref(ins), ctypes.byref(outs), None) == api.EINVAL
    assert lib.ciscvx_socp_fill(sp._h, 0, ctypes.byref(ins), ctypes.byref(outs), None) == api.EINVAL


def test_socp_sweep_size_sampled_periods(env):
    """N = 400 intervals of the 7-link chain, 64 instances in one call (the
    bench's per-instance size).  The rows of period k touch periods k and k+1
    only, so the oracle's assembly of the 2-interval slice starting at node k
    gives them exactly (columns shifted by the periods before k); sampled
    periods of sampled instances are compared row by row, with their scales
    and right-hand sides."""
    import scipy.sparse as sps
    torch, oracle, osocp, api = env
    R = _robot("cheetah7", "default")
    m = api.Model(R)
    rng = np.random.default_rng(8)
    N, n_inst, layout = 400, 64, "node"
    prm = _params(m, rng)
    its = [_iterate(m, N, layout, rng) for _ in range(n_inst)]
    sp = _socp(api, m, N, layout, prm)
    st, d = sp.structure(), sp.dims
    out = sp.fill(n_inst, _linearize(torch, api, m, layout, its, "fp64"))
    api.sync_status(m)
    Lf = osocp.Layout(R, N, layout)
    Ls = osocp.Layout(R, 2, layout)
    per_col = Ls.col["xm", 1][0] - Ls.col["xm", 0][0]
    nA_per = 2 * m.nxt
    nG_node = 16 * m.nc + 2 * m.nxt + 2 * m.nj + 4 * m.nc
    nG_int = 2 * api.psi_rows(m) + 2 * m.nxt + 2
    for inst in (0, 37, 63):
        Xp, Xm, U, s, Phi, Gam = its[inst]
        A = sps.csc_matrix((out["A_values"][inst].cpu().numpy(), st["A_rowind"], st["A_colptr"]),
                           shape=(d["n_eq"], d["n_var"])).tocsr()
        G = sps.csc_matrix((out["G_values"][inst].cpu().numpy(), st["G_rowind"], st["G_colptr"]),
                           shape=(d["n_ineq"], d["n_var"])).tocsr()
        b, h = out["b"][inst].cpu().numpy(), out["h"][inst].cpu().numpy()
        rA, rG = out["rho_A"][inst].cpu().numpy(), out["rho_G"][inst].cpu().numpy()
        for k in (0, 1, 199, N - 2):
            sl = slice(k, k + 3)
            ref = osocp.assemble(R, 2, layout, prm, Xp[sl], Xm[sl], U[sl], s[k:k + 2], Phi[sl], Gam[sl],
                                 NSUB, DELTA, EPS, np.full(m.nc, 0.4))
            shift = Lf.col["xm", k][0] - Ls.col["xm", 0][0]
            ncols = 2 * per_col
            for M, vec, rho, rows_f, rows_s, Mr, vr, rr in (
                    (A, b, rA, slice(k * nA_per, (k + 1) * nA_per), slice(0, nA_per), ref["A"], ref["b"], ref["rho_A"]),
                    (G, h, rG, slice(k * (nG_node + nG_int), (k + 1) * (nG_node + nG_int)), slice(0, nG_node + nG_int),
                     ref["G"], ref["h"], ref["rho_G"])):
                got = M[rows_f].toarray()
                assert np.abs(got[:, :shift]).max(initial=0) == 0
                assert np.abs(got[:, shift + ncols:]).max(initial=0) == 0
                assert block_err(got[:, shift:shift + ncols], Mr[rows_s, :ncols]) <= TOL_FP64
                assert block_err(vec[rows_f], vr[rows_s]) <= TOL_FP64
                assert block_err(rho[rows_f], rr[rows_s]) <= TOL_FP64


def test_socp_fp32_inputs_widen_exactly(env):
    """FP32 Phi blocks are widened exactly: the fill from FP32 blocks equals,
    bit for bit, the fill from the same blocks converted to FP64 by torch
    (zeros, negative values and values of every magnitude included)."""
    torch, oracle, osocp, api = env
    R = _robot("biped", "cross")
    m = api.Model(R)
    rng = np.random.default_rng(12)
    N = 5
    prm = _params(m, rng)
    it = _iterate(m, N, "interval", rng)
    sp = _socp(api, m, N, "interval", prm)
    ins = _linearize(torch, api, m, "interval", [it], "fp32_phi")
    gen = torch.Generator(device=ins["A"].device).manual_seed(3)
    for k in ("A", "Bm", "Bp", "S"):  # spread the magnitudes and plant exact zeros
        t = ins[k]
        scale = torch.pow(2.0, torch.randint(-60, 60, t.shape, generator=gen, device=t.device).float())
        ins[k] = torch.where(torch.rand(t.shape, generator=gen, device=t.device) < 0.1,
                             torch.zeros_like(t), t * scale).contiguous()
    o32 = sp.fill(1, ins, precision="fp32_phi")
    ins64 = dict(ins, **{k: ins[k].double() for k in ("A", "Bm", "Bp", "S")})
    o64 = sp.fill(1, ins64, precision="fp64")
    for k in o32:
        assert torch.equal(o32[k], o64[k]), k


@pytest.mark.parametrize("precision", ["fp64", "fp32_phi"])
@pytest.mark.parametrize("layout,variant", [("node", "default"), ("interval", "default"), ("node", "cross"),
                                            ("node", "paper"), ("interval", "sine")])
def test_socp_from_compact_outputs(env, precision, layout, variant):
    """The fill from compact A / B- / B+ (ciscvx_discretize_compact) equals the
    fill from the dense blocks bit for bit: the same values feed the same
    arithmetic, only their addresses differ."""
    torch, oracle, osocp, api = env
    R = _robot("biped", variant)
    m = api.Model(R)
    rng = np.random.default_rng(21)
    N, n_inst = 7, 3
    prm = _params(m, rng)
    its = [_iterate(m, N, layout, rng) for _ in range(n_inst)]
    dense = _linearize(torch, api, m, layout, its, precision)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)  # noqa: E731
    comp = dict(dense)
    parts = {"A": [], "Bm": [], "Bp": []}
    for Xp, Xm, U, s, Phi, Gam in its:
        c = api.discretize_compact(m, t(Xp), t(U), t(s), NSUB, precision, layout)
        for k in parts:
            parts[k].append(c[k].reshape(-1))
    for k in parts:
        comp[k] = torch.cat(parts[k]).contiguous()
    sd = _socp(api, m, N, layout, prm)
    scaling = {k: (prm.get(f"scale_{k}"), prm.get(f"offset_{k}")) for k in ("x", "u", "phi", "gam")}
    scaling["s"] = (prm.get("scale_s", 0.0), prm.get("offset_s", 0.0))
    sc = api.Socp(m, N, layout, w_px=prm["w_px"], w_ep=prm["w_ep"], w_torque=prm["w_torque"],
                  s_min=prm["s_min"], s_max=prm["s_max"], torque_max=prm["torque_max"],
                  x_init=prm["x_init"], x_final=prm["x_final"], scaling=scaling, phi_format="compact")
    assert sc.dims == sd.dims
    o_d = sd.fill(n_inst, dense, precision=precision)
    o_c = sc.fill(n_inst, comp, precision=precision)
    for k in o_d:
        assert torch.equal(o_d[k], o_c[k]), k
