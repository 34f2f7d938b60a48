"""TEST INFRASTRUCTURE ONLY: the SCP subproblem assembled as a canonical SOCP,
written out densely from its definition.

Sec. V: each prox-linear SCP iteration linearizes the nonconvex constraints
of the CITO problem (Eq. (17)) at the iterate zbar, penalizes their violation
with an exact l1 penalty, keeps the convex constraints, and adds a quadratic
proximal term.  Sec. VI: the result is put in the canonical form of a conic
solver (A z = b, h - G z in a product of the nonnegative orthant and
second-order cones, objective 1/2 z^T P z + c^T z), with an affine scaling of
the variables and a row-wise normalization of the constraint matrices.

The linearizations come from this package's own dual-number Jacobians
(``discretize`` at X = the post-impact states, ``node``, ``psi``); the
variable and row order, the convex set U and the objective are the ones the
library's header states for ``ciscvx_socp_*``.  Everything here is dense
numpy in FP64, one row at a time, for small N only.
"""
import numpy as np

from . import oracle as _o


class Layout:
    """Column and row indices of the subproblem's variables and constraints."""

    def __init__(self, R, N, layout):
        m = _o._model(R)
        self.nb, self.nj, self.nc, self.nxt, self.nu = m.nb, m.nj, m.nc, m.nxt, m.nu
        self.aux, self.jelim = bool(m.aux), bool(m.jelim)
        self.ny = self.nxt - 6 * self.nb
        self.nx = 6 * self.nb
        self.npsi = 3 * self.nc if self.aux else self.nc
        self.N, self.node = N, layout in ("node", 0)
        self.mu = np.asarray(R["contact_mu"], dtype=np.float64).reshape(-1)
        nxt, nu, nc = self.nxt, self.nu, self.nc
        self.col = {}
        self.problem = []        # column ranges of problem variables, with their kind
        c = 0

        def take(name, k, n, kind=None):
            nonlocal c
            self.col[name, k] = np.arange(c, c + n)
            if kind is not None:
                self.problem.append((kind, c, n))
            c += n

        for k in range(N + 1):
            take("xm", k, nxt, "x")
            take("xp", k, nxt, "x")
            take("phi", k, 2 * nc, "phi")
            take("gam", k, nc, "gam")
            if self.node:
                take("u", k, nu, "u")
            take("nuGp", k, nxt)
            take("nuGm", k, nxt)
            take("tth", k, 8 * nc)
            if k < N:
                if not self.node:
                    take("uL", k, nu, "u")
                    take("uR", k, nu, "u")
                take("s", k, 1, "s")
                take("nuFp", k, nxt)
                take("nuFm", k, nxt)
                take("tpsi", k, self.npsi)
        self.n_var = c
        self.is_problem = np.zeros(c, dtype=bool)
        for _, c0, n in self.problem:
            self.is_problem[c0:c0 + n] = True

    def uL(self, k):
        return self.col["u", k] if self.node else self.col["uL", k]

    def uR(self, k):
        return self.col["u", k + 1] if self.node else self.col["uR", k]

    def controls(self):
        """Control vectors in the order their input rows and cones appear, per period."""
        out = []
        for k in range(self.N + 1):
            if self.node:
                out.append((k, "node", self.col["u", k]))
            elif k < self.N:
                out.append((k, "interval", self.col["uL", k]))
                out.append((k, "interval", self.col["uR", k]))
        return out

    def contact_inputs(self, ucols, i):
        c0 = (1 if self.jelim else 3) * self.nj + 3 * i
        return ucols[c0], ucols[c0 + 1], ucols[c0 + 2]


def _iterate(L, Xp, Xm, U, s, Phi, Gam):
    z = np.zeros(L.n_var)
    for k in range(L.N + 1):
        z[L.col["xp", k]] = Xp[k]
        z[L.col["xm", k]] = Xm[k]
        if L.nc:
            z[L.col["phi", k]] = Phi[k]
            z[L.col["gam", k]] = Gam[k]
        if L.node:
            z[L.col["u", k]] = U[k]
        if k < L.N:
            if not L.node:
                z[L.col["uL", k]] = U[k, 0]
                z[L.col["uR", k]] = U[k, 1]
            z[L.col["s", k]] = s[k]
    return z


def _scaling(L, prm):
    D, o = np.ones(L.n_var), np.zeros(L.n_var)
    per = {"x": ("scale_x", "offset_x", L.nxt), "u": ("scale_u", "offset_u", L.nu),
           "phi": ("scale_phi", "offset_phi", 2 * L.nc), "gam": ("scale_gam", "offset_gam", L.nc)}
    for kind, c0, n in L.problem:
        if kind == "s":
            D[c0] = prm.get("scale_s", 1.0) or 1.0
            o[c0] = prm.get("offset_s", 0.0)
            continue
        ks, ko, _ = per[kind]
        if prm.get(ks) is not None:
            D[c0:c0 + n] = prm[ks]
        if prm.get(ko) is not None:
            o[c0:c0 + n] = prm[ko]
    return D, o


def assemble(R, N, layout, prm, Xp, Xm, U, s, Phi, Gam, n_sub, delta, eps, restitution):
    """Dense canonical SOCP at the iterate (Xp, Xm, U, s, Phi, Gam).

    prm: dict with w_px, w_ep, w_torque, s_min, s_max, torque_max [nj],
    x_init [nx], x_final [nx] and optional scale_*/offset_* vectors.
    Returns dict A, b, G, h, P, c (scaled and normalized), rho_A, rho_G,
    n_nonneg, n_soc, D, o, zbar, layout, and the unscaled parts A0, b0, G0, h0."""
    L = Layout(R, N, layout)
    nxt, nc, nj, nx, ny = L.nxt, L.nc, L.nj, L.nx, L.ny
    Xp, Xm, U, s = (np.asarray(a, dtype=np.float64) for a in (Xp, Xm, U, s))
    Phi = np.asarray(Phi, dtype=np.float64).reshape(N + 1, 2 * nc)
    Gam = np.asarray(Gam, dtype=np.float64).reshape(N + 1, nc)
    zbar = _iterate(L, Xp, Xm, U, s, Phi, Gam)
    lin = _o.discretize(R, Xp, U, s, n_sub, layout)
    nd = _o.node(R, Xp, Xm, Phi, Gam, delta, restitution)
    ps = _o.psi(R, Xp, Xm, delta, eps) if nc else None

    A_rows, b_rows, G_rows, h_rows, soc_rows = [], [], [], [], []

    def row():
        return np.zeros(L.n_var)

    def node_cols(k):
        return np.concatenate([L.col["xp", k], L.col["xm", k], L.col["phi", k], L.col["gam", k]])

    def input_rows(ucols):
        for j in range(nj):
            for sg in (1.0, -1.0):
                r = row()
                r[ucols[j]] = sg
                G_rows.append(r)
                h_rows.append(prm["torque_max"][j])
        for i in range(nc):
            a, b_, c_ = L.contact_inputs(ucols, i)
            if L.aux:
                r = row()
                r[c_] = -1.0          # -gamma <= 0
                G_rows.append(r)
                h_rows.append(0.0)
            else:
                for col in (a, b_, c_):  # -lambda_n, -lambda_t+, -lambda_t- <= 0
                    r = row()
                    r[col] = -1.0
                    G_rows.append(r)
                    h_rows.append(0.0)
                r = row()             # lambda_t+ + lambda_t- - mu lambda_n <= 0
                r[b_] = 1.0
                r[c_] = 1.0
                r[a] = -L.mu[i]
                G_rows.append(r)
                h_rows.append(0.0)

    for k in range(N + 1):
        # G~ rows of node k (equality, penalized)
        cols = node_cols(k)
        for r_ in range(nxt):
            r = row()
            r[cols] = nd["Jg"][k, r_]
            jz = r @ zbar
            r[L.col["nuGp", k][r_]] -= 1.0
            r[L.col["nuGm", k][r_]] += 1.0
            A_rows.append(r)
            b_rows.append(jz - nd["g"][k, r_])
        # dynamics rows of interval k
        if k < N:
            uL, uR = L.uL(k), L.uR(k)
            for r_ in range(nxt):
                r = row()
                r[L.col["xp", k]] += lin["A"][k, r_]
                r[uL] += lin["Bm"][k, r_]
                r[uR] += lin["Bp"][k, r_]
                r[L.col["s", k][0]] += lin["S"][k, r_]
                jz = r @ zbar
                r[L.col["xm", k + 1][r_]] -= 1.0
                r[L.col["nuFp", k][r_]] -= 1.0
                r[L.col["nuFm", k][r_]] += 1.0
                A_rows.append(r)
                b_rows.append(jz - (lin["defect"][k, r_] + Xp[k + 1, r_]))
        # nonnegative rows of period k: Theta, its slacks, nuG slacks, inputs of u_k
        for r_ in range(8 * nc):
            r = row()
            r[cols] = nd["Jth"][k, r_]
            hz = r @ zbar - nd["theta"][k, r_]
            r[L.col["tth", k][r_]] = -1.0
            G_rows.append(r)
            h_rows.append(hz)
        for r_ in range(8 * nc):
            r = row()
            r[L.col["tth", k][r_]] = -1.0
            G_rows.append(r)
            h_rows.append(0.0)
        for name in ("nuGp", "nuGm"):
            for r_ in range(nxt):
                r = row()
                r[L.col[name, k][r_]] = -1.0
                G_rows.append(r)
                h_rows.append(0.0)
        if L.node:
            input_rows(L.col["u", k])
        if k < N:
            yp = L.col["xp", k][nx:]
            ym = L.col["xm", k + 1][nx:]
            for r_ in range(L.npsi):
                r = row()
                r[yp] += ps["J"][k, r_, :ny]
                r[ym] += ps["J"][k, r_, ny:]
                hz = r @ zbar - ps["psi"][k, r_]
                r[L.col["tpsi", k][r_]] = -1.0
                G_rows.append(r)
                h_rows.append(hz)
            for r_ in range(L.npsi):
                r = row()
                r[L.col["tpsi", k][r_]] = -1.0
                G_rows.append(r)
                h_rows.append(0.0)
            for name in ("nuFp", "nuFm"):
                for r_ in range(nxt):
                    r = row()
                    r[L.col[name, k][r_]] = -1.0
                    G_rows.append(r)
                    h_rows.append(0.0)
            r = row()
            r[L.col["s", k][0]] = 1.0
            G_rows.append(r)
            h_rows.append(prm["s_max"])
            r = row()
            r[L.col["s", k][0]] = -1.0
            G_rows.append(r)
            h_rows.append(-prm["s_min"])
            if not L.node:
                input_rows(L.col["uL", k])
                input_rows(L.col["uR", k])
    # boundary conditions x-_0 = x_init, x+_N = x_final (Eq. (17g))
    for cols, val in ((L.col["xm", 0][:nx], prm["x_init"]), (L.col["xp", N][:nx], prm["x_final"])):
        for r_ in range(nx):
            r = row()
            r[cols[r_]] = 1.0
            A_rows.append(r)
            b_rows.append(val[r_])
    n_nonneg = len(G_rows)
    # friction cones (Eq. (12) contact model): (mu phi_n, phi_t) in Q^2
    n_soc = 0
    if L.aux:
        for _, _, ucols in L.controls():
            for i in range(nc):
                pt, pn, _ = L.contact_inputs(ucols, i)
                r0, r1 = row(), row()
                r0[pn] = -L.mu[i]
                r1[pt] = -1.0
                G_rows += [r0, r1]
                h_rows += [0.0, 0.0]
                n_soc += 1

    A0, b0 = np.array(A_rows), np.array(b_rows)
    G0, h0 = np.array(G_rows).reshape(-1, L.n_var), np.array(h_rows)

    # objective: proximal term, torque cost of the FOH torques, exact penalty
    P0 = np.zeros((L.n_var, L.n_var))
    c0 = np.zeros(L.n_var)
    prob = np.nonzero(L.is_problem)[0]
    P0[prob, prob] = prm["w_px"]
    c0[L.is_problem] = -prm["w_px"] * zbar[L.is_problem]
    c0[~L.is_problem] = prm["w_ep"]
    w = prm["w_torque"]
    for k in range(N):
        a, b_ = L.uL(k)[:nj], L.uR(k)[:nj]
        P0[a, a] += 2 * w / 3
        P0[b_, b_] += 2 * w / 3
        P0[a, b_] += w / 3
        P0[b_, a] += w / 3

    # affine scaling, then row normalization
    D, o = _scaling(L, prm)
    A1, b1 = A0 * D[None, :], b0 - A0 @ o
    G1, h1 = G0 * D[None, :], h0 - G0 @ o
    P1 = D[:, None] * P0 * D[None, :]
    c1 = D * (P0 @ o + c0)

    def rho_of(M):
        mx = np.abs(M[:, L.is_problem]).max(axis=1) if M.shape[0] else np.zeros(0)
        return np.where(mx > 0, 1.0 / np.where(mx > 0, mx, 1.0), 1.0)

    rA = rho_of(A1)
    rG = rho_of(G1)
    for q in range(n_soc):
        r0 = n_nonneg + 2 * q
        rG[r0:r0 + 2] = rG[r0:r0 + 2].min()
    return {"A": rA[:, None] * A1, "b": rA * b1, "G": rG[:, None] * G1, "h": rG * h1,
            "P": P1, "c": c1, "rho_A": rA, "rho_G": rG, "n_nonneg": n_nonneg, "n_soc": n_soc,
            "D": D, "o": o, "zbar": zbar, "layout": L, "A0": A0, "b0": b0, "G0": G0, "h0": h0}
