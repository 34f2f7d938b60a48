"""Pin of the oracle's Phi-contracted VJP against central differences (no GPU).

L = sum_k w_k . defect_k + sum_k rho_k . penalty_k, defect_k = F~(x~_k, U_k,
s_k) - x~_{k+1} (Eq. (17b)), penalty_k = y(1) - y_k.  The finite differences
use only the oracle's plain FP64 flow map.
"""
import numpy as np
import pytest

from paper_2604_09993_gb300 import synth


def _loss(oracle_mod, R, nx, X, U, s, w, rho, n_sub, layout):
    N = len(s)
    L = 0.0
    for k in range(N):
        uL, uR = (U[k], U[k + 1]) if layout == "node" else (U[k, 0], U[k, 1])
        x1 = oracle_mod.flow(R, n_sub, X[k], uL, uR, s[k])
        L += w[k] @ (x1 - X[k + 1]) + rho[k] @ (x1[nx:] - X[k, nx:])
    return L


@pytest.mark.parametrize("layout", ["node", "interval"])
def test_vjp_matches_central_differences(oracle_mod, layout):
    p = synth.hopper_fp64(seed=1, N=3, n_sub=2)
    R = p.robot.as_dict()
    nx = p.robot.nx
    U = p.U if layout == "node" else p.U_interval()
    gX, gU, gs, L = oracle_mod.vjp(R, p.X, U, p.s, p.w, p.rho, p.n_sub, layout=layout)
    f = lambda X, U, s: _loss(oracle_mod, R, nx, X, U, s, p.w, p.rho, p.n_sub, layout)  # noqa: E731
    assert abs(L - f(p.X, U, p.s)) < 1e-12 * max(1.0, abs(L))
    e = 1e-6
    for arr, g in ((p.X, gX), (U, gU), (p.s, gs)):
        flat = arr.reshape(-1)
        gf = g.reshape(-1)
        for i in range(flat.size):
            save = flat[i]
            flat[i] = save + e
            lp = f(p.X, U, p.s)
            flat[i] = save - e
            lm = f(p.X, U, p.s)
            flat[i] = save
            fd = (lp - lm) / (2 * e)
            assert abs(fd - gf[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, gf[i])
