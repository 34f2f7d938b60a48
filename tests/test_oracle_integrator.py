"""Pins of the oracle's integrator and IND (no GPU).

The oracle's RK4 + first-order hold + time dilation + dual-number IND
(Sec. IV-B Eqs. (14)-(15), Sec. VI) is run on a LINEAR right-hand side
F = A_c x + B_c u, where the exact discrete map has a closed form:

* With w(tau) = u(tau) and d = u_R - u_L, the FOH system is the autonomous
  linear system z' = M z, z = (x, w, d), M = [[s A_c, s B_c, 0], [0, 0, I],
  [0, 0, 0]].  RK4 on z' = M z is z <- T4(h M) z exactly, T4 the degree-4
  Taylor polynomial, so the whole interval is E = T4(h M)^n.
* d/ds of that product is the top-right block of T4(h [[M, M_1], [0, M]])^n
  with M_1 = dM/ds (the derivative of a matrix polynomial along a direction is
  the off-diagonal block of the polynomial of the block-triangular matrix).
* As n grows, RK4 converges to the exact flow expm(M) with error O(h^4).
"""
import numpy as np
import pytest
import scipy.linalg as sla


def _t4(X):
    I = np.eye(X.shape[0])
    X2 = X @ X
    return I + X + X2 / 2.0 + X2 @ X / 6.0 + X2 @ X2 / 24.0


def _aug(Ac, Bc, s):
    n, m = Bc.shape
    K = n + 2 * m
    M = np.zeros((K, K))
    M[:n, :n] = s * Ac
    M[:n, n:n + m] = s * Bc
    M[n:n + m, n + m:] = np.eye(m)
    M1 = np.zeros((K, K))
    M1[:n, :n] = Ac
    M1[:n, n:n + m] = Bc
    return M, M1


def _closed_form(Ac, Bc, s, n_sub, x0, uL, uR):
    n, m = Bc.shape
    M, M1 = _aug(Ac, Bc, s)
    K = M.shape[0]
    h = 1.0 / n_sub
    big = np.zeros((2 * K, 2 * K))
    big[:K, :K] = h * M
    big[K:, K:] = h * M
    big[:K, K:] = h * M1
    P = np.linalg.matrix_power(_t4(big), n_sub)
    E, dE = P[:K, :K], P[:K, K:]
    z0 = np.concatenate([x0, uL, uR - uL])
    x1 = (E @ z0)[:n]
    A = E[:n, :n]
    Bm = E[:n, n:n + m] - E[:n, n + m:]
    Bp = E[:n, n + m:]
    S = (dE @ z0)[:n]
    return x1, A, Bm, Bp, S


@pytest.mark.parametrize("n_sub", [1, 3, 8])
@pytest.mark.parametrize("s", [0.0, 0.37, 1.3])
def test_linear_system_matches_rk4_polynomial(oracle_mod, n_sub, s):
    rng = np.random.default_rng(11)
    n, m = 5, 3
    Ac = rng.standard_normal((n, n))
    Bc = rng.standard_normal((n, m))
    x0, uL, uR = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
    got = oracle_mod.linear_interval(Ac, Bc, n_sub, x0, uL, uR, s)
    ref = _closed_form(Ac, Bc, s, n_sub, x0, uL, uR)
    for g, r, name in zip(got, ref, ["x1", "A", "Bm", "Bp", "S"]):
        scale = max(1.0, np.abs(r).max())
        assert np.abs(g - r).max() <= 1e-12 * scale, name


def test_linear_system_fourth_order_convergence(oracle_mod):
    """Errors of x, A, B-, B+ and S against the exact FOH flow (Van Loan block exponential) fall ~16x per halving of h."""
    rng = np.random.default_rng(5)
    n, m = 4, 2
    Ac = rng.standard_normal((n, n)) * 0.8
    Bc = rng.standard_normal((n, m))
    x0, uL, uR = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
    s = 0.9
    M, M1 = _aug(Ac, Bc, s)
    E = sla.expm(M)
    A_ex = E[:n, :n]
    Bp_ex = E[:n, n + m:]
    Bm_ex = E[:n, n:n + m] - Bp_ex
    z0 = np.concatenate([x0, uL, uR - uL])
    x_ex = E[:n, :] @ z0
    # d/ds expm(M(s)) is the top-right block of expm([[M, M1], [0, M]]), M1 = dM/ds
    K = M.shape[0]
    big = np.zeros((2 * K, 2 * K))
    big[:K, :K] = M
    big[K:, K:] = M
    big[:K, K:] = M1
    S_ex = (sla.expm(big)[:K, K:] @ z0)[:n]
    assert np.allclose(A_ex, sla.expm(s * Ac), rtol=1e-13, atol=1e-13)
    errs = []
    for n_sub in (2, 4, 8, 16):
        x1, A, Bm, Bp, S = oracle_mod.linear_interval(Ac, Bc, n_sub, x0, uL, uR, s)
        errs.append(max(np.abs(A - A_ex).max(), np.abs(Bm - Bm_ex).max(),
                        np.abs(Bp - Bp_ex).max(), np.abs(x1 - x_ex).max(), np.abs(S - S_ex).max()))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    for r in ratios:
        assert 12.0 < r < 20.0, (errs, ratios)


def test_s_derivative_matches_central_difference_linear(oracle_mod):
    rng = np.random.default_rng(9)
    n, m = 3, 2
    Ac, Bc = rng.standard_normal((n, n)), rng.standard_normal((n, m))
    x0, uL, uR = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
    s, e = 0.6, 1e-6
    S = oracle_mod.linear_interval(Ac, Bc, 4, x0, uL, uR, s)[4]
    xp = oracle_mod.linear_interval(Ac, Bc, 4, x0, uL, uR, s + e)[0]
    xm = oracle_mod.linear_interval(Ac, Bc, 4, x0, uL, uR, s - e)[0]
    assert np.abs(S - (xp - xm) / (2 * e)).max() < 1e-8
