"""Pins of the oracle's Psi^{delta,eps}(y-_{k+1}, y+_k) <= 0 (Eq. (17c)): the
Fischer-Burmeister-relaxed (Eq. (16)) integral cross-complementarity of the
auxiliary-state increments (Eq. (11) on the pairs of Eq. (12)) and the relaxed
path-constraint rows of Eq. (13).

Nothing here re-types the oracle's rows:
* for a, b >= 0, FB^delta(a, b) <= 0 holds exactly when 2 a b <= delta
  (square a + b <= sqrt(a^2 + b^2 + delta));
* as delta -> 0, FB(3, 4) -> 3 + 4 - 5 = 2 and FB(a, 0) -> 0; FB(0, 0) = -sqrt(delta);
* with zero contact inputs on flat ground, the phi_n, gamma and rho^c
  integrands vanish and lambda^c is the tangential velocity of the contact
  point: the (phi_n, lambda^c) row is FB(0, dx_c), dx_c the contact point's x
  displacement over the interval measured from the poses by rotation
  matrices, and the (gamma, rho^c) row is FB(0, 0) = -sqrt(delta);
* on a consistent trajectory (y-_{k+1} = the flow of x~_k) the path-constraint
  rows plus eps equal the penalty increments of the discretization;
* the Jacobian in y+_k is minus that in y-_{k+1} (Psi depends on the
  increment only) and matches central differences.
"""
import numpy as np
import pytest

import oracle
from paper_2604_09993_gb300 import synth


def _robot(name="cheetah7", cross=True, seed=5):
    rng = np.random.default_rng(seed)
    R = getattr(synth, name)(rng)
    return synth.with_cross_states(R) if cross else R


def _nodes_with_increments(R, D, rng):
    """Node states whose y increments over each interval are the rows of D."""
    N = D.shape[0]
    nx = 6 * R.nb
    Xp = rng.uniform(-1, 1, (N + 1, R.nxt))
    Xm = rng.uniform(-1, 1, (N + 1, R.nxt))
    Xm[1:, nx:] = Xp[:-1, nx:] + D
    return Xp, Xm


def _rot(th):
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]])


def test_row_count():
    R = _robot()
    rng = np.random.default_rng(0)
    Xp, Xm = _nodes_with_increments(R, np.zeros((3, R.nxt - 6 * R.nb)), rng)
    out = oracle.psi(R.as_dict(), Xp, Xm, 0.1, 1e-4)
    assert out["psi"].shape == (3, 3 * R.nc)
    R0 = _robot(cross=False)
    Xp, Xm = _nodes_with_increments(R0, np.zeros((3, R0.nc)), rng)
    assert oracle.psi(R0.as_dict(), Xp, Xm, 0.1, 1e-4)["psi"].shape == (3, R0.nc)


def test_fb_sign_is_the_product_bound():
    """FB^delta(a, b) <= 0 with a, b >= 0  <=>  2ab <= delta."""
    R = _robot()
    rng = np.random.default_rng(1)
    N, nc, ny = 400, R.nc, R.nxt - 6 * R.nb
    delta = 0.3
    D = np.zeros((N, ny))
    D[:, : 4 * nc] = rng.exponential(0.5, (N, 4 * nc))
    Xp, Xm = _nodes_with_increments(R, D, rng)
    psi = oracle.psi(R.as_dict(), Xp, Xm, delta, 0.0)["psi"]
    checked = 0
    for i in range(nc):
        for row, (a, b) in ((2 * i, (D[:, 4 * i], D[:, 4 * i + 1])),
                            (2 * i + 1, (D[:, 4 * i + 2], D[:, 4 * i + 3]))):
            margin = np.abs(2 * a * b - delta) > 1e-6
            assert np.array_equal(psi[margin, row] <= 0, (2 * a * b <= delta)[margin])
            checked += margin.sum()
    assert checked > 0.9 * 2 * nc * N


def test_fb_textbook_values():
    R = _robot()
    rng = np.random.default_rng(2)
    ny = R.nxt - 6 * R.nb
    D = np.zeros((3, ny))
    D[0, 0:2] = (3.0, 4.0)          # contact 0, pair (phi_n, lambda^c)
    D[1, 0:2] = (2.5, 0.0)
    D[2, 2:4] = (0.0, 0.0)
    Xp, Xm = _nodes_with_increments(R, D, rng)
    tiny = 1e-24
    psi = oracle.psi(R.as_dict(), Xp, Xm, tiny, 0.0)["psi"]
    assert psi[0, 0] == pytest.approx(2.0, abs=1e-12)
    assert psi[1, 0] == pytest.approx(0.0, abs=1e-12)
    delta = 0.49
    psi = oracle.psi(R.as_dict(), Xp, Xm, delta, 0.0)["psi"]
    assert psi[2, 1] == pytest.approx(-0.7, abs=1e-15)


@pytest.mark.parametrize("name", ["hopper", "cheetah7"])
def test_pairing_from_contact_kinematics(name):
    """Zero contact inputs: row (phi_n, lambda^c) = FB(0, dx_c), row (gamma, rho^c) = -sqrt(delta)."""
    R = _robot(name)
    rng = np.random.default_rng(4)
    nb, nj, nc, nu = R.nb, R.nj, R.nc, R.nu
    N, nsub, delta = 3, 64, 0.04
    X = np.zeros((N + 1, R.nxt))
    X[:, : 6 * nb] = rng.uniform(-0.3, 0.3, (N + 1, 6 * nb))
    U = np.zeros((N + 1, nu))
    U[:, : 3 * nj] = rng.standard_normal((N + 1, 3 * nj))   # joint torques and forces only
    s = rng.uniform(0.05, 0.15, N)
    d = oracle.discretize(R.as_dict(), X, U, s, nsub)
    Xm = X.copy()
    Xm[1:] = X[1:] + d["defect"]          # y-_{k+1} = the flow of x~_k
    psi = oracle.psi(R.as_dict(), X, Xm, delta, 0.0)["psi"]
    for k in range(N):
        x0, x1 = X[k], Xm[k + 1]
        for i in range(nc):
            b = R.contact_body[i]
            xc0 = x0[3 * b] + (_rot(x0[3 * b + 2]) @ R.contact_rho[i])[0]
            xc1 = x1[3 * b] + (_rot(x1[3 * b + 2]) @ R.contact_rho[i])[0]
            dx = xc1 - xc0
            assert abs(dx) > 1e-4
            assert psi[k, 2 * i] == pytest.approx(dx - np.sqrt(dx * dx + delta), abs=1e-7)
            assert psi[k, 2 * i + 1] == pytest.approx(-np.sqrt(delta), abs=1e-14)


@pytest.mark.parametrize("cross", [False, True])
def test_path_rows_are_penalty_increments(cross):
    R = _robot("cheetah7", cross=cross)
    rng = np.random.default_rng(6)
    N, nsub, eps = 4, 4, 1e-4
    X = np.zeros((N + 1, R.nxt))
    X[:, : 6 * R.nb] = rng.uniform(-0.3, 0.3, (N + 1, 6 * R.nb))
    X[:, 6 * R.nb:] = rng.uniform(-1, 1, (N + 1, R.nxt - 6 * R.nb))
    U = rng.standard_normal((N + 1, R.nu))
    s = rng.uniform(0.05, 0.15, N)
    d = oracle.discretize(R.as_dict(), X, U, s, nsub)
    assert np.abs(d["penalty"]).max() > 1e-3
    Xm = X.copy()
    Xm[1:] = X[1:] + d["defect"]
    psi = oracle.psi(R.as_dict(), X, Xm, 0.1, eps)["psi"]
    rows = psi[:, 2 * R.nc:] if cross else psi
    np.testing.assert_allclose(rows + eps, d["penalty"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("cross", [False, True])
def test_jacobian(cross):
    R = _robot("hopper", cross=cross)
    rng = np.random.default_rng(7)
    ny = R.nxt - 6 * R.nb
    N, delta, eps = 5, 0.2, 1e-3
    Xp, Xm = _nodes_with_increments(R, rng.uniform(-1, 1, (N, ny)), rng)
    out = oracle.psi(R.as_dict(), Xp, Xm, delta, eps)
    J = out["J"]
    np.testing.assert_array_equal(J[:, :, :ny], -J[:, :, ny:])
    h = 1e-6
    for k in range(N):
        for j in range(ny):
            Xa, Xb = Xm.copy(), Xm.copy()
            Xa[k + 1, 6 * R.nb + j] += h
            Xb[k + 1, 6 * R.nb + j] -= h
            fd = (oracle.psi(R.as_dict(), Xp, Xa, delta, eps)["psi"][k]
                  - oracle.psi(R.as_dict(), Xp, Xb, delta, eps)["psi"][k]) / (2 * h)
            np.testing.assert_allclose(J[k, :, ny + j], fd, atol=1e-8)
