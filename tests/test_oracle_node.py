"""Pins of the oracle's node constraints (impact map G~ and relaxed impulse
conditions Theta^delta, Eqs. (17e)-(17f); impact model Eq. (6), Sec. II-B;
Fischer-Burmeister relaxation Eq. (16)).

Nothing here re-types the oracle's formulas.  The impact map is pinned by
solving the full KKT system of Eq. (6a) with the joint constraint
grad C v+ = 0, with numpy and with grad C and J_c from rotation matrices
(dR(theta)/dtheta = R(theta + pi/2)).  Physical invariants are checked at its
solution: linear and angular momentum change equal the contact impulse and
its moment, since joint impulses are internal.  The relaxed complementarity
rows are pinned by configurations whose complementarity pairs are satisfied
or violated by construction; contact-point velocities there come from finite
differences of the contact position.  The Jacobians are pinned by central
finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_2604_09993_gb300 import synth


def _rot(th):
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]])


def _robot_objects():
    rng = np.random.default_rng(17)
    return {"hopper": synth.hopper(rng), "biped": synth.biped(rng), "cheetah7": synth.cheetah7(rng)}


def _robots():
    return {k: r.as_dict() for k, r in _robot_objects().items()}


def _geometry(R, q):
    """grad C [2nj, nq] and contact Jacobians [nc][2, nq], from rotation matrices."""
    nb = len(R["mass"])
    nq = 3 * nb
    jp, jc = R["joint_parent"], R["joint_child"]
    G = np.zeros((2 * len(jp), nq))
    for j in range(len(jp)):
        for body, rho, sign in ((jc[j], R["joint_rho_child"][j], 1.0), (jp[j], R["joint_rho_parent"][j], -1.0)):
            G[2 * j:2 * j + 2, 3 * body:3 * body + 2] += sign * np.eye(2)
            G[2 * j:2 * j + 2, 3 * body + 2] += sign * (_rot(q[3 * body + 2] + np.pi / 2) @ rho)
    Jc = []
    for i, b in enumerate(R["contact_body"]):
        J = np.zeros((2, nq))
        J[:, 3 * b:3 * b + 2] = np.eye(2)
        J[:, 3 * b + 2] = _rot(q[3 * b + 2] + np.pi / 2) @ R["contact_rho"][i]
        Jc.append(J)
    return G, Jc


def _mass(R):
    return np.concatenate([[m, m, I] for m, I in zip(R["mass"], R["inertia"])])


def _kkt_post_velocity(R, q, vm, Phi):
    """v+ from [M -G^T; G 0][v+; Lambda] = [M v- + J_c^T Phi; 0]."""
    G, Jc = _geometry(R, q)
    Mv = _mass(R)
    nq, nr = len(Mv), G.shape[0]
    imp = sum((J.T @ Phi[2 * i:2 * i + 2] for i, J in enumerate(Jc)), np.zeros(nq))
    A = np.zeros((nq + nr, nq + nr))
    A[:nq, :nq] = np.diag(Mv)
    A[:nq, nq:] = -G.T
    A[nq:, :nq] = G
    rhs = np.concatenate([Mv * vm + imp, np.zeros(nr)])
    return np.linalg.solve(A, rhs)[:nq]


def _node_inputs(R, rng):
    nb, nc = len(R["mass"]), len(R["contact_body"])
    nq, nxt = 3 * nb, 6 * nb + nc
    xm = rng.uniform(-1, 1, nxt)
    Phi = rng.standard_normal(2 * nc)
    Gam = rng.uniform(0.0, 1.0, nc)
    return nq, nxt, xm, Phi, Gam


@pytest.mark.parametrize("name", ["hopper", "biped", "cheetah7"])
def test_impact_map_zero_at_kkt_solution(name):
    R = _robots()[name]
    rng = np.random.default_rng(3)
    nq, nxt, xm, Phi, Gam = _node_inputs(R, rng)
    vp = _kkt_post_velocity(R, xm[:nq], xm[nq:2 * nq], Phi)
    xp = xm.copy()
    xp[nq:2 * nq] = vp
    g, _ = oracle.node_value(R, xp, xm, Phi, Gam, 1e-4, np.full(len(Gam), 0.5))
    scale = np.max(np.abs(_mass(R) * vp)) + np.max(np.abs(Phi))
    assert np.max(np.abs(g)) <= 1e-12 * scale, np.max(np.abs(g))
    # joint velocity constraints hold after impact
    G, Jc = _geometry(R, xm[:nq])
    assert np.max(np.abs(G @ vp)) <= 1e-12 * np.max(np.abs(vp))
    # a different v+ leaves a residual of M times the difference in the v rows
    dv = rng.standard_normal(nq)
    xp2 = xp.copy()
    xp2[nq:2 * nq] += dv
    g2, _ = oracle.node_value(R, xp2, xm, Phi, Gam, 1e-4, np.full(len(Gam), 0.5))
    assert np.allclose(g2[nq:2 * nq], _mass(R) * dv, rtol=1e-12, atol=1e-12 * scale)


@pytest.mark.parametrize("name", ["hopper", "cheetah7"])
def test_impact_momentum_balance(name):
    """Joint impulses are internal: at the post-impact velocity the change of
    linear momentum equals the total contact impulse and, on a pose that meets
    the joint constraints (so each joint's two impulses act at one point), the
    change of angular momentum about the origin equals its moment."""
    robot = _robot_objects()[name]
    R = robot.as_dict()
    rng = np.random.default_rng(8)
    nq, nxt, xm, Phi, Gam = _node_inputs(R, rng)
    qb, _ = synth.fk(robot, (0.2, 0.7), 0.3, rng.uniform(-0.6, 0.6, robot.nj))
    xm[:nq] = qb.reshape(-1)
    q, vm = xm[:nq], xm[nq:2 * nq]
    vp = _kkt_post_velocity(R, q, vm, Phi)
    # the oracle's residual vanishes there (so its v+ is this one)
    xp = xm.copy()
    xp[nq:2 * nq] = vp
    g, _ = oracle.node_value(R, xp, xm, Phi, Gam, 1e-4, np.zeros(len(Gam)))
    assert np.max(np.abs(g)) <= 1e-11
    m, I = np.asarray(R["mass"]), np.asarray(R["inertia"])
    dv = (vp - vm).reshape(-1, 3)
    pos = q.reshape(-1, 3)[:, :2]
    lin = (m[:, None] * dv[:, :2]).sum(0)
    ang = (I * dv[:, 2]).sum() + (m * (pos[:, 0] * dv[:, 1] - pos[:, 1] * dv[:, 0])).sum()
    imp = Phi.reshape(-1, 2)  # (Phi_t, Phi_n) = world (x, y) on flat ground
    cp = np.array([q[3 * b:3 * b + 2] + _rot(q[3 * b + 2]) @ R["contact_rho"][i]
                   for i, b in enumerate(R["contact_body"])])
    assert np.allclose(lin, imp.sum(0), atol=1e-11)
    assert abs(ang - (cp[:, 0] * imp[:, 1] - cp[:, 1] * imp[:, 0]).sum()) <= 1e-11


def test_free_link_impulse_closed_form():
    """One link, no joints: v+ = v- + M^-1 J_c^T Phi (textbook rigid-body impulse)."""
    R = {"mass": np.array([2.0]), "inertia": np.array([0.3]),
         "joint_parent": np.zeros(0, dtype=np.int32), "joint_child": np.zeros(0, dtype=np.int32),
         "joint_rho_parent": np.zeros((0, 2)), "joint_rho_child": np.zeros((0, 2)),
         "contact_body": np.array([0], dtype=np.int32), "contact_rho": np.array([[0.1, -0.4]]),
         "contact_mu": np.array([0.8]), "gravity": 9.81}
    xm = np.array([0.3, 0.5, 0.7, -0.2, -1.1, 0.4, 0.0])
    Phi = np.array([0.25, 1.5])
    r = _rot(0.7) @ R["contact_rho"][0]
    torque = r[0] * Phi[1] - r[1] * Phi[0]
    xp = xm.copy()
    xp[3:6] += [Phi[0] / 2.0, Phi[1] / 2.0, torque / 0.3]
    g, _ = oracle.node_value(R, xp, xm, Phi, [0.0], 1e-4, [0.0])
    assert np.max(np.abs(g)) <= 1e-15


def test_impact_map_identity_without_impulse():
    """Phi = 0 and v- already satisfying the joint constraints: v+ = v- is the solution."""
    R = _robots()["biped"]
    rng = np.random.default_rng(2)
    nq, nxt, xm, Phi, Gam = _node_inputs(R, rng)
    G, _ = _geometry(R, xm[:nq])
    _, _, Vt = np.linalg.svd(G)
    null = Vt[G.shape[0]:]
    xm[nq:2 * nq] = null.T @ rng.standard_normal(null.shape[0])
    g, _ = oracle.node_value(R, xm, xm, np.zeros_like(Phi), Gam, 1e-4, np.zeros(len(Gam)))
    assert np.max(np.abs(g)) <= 1e-12


@pytest.mark.parametrize("name", ["hopper", "cheetah7"])
def test_node_jacobians_match_finite_differences(name):
    R = _robots()[name]
    rng = np.random.default_rng(6)
    nq, nxt, xm, Phi, Gam = _node_inputs(R, rng)
    xp = xm + 0.3 * rng.standard_normal(nxt)
    nc = len(Gam)
    e = rng.uniform(0, 1, nc)
    delta = 1e-2
    out = oracle.node(R, xp[None], xm[None], Phi[None], Gam[None], delta, e)
    z0 = np.concatenate([xp, xm, Phi, Gam])

    def f(z):
        g, th = oracle.node_value(R, z[:nxt], z[nxt:2 * nxt], z[2 * nxt:2 * nxt + 2 * nc],
                                  z[2 * nxt + 2 * nc:], delta, e)
        return np.concatenate([g, th])

    J = np.concatenate([out["Jg"][0], out["Jth"][0]])
    h = 1e-6
    Jfd = np.empty_like(J)
    for c in range(len(z0)):
        zp, zm = z0.copy(), z0.copy()
        zp[c] += h
        zm[c] -= h
        Jfd[:, c] = (f(zp) - f(zm)) / (2 * h)
    assert np.max(np.abs(J - Jfd)) <= 1e-6 * max(1.0, np.max(np.abs(J)))
    assert np.allclose(out["g"][0], f(z0)[:nxt], rtol=0, atol=1e-14)


def test_node_jacobian_structure():
    """The blocks the kernel leaves implicit: dq-rows = [I, -I], dy-rows = [I, -I],
    dv-rows/dv+ = M, dv-rows/dp- = 0 and d/dx~+ zero outside v+, dG~/dGamma = 0;
    dv-rows/dv- is symmetric (= -M P with P the M-orthogonal projection)."""
    R = _robots()["cheetah7"]
    rng = np.random.default_rng(9)
    nq, nxt, xm, Phi, Gam = _node_inputs(R, rng)
    xp = xm + rng.standard_normal(nxt)
    nc = len(Gam)
    out = oracle.node(R, xp[None], xm[None], Phi[None], Gam[None], 1e-3, np.full(nc, 0.2))
    J = out["Jg"][0]
    I = np.eye(nq)
    assert np.array_equal(J[:nq, :nq], I) and np.array_equal(J[:nq, nxt:nxt + nq], -I)
    assert not np.any(J[:nq, nq:nxt]) and not np.any(J[:nq, nxt + nq:])
    ny = slice(2 * nq, nxt)
    assert np.array_equal(J[ny, 2 * nq:nxt], np.eye(nc))
    assert np.array_equal(J[ny, nxt + 2 * nq:2 * nxt], -np.eye(nc))
    assert np.count_nonzero(J[ny]) == 2 * nc
    V = slice(nq, 2 * nq)
    assert np.allclose(J[V, nq:2 * nq], np.diag(_mass(R)), rtol=1e-15, atol=0)
    assert not np.any(J[V, :nq]) and not np.any(J[V, 2 * nq:nxt])
    assert not np.any(J[V, nxt + 0:nxt + nq:3]) and not np.any(J[V, nxt + 1:nxt + nq:3])
    assert not np.any(J[V, nxt + 2 * nq:2 * nxt]) and not np.any(J[:, 2 * nxt + 2 * nc:])
    # Theta depends on contact i's link only through (p_y-, theta-, v_x+, v_y+,
    # omega+, v_y-, omega-) and on (Phi_t, Phi_n, Gamma) of contact i
    Jt = out["Jth"][0]
    for i, b in enumerate(R["contact_body"]):
        cols = [nxt + 3 * b + 1, nxt + 3 * b + 2, nq + 3 * b, nq + 3 * b + 1, nq + 3 * b + 2,
                nxt + nq + 3 * b + 1, nxt + nq + 3 * b + 2, 2 * nxt + 2 * i, 2 * nxt + 2 * i + 1,
                2 * nxt + 2 * nc + i]
        mask = np.ones(Jt.shape[1], bool)
        mask[cols] = False
        assert not np.any(Jt[8 * i:8 * i + 8][:, mask])
    Gvm = J[V, nxt + nq:nxt + 2 * nq]
    assert np.allclose(Gvm, Gvm.T, atol=1e-13)
    assert np.max(np.linalg.eigvalsh(Gvm)) <= 1e-12  # -M P is negative semidefinite


def _contact_point(R, q, i):
    b = R["contact_body"][i]
    return q[3 * b:3 * b + 2] + _rot(q[3 * b + 2]) @ R["contact_rho"][i]


def _point_velocity(R, q, v, i, h=1e-6):
    """d/dt of the contact point along q' = v, by central differences."""
    return (_contact_point(R, q + h * v, i) - _contact_point(R, q - h * v, i)) / (2 * h)


def test_theta_rows_on_satisfied_and_violated_pairs():
    """Hopper, one contact.  Build a node where every complementarity pair of
    Eqs. (6b)-(6e) has one side exactly zero: foot on the ground, Newton's
    restitution law met, foot not sliding, friction strictly inside the cone
    with Gamma = 0.  With a tiny delta every FB row is then <= 0 and close to 0,
    and the sign rows match.  Breaking one pair at a time makes its FB row
    clearly positive."""
    R = dict(_robots()["hopper"], contact_mu=np.array([0.6]))
    nb = len(R["mass"])
    nq, nxt = 3 * nb, 6 * nb + 1
    rng = np.random.default_rng(1)
    q = rng.uniform(-0.5, 0.5, nq)
    q[3 * R["contact_body"][0] + 1] -= _contact_point(R, q, 0)[1]  # contact point at y = 0
    e = np.array([0.4])
    vm = rng.standard_normal(nq)
    vp = rng.standard_normal(nq)
    b = R["contact_body"][0]
    # adjust the foot link's linear velocity so that the contact point of v+
    # has zero tangential velocity and normal velocity -e times that of v-
    pm = _point_velocity(R, q, vm, 0)
    pp = _point_velocity(R, q, vp, 0)
    vp[3 * b] -= pp[0]
    vp[3 * b + 1] -= pp[1] + e[0] * pm[1]
    xm = np.concatenate([q, vm, [0.0]])
    xp = np.concatenate([q, vp, [0.0]])
    mu = R["contact_mu"][0]
    Phi = np.array([0.3 * mu * 2.0, 2.0])  # |Phi_t| < mu Phi_n
    delta = 1e-14
    _, th = oracle.node_value(R, xp, xm, Phi, [0.0], delta, e)
    assert np.all(th[:4] <= 1e-12) and np.all(th[:4] >= -1e-5), th[:4]
    assert th[4] == -2.0 and abs(th[5]) <= 1e-9 and th[6] == 0.0 and th[7] < 0.0
    # violate one pair at a time
    xm_up = xm.copy()
    xm_up[3 * b + 1] += 0.05  # foot 5 cm above ground while Phi_n > 0
    _, t1 = oracle.node_value(R, xp, xm_up, Phi, [0.0], delta, e)
    assert t1[0] > 0.04
    xp_b = xp.copy()
    xp_b[nq + 3 * b + 1] += 0.3  # bounces back faster than the restitution law
    _, t2 = oracle.node_value(R, xp_b, xm, Phi, [0.0], delta, e)
    assert t2[1] > 0.03 and abs(t2[0] - th[0]) < 1e-12
    xp_s = xp.copy()
    xp_s[nq + 3 * b] += 0.3  # foot slides
    _, t3 = oracle.node_value(R, xp_s, xm, Phi, [0.0], delta, e)
    assert t3[2] > 0.03
    _, t4 = oracle.node_value(R, xp, xm, Phi, [0.7], delta, e)  # Gamma > 0 inside the cone
    assert t4[3] > 0.05 and t4[2] > 0.0  # stationarity now broken too
    # on the cone boundary |Phi_t| = mu Phi_n: rho = 0, so FB(Gamma, rho) ~ 0 for Gamma > 0
    _, t5 = oracle.node_value(R, xp, xm, np.array([mu * 2.0, 2.0]), [0.7], delta, e)
    assert abs(t5[7]) <= 1e-14 and -1e-5 <= t5[3] <= 1e-12


def test_fischer_burmeister_limits():
    """FB^delta(a, b) -> min-type behaviour: for a, b >= 0 it is <= 0 iff
    a b <= delta / 2, and equals -sqrt(delta) at a = b = 0 (row 0 with Phi_n = 0
    and the foot on the ground)."""
    R = _robots()["hopper"]
    nb = len(R["mass"])
    nq = 3 * nb
    q = np.zeros(nq)
    q[3 * R["contact_body"][0] + 1] -= _contact_point(R, q, 0)[1]
    xm = np.concatenate([q, np.zeros(nq), [0.0]])
    for delta in (1e-2, 1e-6):
        _, th = oracle.node_value(R, xm, xm, np.zeros(2), [0.0], delta, [0.0])
        assert abs(th[0] + np.sqrt(delta)) <= 1e-15
        xa = xm.copy()
        xa[3 * R["contact_body"][0] + 1] += 0.5
        for pn in (0.5 * delta / 0.5 * 0.99, 0.5 * delta / 0.5 * 1.01):  # a b just below / above delta/2
            _, th = oracle.node_value(R, xm, xa, np.array([0.0, pn]), [0.0], delta, [0.0])
            assert (th[0] <= 0) == (pn * 0.5 <= delta / 2)


def test_theta_rows_sliding_contact():
    """A sliding foot: tangential impulse on the cone boundary opposing the
    slip, Gamma chosen so that the stationarity condition Eq. (6d) holds.
    Then FB(Phi_n, |lambda^c|~) and FB(Gamma, rho) are both ~0; Gamma off by
    10 % breaks the stationarity row only."""
    R = dict(_robots()["hopper"], contact_mu=np.array([0.6]))
    nb = len(R["mass"])
    nq = 3 * nb
    b = R["contact_body"][0]
    rng = np.random.default_rng(4)
    q = rng.uniform(-0.5, 0.5, nq)
    q[3 * b + 1] -= _contact_point(R, q, 0)[1]
    e = np.array([0.0])
    vm = rng.standard_normal(nq)
    vp = rng.standard_normal(nq)
    pp = _point_velocity(R, q, vp, 0)
    vp[3 * b + 1] -= pp[1]  # normal velocity 0 after impact (e = 0)
    vt = _point_velocity(R, q, vp, 0)[0]
    assert abs(vt) > 0.1
    pn = 1.7
    pt = -np.sign(vt) * 0.6 * pn
    gam = abs(vt) * np.sqrt(1.0 + pt * pt) / abs(pt)
    xm = np.concatenate([q, vm, [0.0]])
    xp = np.concatenate([q, vp, [0.0]])
    delta = 1e-14
    _, th = oracle.node_value(R, xp, xm, np.array([pt, pn]), [gam], delta, e)
    assert np.all(th[:4] <= 1e-12) and np.all(th[:4] >= -1e-5), th[:4]
    assert abs(th[7]) <= 1e-14  # on the cone
    _, t2 = oracle.node_value(R, xp, xm, np.array([pt, pn]), [1.1 * gam], delta, e)
    assert t2[2] > 1e-3 and t2[3] <= 1e-12
