"""Seeded synthetic robots and problem instances for the CI-SCvx discretization.

This module is the ONE piece shared by the CUDA path's callers and the oracle's
callers: it draws robots (link masses and lengths), node states, FOH controls,
dilation factors and VJP cotangents with ``numpy.random.default_rng``.  It holds
none of the method's arithmetic — no dynamics, no integration, no derivatives;
the only geometry here is the forward kinematics that places links on a pose.

Robots are planar chains in maximal coordinates (the paper's model, Sec. II):
each link is a uniform rod with inertia m L^2 / 12; limb rods lie along their
local y axis with proximal anchor (0, +L/2) and distal anchor (0, -L/2); a
contact point sits at the distal end of each foot link.  The hopper torso is a
vertical rod with the hip at (0, -L/2); the biped and the 7-link chain have a
horizontal torso along local x with the hind hip at (-L/2, 0) and the front hip
at (+L/2, 0).  Rotation convention: a body-frame point rho sits at
p + R(theta) rho in the world, R = [[cos, -sin], [sin, cos]].

Draw order for one instance: links (m, L) -> node-state noise -> controls ->
dilation s -> cotangents w.  Batched configurations draw the shared robots from
the root generator and give instance i the child generator ``rng.spawn``'s i-th
stream, so any subset of instances can be regenerated alone.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

GRAVITY = 9.81
MU = 1.0  # friction coefficient used for every contact (Sec. VI settings)


@dataclass
class Robot:
    name: str
    mass: np.ndarray            # [nb]
    length: np.ndarray          # [nb]
    inertia: np.ndarray         # [nb]
    joint_parent: np.ndarray    # [nj] int
    joint_child: np.ndarray     # [nj] int
    joint_rho_parent: np.ndarray  # [nj, 2]
    joint_rho_child: np.ndarray   # [nj, 2]
    contact_body: np.ndarray    # [nc] int
    contact_rho: np.ndarray     # [nc, 2]
    contact_mu: np.ndarray      # [nc]
    gravity: float = GRAVITY
    legs: list = field(default_factory=list)  # per leg: list of joint indices (for gait poses)
    torso_horizontal: bool = True
    aux_model: int = 0  # 0: one path-penalty state per contact; 1: Eq. (12) (4 + 1 states per contact)
    joint_forces: int = 0  # 0: joint reaction forces are inputs; 1: eliminated by Eq. (3)
    scheme: int = 0        # integrator: 0 classical RK4, 1 Runge-Kutta-Fehlberg 4(5)
    terrain: tuple = (0.0, 0.0)  # contact surface y = a sin(k x) as (a, k); (0, 0) is flat ground

    @property
    def nb(self):
        return len(self.mass)

    @property
    def nj(self):
        return len(self.joint_parent)

    @property
    def nc(self):
        return len(self.contact_body)

    @property
    def nx(self):
        return 6 * self.nb

    @property
    def ny(self):
        return (5 if self.aux_model else 1) * self.nc

    @property
    def nxt(self):
        return 6 * self.nb + self.ny

    @property
    def nu(self):
        return (1 if self.joint_forces else 3) * self.nj + 3 * self.nc

    def as_dict(self):
        return {
            "mass": self.mass, "inertia": self.inertia,
            "joint_parent": self.joint_parent, "joint_child": self.joint_child,
            "joint_rho_parent": self.joint_rho_parent, "joint_rho_child": self.joint_rho_child,
            "contact_body": self.contact_body, "contact_rho": self.contact_rho,
            "contact_mu": self.contact_mu, "gravity": self.gravity, "aux_model": self.aux_model,
            "joint_forces": self.joint_forces, "scheme": self.scheme,
            "terrain": tuple(float(v) for v in self.terrain),
        }


def _chain_robot(name, m, L, torso_horizontal, leg_lengths):
    """Torso (body 0) plus legs; leg_lengths = number of links per leg."""
    m = np.asarray(m, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    I = m * L * L / 12.0
    parents, children, rp, rc, legs, cbody, crho = [], [], [], [], [], [], []
    b = 1
    nlegs = len(leg_lengths)
    for leg, nlink in enumerate(leg_lengths):
        if torso_horizontal:
            hip = (-0.5 * L[0], 0.0) if (nlegs == 2 and leg == 0) else (0.5 * L[0], 0.0)
        else:
            hip = (0.0, -0.5 * L[0])
        prev, prev_anchor = 0, hip
        js = []
        for _ in range(nlink):
            parents.append(prev)
            children.append(b)
            rp.append(prev_anchor)
            rc.append((0.0, 0.5 * L[b]))
            js.append(len(parents) - 1)
            prev, prev_anchor = b, (0.0, -0.5 * L[b])
            b += 1
        legs.append(js)
        cbody.append(prev)
        crho.append(prev_anchor)
    nc = len(cbody)
    return Robot(
        name=name, mass=m, length=L, inertia=I,
        joint_parent=np.asarray(parents, dtype=np.int32),
        joint_child=np.asarray(children, dtype=np.int32),
        joint_rho_parent=np.asarray(rp, dtype=np.float64).reshape(-1, 2),
        joint_rho_child=np.asarray(rc, dtype=np.float64).reshape(-1, 2),
        contact_body=np.asarray(cbody, dtype=np.int32),
        contact_rho=np.asarray(crho, dtype=np.float64).reshape(-1, 2),
        contact_mu=np.full(nc, MU), legs=legs, torso_horizontal=torso_horizontal,
    )


def hopper(rng):
    """Planar 3-link hopper: torso, thigh, shin; one foot contact (n_x~ = 19, n_u = 9)."""
    m = rng.uniform(1.0, 5.0, 3)
    L = rng.uniform(0.2, 0.5, 3)
    return _chain_robot("hopper", m, L, torso_horizontal=False, leg_lengths=[2])


def biped(rng):
    """Planar 5-link biped: torso plus 2 legs x (thigh, shin) (n_x~ = 32, n_u = 18)."""
    m = rng.uniform(1.0, 5.0, 5)
    L = rng.uniform(0.2, 0.5, 5)
    return _chain_robot("biped", m, L, torso_horizontal=True, leg_lengths=[2, 2])


def cheetah7(rng):
    """HalfCheetah-shaped 7-link chain: torso plus 2 legs x 3 links (n_x~ = 44, n_u = 24)."""
    m = rng.uniform(0.5, 6.0, 7)
    L = rng.uniform(0.1, 0.6, 7)
    return _chain_robot("cheetah7", m, L, torso_horizontal=True, leg_lengths=[3, 3])


def monoped(rng):
    """Planar 2-link monoped: a body and one leg link carrying the foot contact
    (n_x~ = 13, n_u = 9 with joint reaction forces as inputs)."""
    m = rng.uniform(1.0, 5.0, 2)
    L = rng.uniform(0.2, 0.5, 2)
    return _chain_robot("monoped", m, L, torso_horizontal=False, leg_lengths=[1])


def chain32(rng):
    """The largest model the library takes: a torso plus legs of 15 and 16 links
    (32 links, n_x~ = 194, n_u = 99; every link has six inputs)."""
    m = rng.uniform(0.5, 6.0, 32)
    L = rng.uniform(0.1, 0.6, 32)
    return _chain_robot("chain32", m, L, torso_horizontal=True, leg_lengths=[15, 16])


ROBOTS = {"hopper": hopper, "biped": biped, "cheetah7": cheetah7}


def with_cross_states(robot: Robot) -> Robot:
    """The same robot with the full Eq. (12) auxiliary state: four
    cross-complementarity states + one path-penalty state per contact, and
    contact inputs (phi_t, phi_n, gamma) in place of (lambda_n, lambda_t+, lambda_t-)."""
    return replace(robot, aux_model=1)


def with_paper_dynamics(robot: Robot, joint_forces=1, scheme=1, terrain=None) -> Robot:
    """The same robot with the paper's own modelling choices: joint reaction
    forces eliminated at the acceleration level (inputs: joint torques and
    contact inputs), the Runge-Kutta-Fehlberg 4(5) integrator and, if given,
    the sinusoidal contact surface y = a sin(k x) as (a, k)."""
    t = robot.terrain if terrain is None else (float(terrain[0]), float(terrain[1]))
    return replace(robot, joint_forces=int(joint_forces), scheme=int(scheme), terrain=t)


# Sinusoidal surface of the biped scenario (Sec. VI-B), synthetic dimensions:
# 5 cm amplitude, 1 m wavelength.
TERRAIN_SINE = (0.05, 2.0 * np.pi)


# ---------------------------------------------------------------------------
# Poses (forward kinematics only)
# ---------------------------------------------------------------------------
def _rot(th):
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]])


def fk(robot: Robot, torso_xy, torso_theta, rel_angles, torso_v=(0.0, 0.0), torso_omega=0.0,
       rel_rates=None):
    """Place every link so that joint anchors coincide (and, with rates, so do
    anchor velocities).  Returns q [nb, 3] and v [nb, 3]."""
    nb = robot.nb
    q = np.zeros((nb, 3))
    v = np.zeros((nb, 3))
    q[0] = (torso_xy[0], torso_xy[1], torso_theta)
    v[0] = (torso_v[0], torso_v[1], torso_omega)
    rel_rates = np.zeros(robot.nj) if rel_rates is None else np.asarray(rel_rates)
    for j in range(robot.nj):  # parents come before children
        p, c = robot.joint_parent[j], robot.joint_child[j]
        q[c, 2] = q[p, 2] + rel_angles[j]
        v[c, 2] = v[p, 2] + rel_rates[j]
        arm_p = _rot(q[p, 2]) @ robot.joint_rho_parent[j]
        arm_c = _rot(q[c, 2]) @ robot.joint_rho_child[j]
        q[c, :2] = q[p, :2] + arm_p - arm_c
        # point velocity p' + omega x r with omega x r = (-omega r_y, omega r_x)
        va = v[p, :2] + v[p, 2] * np.array([-arm_p[1], arm_p[0]])
        v[c, :2] = va - v[c, 2] * np.array([-arm_c[1], arm_c[0]])
    return q, v


def _lowest_contact_y(robot, q):
    ys = [q[b, 1] + (_rot(q[b, 2]) @ robot.contact_rho[i])[1] for i, b in enumerate(robot.contact_body)]
    return min(ys) if ys else 0.0


def gait_pose(robot: Robot, phase, torso_x):
    """Nominal pose: level torso, relative joint angles 0.3 sin(phase + phi_leg)
    with phi = 0 for the hind leg and pi for the front leg, lowest foot on y = 0.
    The hopper (one leg) stands straight up (all relative angles 0)."""
    rel = np.zeros(robot.nj)
    if robot.torso_horizontal:
        for leg, js in enumerate(robot.legs):
            phi = 0.0 if leg == 0 else np.pi
            rel[js] = 0.3 * np.sin(phase + phi)
    q, _ = fk(robot, (torso_x, 0.0), 0.0, rel)
    q[:, 1] -= _lowest_contact_y(robot, q)
    return q


_POSE_CACHE: dict = {}


def _gait_poses(robot: Robot, N):
    """gait_pose at phases 2 pi k / N, k = 0..N, with the torso at x = 0 (cached)."""
    key = (robot.name, robot.mass.tobytes(), robot.length.tobytes(), N)
    if key not in _POSE_CACHE:
        _POSE_CACHE[key] = np.stack([gait_pose(robot, 2.0 * np.pi * k / max(N, 1), 0.0)
                                     for k in range(N + 1)])
    return _POSE_CACHE[key]


def node_states(robot: Robot, N, s, noise_q, noise_v, speed=1.0):
    """Nominal node poses (gait, zero velocity, y = 0) plus the given noise.
    The torso advances along x at `speed` times the dilated time t_k = sum s;
    moving the torso translates every link rigidly, so the cached poses are
    shifted in x."""
    nb = robot.nb
    q = _gait_poses(robot, N).copy()  # [N+1, nb, 3]
    if robot.torso_horizontal:
        t = np.concatenate([[0.0], np.cumsum(s)])
        q[:, :, 0] += speed * t[:, None]
    X = np.zeros((N + 1, robot.nxt))
    X[:, : 3 * nb] = q.reshape(N + 1, -1) + noise_q
    X[:, 3 * nb: 6 * nb] = noise_v
    return X


# ---------------------------------------------------------------------------
# Problem instances
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    robot: Robot
    N: int
    n_sub: int
    X: np.ndarray       # [N+1, nxt]
    U: np.ndarray       # [N+1, nu] (node layout)
    s: np.ndarray       # [N]
    w: np.ndarray | None = None    # [N, nxt]
    rho: np.ndarray | None = None  # [N, nc]
    layout: str = "node"

    def U_interval(self):
        """The same controls in interval layout [N, 2, nu]."""
        return np.stack([self.U[:-1], self.U[1:]], axis=1).copy()


def draw_instance(robot: Robot, rng, N, n_sub, q_noise, u_dist, s_range, with_cotangents=False,
                  rho=10.0):
    nb = robot.nb
    nq = rng.uniform(-q_noise, q_noise, (N + 1, 3 * nb))
    nv = rng.uniform(-q_noise, q_noise, (N + 1, 3 * nb))
    if u_dist == "uniform":
        U = rng.uniform(-1.0, 1.0, (N + 1, robot.nu))
    else:
        U = rng.standard_normal((N + 1, robot.nu))
    s = rng.uniform(s_range[0], s_range[1], N)
    X = node_states(robot, N, s, nq, nv)
    w = rng.standard_normal((N, robot.nxt)) if with_cotangents else None
    r = np.full((N, robot.nc), float(rho)) if with_cotangents else None
    return Problem(robot, N, n_sub, X, U, s, w, r)


# Per-robot conventions: hopper poses get +-0.05 noise and U[-1,1] controls;
# biped and 7-link chain get +-0.1 noise about the gait and N(0,1) controls.
_ROBOT_STYLE = {
    "hopper": dict(q_noise=0.05, u_dist="uniform"),
    "biped": dict(q_noise=0.1, u_dist="normal"),
    "cheetah7": dict(q_noise=0.1, u_dist="normal"),
}


def hopper_fp64(seed=0, N=10, n_sub=4):
    """Hopper, N = 10 intervals, 4 RK4 substeps, s ~ U[0.05, 0.15] (plain FP64 case)."""
    rng = np.random.default_rng(seed)
    robot = hopper(rng)
    return draw_instance(robot, rng, N, n_sub, s_range=(0.05, 0.15), with_cotangents=True,
                         **_ROBOT_STYLE["hopper"])


def cheetah_n50(seed=0, N=50, n_sub=10):
    """7-link chain, N = 50, 10 substeps, gait +- 0.1, u ~ N(0,1), s ~ U[0.05, 0.15]."""
    rng = np.random.default_rng(seed)
    robot = cheetah7(rng)
    return draw_instance(robot, rng, N, n_sub, s_range=(0.05, 0.15), with_cotangents=True,
                         **_ROBOT_STYLE["cheetah7"])


def cheetah_adjoint(seed=0, N=100, n_sub=10):
    """7-link chain, N = 100, 10 substeps, w ~ N(0,1), rho = 10 (adjoint case)."""
    return cheetah_n50(seed=seed, N=N, n_sub=n_sub)


@dataclass
class Batch:
    robots: list          # distinct robots (models)
    model_idx: np.ndarray  # [n_inst]
    Ns: np.ndarray
    n_subs: np.ndarray
    seed: int
    s_range: tuple
    styles: list

    def instance(self, i):
        """Regenerate instance i alone from its own child stream."""
        child = np.random.default_rng(self._child_seeds()[i])
        r = self.robots[self.model_idx[i]]
        return draw_instance(r, child, int(self.Ns[i]), int(self.n_subs[i]), s_range=self.s_range,
                             with_cotangents=True, **self.styles[self.model_idx[i]])

    def _child_seeds(self):
        # SeedSequence(seed).spawn is independent of how far the root generator
        # advanced while drawing the robots, so any instance regenerates alone.
        if getattr(self, "_seeds", None) is None:
            self._seeds = np.random.SeedSequence(self.seed).spawn(len(self.model_idx))
        return self._seeds

    def __len__(self):
        return len(self.model_idx)


def mixed_batch(seed=0, n_inst=1024):
    """Heterogeneous batch: hopper : biped : 7-link chain = 1 : 1 : 2, horizons
    N ~ U{10..200}, substeps in {4, 8, 16}, s ~ U[0.05, 0.15]."""
    rng = np.random.default_rng(seed)
    robots = [hopper(rng), biped(rng), cheetah7(rng)]
    kinds = np.array([0] * (n_inst // 4) + [1] * (n_inst // 4) + [2] * (n_inst - 2 * (n_inst // 4)))
    model_idx = rng.permutation(kinds).astype(np.int32)
    Ns = rng.integers(10, 201, n_inst).astype(np.int32)
    n_subs = rng.choice(np.array([4, 8, 16]), n_inst).astype(np.int32)
    styles = [_ROBOT_STYLE[r.name] for r in robots]
    return Batch(robots, model_idx, Ns, n_subs, seed, (0.05, 0.15), styles)


def cheetah_sweep(seed=0, n_inst=4096, N=400, n_sub=20):
    """Throughput/precision sweep: n_inst instances of one 7-link chain, N = 400,
    20 substeps, s ~ U[0.01, 0.05]."""
    rng = np.random.default_rng(seed)
    robots = [cheetah7(rng)]
    return Batch(robots, np.zeros(n_inst, dtype=np.int32), np.full(n_inst, N, dtype=np.int32),
                 np.full(n_inst, n_sub, dtype=np.int32), seed, (0.01, 0.05),
                 [_ROBOT_STYLE["cheetah7"]])


def monoped_paper(seed=0, N=14, n_sub=10):
    """The sizes of the paper's monoped scenario (15 nodes, so N = 14
    intervals, 10 integration steps per interval, flat ground) with the
    paper's modelling choices: joint reaction forces eliminated (Eq. (3)),
    RKF45 substeps and the full Eq. (12) auxiliary state; synthetic link
    dimensions, pose +- 0.05 about the standing pose, u ~ U[-1, 1],
    s ~ U[0.05, 0.15]."""
    rng = np.random.default_rng(seed)
    robot = with_cross_states(with_paper_dynamics(monoped(rng)))
    return draw_instance(robot, rng, N, n_sub, s_range=(0.05, 0.15), with_cotangents=True,
                         q_noise=0.05, u_dist="uniform")


def cheetah_paper_sweep(seed=0, N=65536, n_sub=10):
    """The paper's own model on the 7-link chain: joint reaction forces
    eliminated (Eq. (3)), RKF45 substeps, the sinusoidal surface; one instance
    of N intervals, gait +- 0.1, u ~ N(0,1), s ~ U[0.01, 0.05]."""
    rng = np.random.default_rng(seed)
    robot = with_paper_dynamics(cheetah7(rng), terrain=TERRAIN_SINE)
    return draw_instance(robot, rng, N, n_sub, s_range=(0.01, 0.05), **_ROBOT_STYLE["cheetah7"])
