"""ctypes front end of ``oracle.cpp`` (test infrastructure; argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _CModel(ctypes.Structure):
    _fields_ = [
        ("nb", ctypes.c_int), ("nj", ctypes.c_int), ("nc", ctypes.c_int),
        ("mass", _dp), ("inertia", _dp),
        ("jparent", _ip), ("jchild", _ip),
        ("jrho_p", _dp), ("jrho_c", _dp),
        ("cbody", _ip), ("crho", _dp), ("cmu", _dp),
        ("g", ctypes.c_double),
        ("aux", ctypes.c_int),
        ("jelim", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("terrain_amp", ctypes.c_double),
        ("terrain_k", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``liboracle.so`` next to it (g++, -O2)."""
    stale = lambda: not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)  # noqa: E731
    if force or stale():
        import fcntl
        with open(_LIB + ".lock", "w") as lk:
            fcntl.flock(lk, fcntl.LOCK_EX)  # one build at a time (parallel test workers)
            if force or stale():
                tmp = _LIB + f".tmp{os.getpid()}"
                subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                                       _SRC, "-o", tmp])
                os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # CISCVX_ORACLE_LIB points at an alternate build of oracle.cpp; the
            # mutation test uses it to show that the pins reject planted errors.
            alt = os.environ.get("CISCVX_ORACLE_LIB")
            lib = ctypes.CDLL(alt if alt else build())
            lib.oracle_dims.argtypes = [ctypes.POINTER(_CModel), _ip, _ip]
            lib.oracle_rhs.argtypes = [ctypes.POINTER(_CModel), _dp, _dp, _dp]
            lib.oracle_flow.argtypes = [ctypes.POINTER(_CModel), ctypes.c_int, _dp, _dp, _dp,
                                        ctypes.c_double, _dp]
            lib.oracle_interval.argtypes = [ctypes.POINTER(_CModel), ctypes.c_int, _dp, _dp, _dp,
                                            ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
            lib.oracle_discretize.argtypes = [ctypes.POINTER(_CModel), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                              _dp, _dp, ctypes.c_int]
            lib.oracle_vjp.argtypes = [ctypes.POINTER(_CModel), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                       ctypes.c_int]
            lib.oracle_linear_interval.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp,
                                                   ctypes.c_int, _dp, _dp, _dp, ctypes.c_double,
                                                   _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
            lib.oracle_tableau.argtypes = [ctypes.c_int, _ip, _dp, _dp, _dp]
            lib.oracle_node.argtypes = [ctypes.POINTER(_CModel), ctypes.c_int, _dp, _dp, _dp, _dp,
                                        ctypes.c_double, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
            lib.oracle_node_value.argtypes = [ctypes.POINTER(_CModel), _dp, _dp, _dp, _dp,
                                              ctypes.c_double, _dp, _dp, _dp]
            lib.oracle_psi.argtypes = [ctypes.POINTER(_CModel), ctypes.c_int, _dp, _dp,
                                       ctypes.c_double, ctypes.c_double, _dp, _dp, ctypes.c_int]
            for f in ("oracle_dims", "oracle_rhs", "oracle_flow", "oracle_interval",
                      "oracle_discretize", "oracle_vjp", "oracle_linear_interval", "oracle_node",
                      "oracle_node_value", "oracle_tableau", "oracle_psi"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


class OracleModel:
    """A robot description held in the oracle's own C layout.

    ``robot`` is a mapping (or object with attributes) giving ``mass`` [nb],
    ``inertia`` [nb], ``joint_parent`` / ``joint_child`` [nj],
    ``joint_rho_parent`` / ``joint_rho_child`` [nj, 2], ``contact_body`` [nc],
    ``contact_rho`` [nc, 2], ``contact_mu`` [nc], ``gravity`` and optionally
    ``aux_model`` (0: one path-penalty state per contact; 1: the full Eq. (12)
    auxiliary state with contact inputs (phi_t, phi_n, gamma)),
    ``joint_forces`` (0: joint reaction forces are inputs; 1: eliminated by
    Eq. (3)), ``scheme`` (0: RK4; 1: RKF45) and ``terrain`` = (amplitude,
    wavenumber) of the contact surface y = a sin(k x) (default flat).
    """

    def __init__(self, robot):
        get = (lambda k: robot[k]) if isinstance(robot, dict) else (lambda k: getattr(robot, k))
        self._keep = {
            "mass": _f64(get("mass")).reshape(-1),
            "inertia": _f64(get("inertia")).reshape(-1),
            "jparent": np.ascontiguousarray(np.asarray(get("joint_parent"), dtype=np.int32).reshape(-1)),
            "jchild": np.ascontiguousarray(np.asarray(get("joint_child"), dtype=np.int32).reshape(-1)),
            "jrho_p": _f64(get("joint_rho_parent")).reshape(-1),
            "jrho_c": _f64(get("joint_rho_child")).reshape(-1),
            "cbody": np.ascontiguousarray(np.asarray(get("contact_body"), dtype=np.int32).reshape(-1)),
            "crho": _f64(get("contact_rho")).reshape(-1),
            "cmu": _f64(get("contact_mu")).reshape(-1),
        }
        k = self._keep
        nb, nj, nc = len(k["mass"]), len(k["jparent"]), len(k["cbody"])
        # zero-length arrays still need a valid pointer
        for key in list(k):
            if k[key].size == 0:
                k[key] = np.zeros(2, dtype=k[key].dtype)
        def opt(key, default):
            try:
                return get(key)
            except (KeyError, AttributeError):
                return default
        aux = int(opt("aux_model", 0))
        jelim = int(opt("joint_forces", 0))
        scheme = int(opt("scheme", 0))
        ta, tk = (float(v) for v in opt("terrain", (0.0, 0.0)))
        self._c = _CModel(nb, nj, nc, _d(k["mass"]), _d(k["inertia"]),
                          k["jparent"].ctypes.data_as(_ip), k["jchild"].ctypes.data_as(_ip),
                          _d(k["jrho_p"]), _d(k["jrho_c"]), k["cbody"].ctypes.data_as(_ip),
                          _d(k["crho"]), _d(k["cmu"]), float(get("gravity")), aux, jelim, scheme,
                          ta, tk)
        self.aux, self.jelim, self.scheme, self.terrain = aux, jelim, scheme, (ta, tk)
        self.nb, self.nj, self.nc = nb, nj, nc
        self.nxt, self.nu = dims(self)
        self.nx = 6 * nb

    @property
    def ptr(self):
        return ctypes.byref(self._c)


def _model(m):
    return m if isinstance(m, OracleModel) else OracleModel(m)


def dims(model):
    lib = _load()
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib.oracle_dims(model.ptr, ctypes.byref(a), ctypes.byref(b)), "dims")
    return a.value, b.value


def rhs(model, xt, u):
    """Unscaled augmented right-hand side (f, Omega) at one point."""
    m = _model(model)
    xt, u = _f64(xt), _f64(u)
    out = np.empty(m.nxt)
    _check(_load().oracle_rhs(m.ptr, _d(xt), _d(u), _d(out)), "rhs")
    return out


def flow(model, n_sub, x0, uL, uR, s):
    """Nonlinear flow map of one interval (plain FP64 RK4)."""
    m = _model(model)
    x0, uL, uR = _f64(x0), _f64(uL), _f64(uR)
    out = np.empty(m.nxt)
    _check(_load().oracle_flow(m.ptr, int(n_sub), _d(x0), _d(uL), _d(uR), float(s), _d(out)), "flow")
    return out


def interval(model, n_sub, x0, uL, uR, s):
    """One interval: returns (x1, A, Bm, Bp, S) from IND."""
    m = _model(model)
    x0, uL, uR = _f64(x0), _f64(uL), _f64(uR)
    x1 = np.empty(m.nxt)
    A = np.empty((m.nxt, m.nxt))
    Bm = np.empty((m.nxt, m.nu))
    Bp = np.empty((m.nxt, m.nu))
    S = np.empty(m.nxt)
    _check(_load().oracle_interval(m.ptr, int(n_sub), _d(x0), _d(uL), _d(uR), float(s), _d(x1),
                                   _d(A), _d(Bm), _d(Bp), _d(S)), "interval")
    return x1, A, Bm, Bp, S


def _layout_code(layout):
    return {"node": 0, "interval": 1, 0: 0, 1: 1}[layout]


def discretize(model, X, U, s, n_sub, layout="node", threads=0):
    """All intervals; returns dict with A, Bm, Bp, S, defect, penalty (FP64)."""
    m = _model(model)
    X, U, s = _f64(X), _f64(U), _f64(s)
    N = s.shape[0]
    out = {
        "A": np.empty((N, m.nxt, m.nxt)), "Bm": np.empty((N, m.nxt, m.nu)),
        "Bp": np.empty((N, m.nxt, m.nu)), "S": np.empty((N, m.nxt)),
        "defect": np.empty((N, m.nxt)), "penalty": np.empty((N, max(m.nc, 0))),
    }
    pen = out["penalty"] if m.nc > 0 else np.empty(1)
    _check(_load().oracle_discretize(m.ptr, N, int(n_sub), _layout_code(layout), _d(X), _d(U),
                                     _d(s), _d(out["A"]), _d(out["Bm"]), _d(out["Bp"]),
                                     _d(out["S"]), _d(out["defect"]), _d(pen), int(threads)),
           "discretize")
    return out


def vjp(model, X, U, s, w, rho, n_sub, layout="node", threads=0):
    """Phi-contracted gradient of L; returns (gX, gU, gs, L)."""
    m = _model(model)
    X, U, s, w = _f64(X), _f64(U), _f64(s), _f64(w)
    rho = _f64(rho) if m.nc > 0 else np.zeros(1)
    N = s.shape[0]
    gX = np.empty_like(X)
    gU = np.empty_like(U)
    gs = np.empty(N)
    L = ctypes.c_double()
    _check(_load().oracle_vjp(m.ptr, N, int(n_sub), _layout_code(layout), _d(X), _d(U), _d(s),
                              _d(w), _d(rho), _d(gX), _d(gU), _d(gs), ctypes.byref(L),
                              int(threads)), "vjp")
    return gX, gU, gs, L.value


def linear_interval(Ac, Bc, n_sub, x0, uL, uR, s, scheme=0):
    """Integrator (scheme 0: RK4, 1: RKF45) + IND on F = Ac x + Bc u; returns (x1, A, Bm, Bp, S)."""
    Ac, Bc = _f64(Ac), _f64(Bc)
    n, mm = Ac.shape[0], Bc.shape[1]
    x0, uL, uR = _f64(x0), _f64(uL), _f64(uR)
    x1 = np.empty(n)
    A = np.empty((n, n))
    Bm = np.empty((n, mm))
    Bp = np.empty((n, mm))
    S = np.empty(n)
    _check(_load().oracle_linear_interval(n, mm, _d(Ac), _d(Bc), int(n_sub), _d(x0), _d(uL),
                                          _d(uR), float(s), _d(x1), _d(A), _d(Bm), _d(Bp),
                                          _d(S), int(scheme)), "linear_interval")
    return x1, A, Bm, Bp, S


def tableau(scheme):
    """Butcher tableau of a scheme: (stages, c [6], a [6, 6], b [6])."""
    st = ctypes.c_int()
    c, a, b = np.empty(6), np.empty((6, 6)), np.empty(6)
    _check(_load().oracle_tableau(int(scheme), ctypes.byref(st), _d(c), _d(a), _d(b)), "tableau")
    return st.value, c, a, b


def _nonempty(a):
    a = _f64(a)
    return a if a.size else np.zeros(1)


def node(model, Xp, Xm, Phi, Gam, delta, e, threads=0):
    """Node constraints G~ and Theta^delta at n nodes with their Jacobians.

    Returns dict g [n, nxt], theta [n, 8 nc], Jg [n, nxt, ncol], Jth [n, 8 nc, ncol]
    with columns z = (x~+ (nxt), x~- (nxt), Phi (2 nc: Phi_t, Phi_n per contact),
    Gamma (nc))."""
    m = _model(model)
    Xp, Xm = _f64(Xp), _f64(Xm)
    n = Xp.shape[0]
    nc = m.nc
    ncol = 2 * m.nxt + 3 * nc
    Phi = _nonempty(np.asarray(Phi, dtype=np.float64).reshape(n, 2 * nc))
    Gam = _nonempty(np.asarray(Gam, dtype=np.float64).reshape(n, nc))
    e = _nonempty(np.asarray(e, dtype=np.float64).reshape(nc))
    out = {"g": np.empty((n, m.nxt)), "theta": np.empty((n, 8 * nc)),
           "Jg": np.empty((n, m.nxt, ncol)), "Jth": np.empty((n, 8 * nc, ncol))}
    th = out["theta"] if nc else np.empty(1)
    jth = out["Jth"] if nc else np.empty(1)
    _check(_load().oracle_node(m.ptr, n, _d(Xp), _d(Xm), _d(Phi), _d(Gam), float(delta), _d(e),
                               _d(out["g"]), _d(th), _d(out["Jg"]), _d(jth), int(threads)), "node")
    return out


def node_value(model, xp, xm, Phi, Gam, delta, e):
    """G~ and Theta^delta at one node in plain FP64 (for finite differences)."""
    m = _model(model)
    nc = m.nc
    g = np.empty(m.nxt)
    th = np.empty(max(8 * nc, 1))
    _check(_load().oracle_node_value(m.ptr, _d(_f64(xp)), _d(_f64(xm)), _d(_nonempty(Phi)),
                                     _d(_nonempty(Gam)), float(delta), _d(_nonempty(e)), _d(g),
                                     _d(th)), "node_value")
    return g, th[:8 * nc]


def psi(model, Xp, Xm, delta, eps, threads=0):
    """Psi^{delta,eps}(y-_{k+1}, y+_k) on the N intervals between N+1 nodes.

    Returns dict psi [N, npsi] and J [N, npsi, 2 ny], columns (y+_k, y-_{k+1});
    npsi = 3 nc for the Eq. (12) auxiliary state, nc for one penalty state per
    contact (rows as in oracle.cpp's oracle_psi)."""
    m = _model(model)
    Xp, Xm = _f64(Xp), _f64(Xm)
    N = Xp.shape[0] - 1
    ny = m.nxt - 6 * m.nb
    npsi = 3 * m.nc if m.aux else m.nc
    out = {"psi": np.empty((N, npsi)), "J": np.empty((N, npsi, 2 * ny))}
    _check(_load().oracle_psi(m.ptr, N, _d(Xp), _d(Xm), float(delta), float(eps),
                              _d(_nonempty(out["psi"])), _d(_nonempty(out["J"])), int(threads)),
           "psi")
    return out
