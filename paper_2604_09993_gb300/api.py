"""Thin Python binding of ``libciscvx.so`` (include/ciscvx.h) with the same entry point names.

Argument marshalling only: tensors are passed to the C ABI as raw device
pointers on PyTorch's current CUDA stream; every step of the computation runs
in the library's CUDA kernels.  There is no fallback: if the library is not
built or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libciscvx.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED = range(7)
PRECISION = {"fp64": 0, "fp32_phi": 1, "tf32_tc": 2, "bf16_tc": 3}
LAYOUT = {"node": 0, "interval": 1}
NODE_THETA_COLS = 12  # CISCVX_NODE_THETA_COLS
OP_DISCRETIZE, OP_VJP = 0, 1
STATIC_SCRATCH_BYTES = 16 * 1024 * 1024  # CISCVX_STATIC_SCRATCH_BYTES

# Every symbol include/ciscvx.h declares.
EXPORTS = (
    "ciscvx_version", "ciscvx_last_error", "ciscvx_model_create", "ciscvx_model_destroy",
    "ciscvx_model_dims", "ciscvx_workspace_size", "ciscvx_discretize", "ciscvx_discretize_vjp",
    "ciscvx_sync_status", "ciscvx_discretize_vjp_static",
    "ciscvx_batch_plan_create", "ciscvx_batch_plan_destroy", "ciscvx_batch_sizes_get",
    "ciscvx_batch_offsets", "ciscvx_batch_get_tune", "ciscvx_batch_discretize",
    "ciscvx_batch_vjp_workspace_size", "ciscvx_batch_discretize_vjp", "ciscvx_batch_autotune",
    "ciscvx_batch_sync_status", "ciscvx_batch_run_host",
    "ciscvx_model_pattern", "ciscvx_model_nnz", "ciscvx_discretize_compact",
    "ciscvx_node_linearize", "ciscvx_batch_discretize_and_vjp", "ciscvx_batch_autotune_fused",
    "ciscvx_batch_get_tune_fused", "ciscvx_discretize_workspace_size", "ciscvx_psi_rows",
    "ciscvx_psi_linearize", "ciscvx_socp_create", "ciscvx_socp_destroy", "ciscvx_socp_get_dims",
    "ciscvx_socp_structure", "ciscvx_socp_fill", "ciscvx_batch_vjp_workspace_sizes",
)
FORMAT = {"dense": 0, "compact": 1}


class Tune(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("lpt_order", ctypes.c_int), ("use_graph", ctypes.c_int), ("occupancy", ctypes.c_int),
                ("split", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class _Sizes(ctypes.Structure):
    _fields_ = [(k, ctypes.c_size_t) for k in ("X", "U", "s", "A", "B", "S", "defect", "penalty", "L")]


class _BatchIO(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("X", "U", "s", "A", "Bm", "Bp", "S", "defect", "penalty")]


class _BatchVjpIO(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("X", "U", "s", "w", "rho", "gX", "gU", "gs", "L")]


_dp = ctypes.POINTER(ctypes.c_double)


class _SocpParams(ctypes.Structure):
    _fields_ = [("w_px", ctypes.c_double), ("w_ep", ctypes.c_double), ("w_torque", ctypes.c_double),
                ("s_min", ctypes.c_double), ("s_max", ctypes.c_double), ("torque_max", _dp),
                ("x_init", _dp), ("x_final", _dp), ("scale_x", _dp), ("offset_x", _dp),
                ("scale_u", _dp), ("offset_u", _dp), ("scale_s", ctypes.c_double),
                ("offset_s", ctypes.c_double), ("scale_phi", _dp), ("offset_phi", _dp),
                ("scale_gam", _dp), ("offset_gam", _dp), ("phi_format", ctypes.c_int)]


class _SocpDims(ctypes.Structure):
    _fields_ = [("n_var", ctypes.c_int), ("n_eq", ctypes.c_int), ("n_ineq", ctypes.c_int),
                ("n_nonneg", ctypes.c_int), ("n_soc", ctypes.c_int), ("nnz_A", ctypes.c_longlong),
                ("nnz_G", ctypes.c_longlong), ("nnz_P", ctypes.c_longlong)]


_SOCP_IN = ("Xp", "Xm", "U", "s", "Phi", "Gam")
_SOCP_IN2 = ("A", "Bm", "Bp", "S", "defect", "g", "Gvm", "Gth", "Gphi", "Gpx", "theta", "dtheta",
             "psi", "dpsi")


class _SocpInputs(ctypes.Structure):
    _fields_ = ([(k, ctypes.c_void_p) for k in _SOCP_IN] + [("phi_precision", ctypes.c_int)] +
                [(k, ctypes.c_void_p) for k in _SOCP_IN2])


_SOCP_OUT = ("A_values", "b", "G_values", "h", "c", "rho_A", "rho_G")


class _SocpOutputs(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in _SOCP_OUT]


class _NodeParams(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("restitution", ctypes.POINTER(ctypes.c_double))]


class CiscvxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ciscvx status {status}: {msg}")
        self.status = status


class _Body(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("inertia", ctypes.c_double)]


class _Joint(ctypes.Structure):
    _fields_ = [("parent", ctypes.c_int), ("child", ctypes.c_int),
                ("rho_parent", ctypes.c_double * 2), ("rho_child", ctypes.c_double * 2)]


class _Contact(ctypes.Structure):
    _fields_ = [("body", ctypes.c_int), ("rho", ctypes.c_double * 2), ("mu", ctypes.c_double)]


class _Desc(ctypes.Structure):
    _fields_ = [("n_bodies", ctypes.c_int), ("n_joints", ctypes.c_int),
                ("n_contacts", ctypes.c_int), ("bodies", ctypes.POINTER(_Body)),
                ("joints", ctypes.POINTER(_Joint)), ("contacts", ctypes.POINTER(_Contact)),
                ("gravity", ctypes.c_double), ("aux_model", ctypes.c_int),
                ("joint_forces", ctypes.c_int), ("scheme", ctypes.c_int),
                ("terrain_amp", ctypes.c_double), ("terrain_wavenumber", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def load(path: str | None = None):
    """Open the library (it must have been built, e.g. by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    lib.ciscvx_version.restype = ctypes.c_int
    lib.ciscvx_last_error.restype = ctypes.c_char_p
    lib.ciscvx_model_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(_vp)]
    lib.ciscvx_model_destroy.argtypes = [_vp]
    lib.ciscvx_model_destroy.restype = None
    lib.ciscvx_model_dims.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.ciscvx_workspace_size.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]
    lib.ciscvx_discretize_workspace_size.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_int,
                                                     ctypes.POINTER(ctypes.c_size_t),
                                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.ciscvx_discretize.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                      ctypes.c_size_t, _vp]
    lib.ciscvx_discretize_vjp.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                          _vp, _vp, ctypes.c_size_t, _vp]
    lib.ciscvx_sync_status.argtypes = [_vp, _vp]
    I32 = ctypes.POINTER(ctypes.c_int32)
    lib.ciscvx_model_pattern.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), I32, I32, I32, I32]
    lib.ciscvx_model_nnz.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.ciscvx_node_linearize.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp,
                                          ctypes.POINTER(_NodeParams), _vp, _vp, _vp, _vp, _vp,
                                          _vp, _vp, _vp]
    lib.ciscvx_psi_rows.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
    lib.ciscvx_psi_linearize.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                         _vp, _vp, _vp]
    lib.ciscvx_socp_create.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_SocpParams),
                                       ctypes.POINTER(_vp)]
    lib.ciscvx_socp_destroy.argtypes = [_vp]
    lib.ciscvx_socp_destroy.restype = None
    lib.ciscvx_socp_get_dims.argtypes = [_vp, ctypes.POINTER(_SocpDims)]
    _ip32 = ctypes.POINTER(ctypes.c_int)
    lib.ciscvx_socp_structure.argtypes = [_vp, _ip32, _ip32, _ip32, _ip32, _ip32, _ip32, _dp]
    lib.ciscvx_socp_fill.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(_SocpInputs),
                                     ctypes.POINTER(_SocpOutputs), _vp]
    lib.ciscvx_discretize_compact.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                              _vp, _vp, _vp, ctypes.c_size_t, _vp]
    lib.ciscvx_discretize_vjp_static.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                                 _vp, _vp, _vp]
    P = ctypes.POINTER
    lib.ciscvx_batch_plan_create.argtypes = [P(_vp), ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                             P(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, P(Tune), P(_vp)]
    lib.ciscvx_batch_plan_destroy.argtypes = [_vp]
    lib.ciscvx_batch_plan_destroy.restype = None
    lib.ciscvx_batch_sizes_get.argtypes = [_vp, P(_Sizes)]
    lib.ciscvx_batch_offsets.argtypes = [_vp, ctypes.c_int, P(_Sizes)]
    lib.ciscvx_batch_get_tune.argtypes = [_vp, P(Tune)]
    lib.ciscvx_batch_discretize.argtypes = [_vp, P(_BatchIO), _vp]
    lib.ciscvx_batch_vjp_workspace_size.argtypes = [_vp, P(ctypes.c_size_t)]
    lib.ciscvx_batch_vjp_workspace_sizes.argtypes = [_vp, P(ctypes.c_size_t), P(ctypes.c_size_t)]
    lib.ciscvx_batch_discretize_vjp.argtypes = [_vp, P(_BatchVjpIO), _vp, ctypes.c_size_t, _vp]
    lib.ciscvx_batch_autotune.argtypes = [_vp, P(_BatchIO), _vp, P(Tune)]
    lib.ciscvx_batch_discretize_and_vjp.argtypes = [_vp, P(_BatchIO), P(_BatchVjpIO), _vp,
                                                    ctypes.c_size_t, _vp]
    lib.ciscvx_batch_autotune_fused.argtypes = [_vp, P(_BatchIO), P(_BatchVjpIO), _vp,
                                                ctypes.c_size_t, _vp, P(Tune)]
    lib.ciscvx_batch_get_tune_fused.argtypes = [_vp, P(Tune)]
    lib.ciscvx_batch_sync_status.argtypes = [_vp, _vp]
    lib.ciscvx_batch_run_host.argtypes = [_vp, ctypes.c_int, P(_BatchIO), P(_BatchIO), P(_BatchVjpIO),
                                          P(_BatchVjpIO), _vp, ctypes.c_size_t, _vp]
    lib.ciscvx_batch_run_host.restype = ctypes.c_int
    for f in ("ciscvx_model_create", "ciscvx_model_dims", "ciscvx_workspace_size",
              "ciscvx_discretize", "ciscvx_discretize_vjp", "ciscvx_sync_status",
              "ciscvx_discretize_vjp_static", "ciscvx_batch_plan_create", "ciscvx_batch_sizes_get",
              "ciscvx_batch_offsets", "ciscvx_batch_get_tune", "ciscvx_batch_discretize",
              "ciscvx_batch_vjp_workspace_size", "ciscvx_batch_discretize_vjp",
              "ciscvx_batch_autotune", "ciscvx_batch_sync_status", "ciscvx_model_pattern",
              "ciscvx_model_nnz", "ciscvx_discretize_compact", "ciscvx_node_linearize",
              "ciscvx_batch_discretize_and_vjp", "ciscvx_batch_autotune_fused",
              "ciscvx_batch_get_tune_fused", "ciscvx_discretize_workspace_size"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st):
    if st != OK:
        raise CiscvxError(st, _lib.ciscvx_last_error().decode())


def _get(robot, key):
    return robot[key] if isinstance(robot, dict) else getattr(robot, key)


class _DescHolder:
    """A ``ciscvx_model_desc`` for a robot description, with the host arrays it points to."""

    def __init__(self, robot):
        mass = np.asarray(_get(robot, "mass"), dtype=np.float64)
        inertia = np.asarray(_get(robot, "inertia"), dtype=np.float64)
        jp = np.asarray(_get(robot, "joint_parent"), dtype=np.int64)
        jc = np.asarray(_get(robot, "joint_child"), dtype=np.int64)
        rp = np.asarray(_get(robot, "joint_rho_parent"), dtype=np.float64).reshape(-1, 2)
        rc = np.asarray(_get(robot, "joint_rho_child"), dtype=np.float64).reshape(-1, 2)
        cb = np.asarray(_get(robot, "contact_body"), dtype=np.int64)
        cr = np.asarray(_get(robot, "contact_rho"), dtype=np.float64).reshape(-1, 2)
        cm = np.asarray(_get(robot, "contact_mu"), dtype=np.float64)
        nb, nj, nc = len(mass), len(jp), len(cb)
        self._bodies = (_Body * max(nb, 1))(*[_Body(mass[i], inertia[i]) for i in range(nb)])
        self._joints = (_Joint * max(nj, 1))(*[
            _Joint(int(jp[j]), int(jc[j]), (ctypes.c_double * 2)(*rp[j]), (ctypes.c_double * 2)(*rc[j]))
            for j in range(nj)])
        self._contacts = (_Contact * max(nc, 1))(*[
            _Contact(int(cb[i]), (ctypes.c_double * 2)(*cr[i]), cm[i]) for i in range(nc)])
        def opt(key, default):
            try:
                return _get(robot, key)
            except (KeyError, AttributeError):
                return default
        aux = int(opt("aux_model", 0))
        jf = int(opt("joint_forces", 0))
        scheme = int(opt("scheme", 0))
        ta, tk = (float(v) for v in opt("terrain", (0.0, 0.0)))
        self.desc = _Desc(nb, nj, nc, self._bodies, self._joints, self._contacts,
                          float(_get(robot, "gravity")), aux, jf, scheme, ta, tk)
        self.nb, self.nj, self.nc, self.aux_model = nb, nj, nc, aux
        self.coupled = bool(jf or scheme or ta != 0.0)


def model_pattern(robot):
    """ciscvx_model_pattern (host only, no GPU): the structural nonzeros of A and
    of B-/B+ in compact order, as int32 arrays (a_row, a_col, b_row, b_col)."""
    lib = load()
    d = _DescHolder(robot)
    na, nb_ = ctypes.c_int(), ctypes.c_int()
    _check(lib.ciscvx_model_pattern(ctypes.byref(d.desc), ctypes.byref(na), ctypes.byref(nb_),
                                    None, None, None, None))
    arrs = [np.zeros(max(n, 1), dtype=np.int32) for n in (na.value, na.value, nb_.value, nb_.value)]
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in arrs]
    _check(lib.ciscvx_model_pattern(ctypes.byref(d.desc), None, None, *ptrs))
    return arrs[0][:na.value], arrs[1][:na.value], arrs[2][:nb_.value], arrs[3][:nb_.value]


class Model:
    """``ciscvx_model`` built from a robot description (synth.Robot or a dict
    with mass, inertia, joint_*, contact_*, gravity)."""

    def __init__(self, robot):
        lib = load()
        self._d = _DescHolder(robot)
        h = _vp()
        _check(lib.ciscvx_model_create(ctypes.byref(self._d.desc), ctypes.byref(h)))
        self._h = h
        nx, ny, nu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.ciscvx_model_dims(h, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nu)))
        self.nx, self.ny, self.nu = nx.value, ny.value, nu.value
        self.nxt = self.nx + self.ny
        self.nb = self._d.nb
        self.nj = self._d.nj
        self.nc = self._d.nc            # contacts (penalty / rho columns)
        self.aux_model = self._d.aux_model
        # eliminated joint forces, a sinusoidal surface or RKF45: the coupled path
        self.coupled = self._d.coupled
        na, nbb = ctypes.c_int(), ctypes.c_int()
        _check(lib.ciscvx_model_nnz(h, ctypes.byref(na), ctypes.byref(nbb)))
        self.nnz_a, self.nnz_b = na.value, nbb.value
        self._robot = robot

    def pattern(self):
        """(a_row, a_col, b_row, b_col) of the compact outputs (see model_pattern)."""
        return model_pattern(self._robot)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ciscvx_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, name, dtype):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def workspace_size(model: Model, op: int, N: int, layout: str = "node") -> int:
    n = ctypes.c_size_t()
    _check(load().ciscvx_workspace_size(model.handle, op, int(N), LAYOUT[layout], ctypes.byref(n)))
    return n.value


def discretize_workspace_size(model: Model, N: int, n_sub: int, precision: str = "fp64",
                              op: int = OP_DISCRETIZE, layout: str = "node"):
    """ciscvx_discretize_workspace_size: (min_bytes, full_bytes) of scratch for `op`."""
    lo, hi = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().ciscvx_discretize_workspace_size(model.handle, int(op), int(N), int(n_sub),
                                                   PRECISION[precision], LAYOUT[layout],
                                                   ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


# default cap on the scratch a discretize call allocates for a coupled model
DISCRETIZE_WS_CAP = 2 << 30


def _coupled_workspace(model: Model, N: int, n_sub: int, precision: str, layout: str, workspace, dev):
    """The scratch of a coupled model's linearization: the given one, else one of
    min(full size, DISCRETIZE_WS_CAP) bytes (at least the minimum); None for
    the other models."""
    import torch
    if not model.coupled:
        return None
    if workspace is None:
        lo, hi = discretize_workspace_size(model, N, n_sub, precision, OP_DISCRETIZE, layout)
        workspace = torch.empty(max(lo, min(hi, DISCRETIZE_WS_CAP)), dtype=torch.uint8, device=dev)
    return workspace


def discretize(model: Model, X, U, s, n_sub: int, precision: str = "fp64", layout: str = "node",
               want_z: bool = False, out: dict | None = None, workspace=None):
    """ciscvx_discretize on device tensors.  Returns dict A, Bm, Bp, S, defect, penalty (, z).
    A model with coupled links needs scratch: `workspace` (a CUDA uint8 tensor),
    else one of min(full size, 2 GiB) (at least the minimum) is allocated."""
    import torch
    f64 = torch.float64
    _need(X, "X", f64); _need(U, "U", f64); _need(s, "s", f64)
    N = s.shape[0]
    nxt, nu, nc = model.nxt, model.nu, model.nc
    pdt = f64 if precision == "fp64" else torch.float32
    dev = X.device
    if out is None:
        out = {
            "A": torch.empty((N, nxt, nxt), dtype=pdt, device=dev),
            "Bm": torch.empty((N, nxt, nu), dtype=pdt, device=dev),
            "Bp": torch.empty((N, nxt, nu), dtype=pdt, device=dev),
            "S": torch.empty((N, nxt), dtype=pdt, device=dev),
            "defect": torch.empty((N, nxt), dtype=f64, device=dev),
            "penalty": torch.empty((N, nc), dtype=f64, device=dev),
        }
        if want_z:
            out["z"] = torch.empty((N, nxt), dtype=f64, device=dev)
    workspace = _coupled_workspace(model, N, n_sub, precision, layout, workspace, dev)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(load().ciscvx_discretize(
        model.handle, int(N), int(n_sub), PRECISION[precision], LAYOUT[layout], _ptr(X), _ptr(U),
        _ptr(s), _ptr(out["A"]), _ptr(out["Bm"]) if nu else None, _ptr(out["Bp"]) if nu else None,
        _ptr(out["S"]), _ptr(out["defect"]), _ptr(out["penalty"]) if nc else None,
        _ptr(out.get("z")), _ptr(workspace) if workspace is not None else None, ws_bytes, _stream()))
    return out


def discretize_compact(model: Model, X, U, s, n_sub: int, precision: str = "fp64",
                       layout: str = "node", want_z: bool = False, out: dict | None = None,
                       workspace=None):
    """ciscvx_discretize_compact: as discretize, with A (N, nnz_a) and Bm/Bp
    (N, nnz_b) holding the structural nonzeros in Model.pattern() order.  A
    model with coupled links needs scratch as for discretize."""
    import torch
    f64 = torch.float64
    _need(X, "X", f64); _need(U, "U", f64); _need(s, "s", f64)
    N = s.shape[0]
    nxt, nc = model.nxt, model.nc
    pdt = f64 if precision == "fp64" else torch.float32
    dev = X.device
    if out is None:
        out = {
            "A": torch.empty((N, model.nnz_a), dtype=pdt, device=dev),
            "Bm": torch.empty((N, model.nnz_b), dtype=pdt, device=dev),
            "Bp": torch.empty((N, model.nnz_b), dtype=pdt, device=dev),
            "S": torch.empty((N, nxt), dtype=pdt, device=dev),
            "defect": torch.empty((N, nxt), dtype=f64, device=dev),
            "penalty": torch.empty((N, nc), dtype=f64, device=dev),
        }
        if want_z:
            out["z"] = torch.empty((N, nxt), dtype=f64, device=dev)
    nzb = model.nnz_b > 0
    workspace = _coupled_workspace(model, N, n_sub, precision, layout, workspace, dev)
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(load().ciscvx_discretize_compact(
        model.handle, int(N), int(n_sub), PRECISION[precision], LAYOUT[layout], _ptr(X), _ptr(U),
        _ptr(s), _ptr(out["A"]), _ptr(out["Bm"]) if nzb else None, _ptr(out["Bp"]) if nzb else None,
        _ptr(out["S"]), _ptr(out["defect"]), _ptr(out["penalty"]) if nc else None,
        _ptr(out.get("z")), _ptr(workspace) if workspace is not None else None, ws_bytes, _stream()))
    return out


def node_linearize(model: Model, Xp, Xm, Phi, Gam, delta: float, restitution,
                   jacobians: bool = True, out: dict | None = None):
    """ciscvx_node_linearize: node constraints G~ / Theta^delta and their Jacobians.

    Xp, Xm [n, nxt], Phi [n, 2 nc], Gam [n, nc]: device float64 tensors;
    restitution: nc host floats.  Returns dict g, theta and, with jacobians,
    Gvm, Gth, Gphi, Gpx, dtheta (layouts in include/ciscvx.h)."""
    import torch
    f64 = torch.float64
    _need(Xp, "Xp", f64); _need(Xm, "Xm", f64)
    n = Xp.shape[0]
    nq, nc, nb = 3 * model.nb, model.nc, model.nb
    dev = Xp.device
    if nc:
        _need(Phi, "Phi", f64); _need(Gam, "Gam", f64)
    if out is None:
        out = {"g": torch.empty((n, model.nxt), dtype=f64, device=dev),
               "theta": torch.empty((n, nc, 8), dtype=f64, device=dev)}
        if jacobians:
            out.update(Gvm=torch.empty((n, nq, nq), dtype=f64, device=dev),
                       Gth=torch.empty((n, nq, nb), dtype=f64, device=dev),
                       Gphi=torch.empty((n, nq, 2 * nc), dtype=f64, device=dev),
                       Gpx=torch.empty((n, nq, nc), dtype=f64, device=dev),
                       dtheta=torch.empty((n, nc, 8, NODE_THETA_COLS), dtype=f64, device=dev))
    e = (ctypes.c_double * max(nc, 1))(*[float(v) for v in np.asarray(restitution, dtype=np.float64).reshape(-1)])
    prm = _NodeParams(float(delta), e)
    has = lambda k: _ptr(out[k]) if out.get(k) is not None and (nc or k not in ("theta", "Gphi", "Gpx", "dtheta")) else None  # noqa: E731
    _check(load().ciscvx_node_linearize(
        model.handle, int(n), _ptr(Xp), _ptr(Xm), _ptr(Phi) if nc else None, _ptr(Gam) if nc else None,
        ctypes.byref(prm), _ptr(out["g"]), has("Gvm"), has("Gth"), has("Gphi"), has("Gpx"),
        has("theta"), has("dtheta"), _stream()))
    return out


def psi_rows(model: Model) -> int:
    """ciscvx_psi_rows: rows of Psi^{delta,eps} per interval (3 nc or nc)."""
    n = ctypes.c_int()
    _check(load().ciscvx_psi_rows(model.handle, ctypes.byref(n)))
    return n.value


def psi_linearize(model: Model, Xp, Xm, delta: float, epsilon: float, jacobian: bool = True,
                  out: dict | None = None):
    """ciscvx_psi_linearize: Psi^{delta,eps}(y-_{k+1}, y+_k) and d Psi / d y-_{k+1}.

    Xp, Xm [N+1, nxt] device float64 tensors.  Returns dict psi [N, n_psi] and,
    with jacobian, dpsi [N, n_psi, n_y] (the Jacobian in y+_k is -dpsi)."""
    import torch
    f64 = torch.float64
    _need(Xp, "Xp", f64); _need(Xm, "Xm", f64)
    N = Xp.shape[0] - 1
    npsi, ny = psi_rows(model), model.nxt - 6 * model.nb
    if out is None:
        out = {"psi": torch.empty((N, npsi), dtype=f64, device=Xp.device)}
        if jacobian:
            out["dpsi"] = torch.empty((N, npsi, ny), dtype=f64, device=Xp.device)
    _check(load().ciscvx_psi_linearize(
        model.handle, int(N), _ptr(Xp), _ptr(Xm), float(delta), float(epsilon),
        _ptr(out["psi"]) if npsi else None,
        _ptr(out["dpsi"]) if npsi and out.get("dpsi") is not None else None, _stream()))
    return out


def discretize_vjp(model: Model, X, U, s, w, rho, n_sub: int, precision: str = "fp64",
                   layout: str = "node", workspace=None, want_L: bool = True):
    """ciscvx_discretize_vjp on device tensors.  Returns (gX, gU, gs, L or None)."""
    import torch
    f64 = torch.float64
    for t, nm in ((X, "X"), (U, "U"), (s, "s"), (w, "w")):
        _need(t, nm, f64)
    if model.nc:
        _need(rho, "rho", f64)
    N = s.shape[0]
    lo, hi = discretize_workspace_size(model, N, n_sub, precision, OP_VJP, layout)
    if workspace is None or workspace.numel() * workspace.element_size() < lo:
        workspace = torch.empty(max(lo, min(hi, DISCRETIZE_WS_CAP), 16), dtype=torch.uint8,
                                device=X.device)
    gX = torch.empty_like(X)
    gU = torch.empty_like(U)
    gs = torch.empty_like(s)
    L = torch.empty((), dtype=f64, device=X.device) if want_L else None
    _check(load().ciscvx_discretize_vjp(
        model.handle, int(N), int(n_sub), PRECISION[precision], LAYOUT[layout], _ptr(X), _ptr(U),
        _ptr(s), _ptr(w), _ptr(rho) if model.nc else None, _ptr(gX), _ptr(gU) if model.nu else None,
        _ptr(gs), _ptr(L), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream()))
    return gX, gU, gs, L


def discretize_vjp_static(model: Model, X, U, s, w, rho, n_sub: int, precision: str = "fp64",
                          layout: str = "node", want_L: bool = True):
    """ciscvx_discretize_vjp_static: the VJP with the library's built-in scratch
    (no workspace, no device allocation inside the call).  Returns (gX, gU, gs, L or None)."""
    import torch
    f64 = torch.float64
    for t, nm in ((X, "X"), (U, "U"), (s, "s"), (w, "w")):
        _need(t, nm, f64)
    if model.nc:
        _need(rho, "rho", f64)
    gX = torch.empty_like(X)
    gU = torch.empty_like(U)
    gs = torch.empty_like(s)
    L = torch.empty((), dtype=f64, device=X.device) if want_L else None
    _check(load().ciscvx_discretize_vjp_static(
        model.handle, int(s.shape[0]), int(n_sub), PRECISION[precision], LAYOUT[layout], _ptr(X),
        _ptr(U), _ptr(s), _ptr(w), _ptr(rho) if model.nc else None, _ptr(gX),
        _ptr(gU) if model.nu else None, _ptr(gs), _ptr(L), _stream()))
    return gX, gU, gs, L


def sync_status(model: Model):
    """Waits for the current stream and raises if the device flagged a non-finite result."""
    _check(load().ciscvx_sync_status(model.handle, _stream()))


def _make_function():
    import torch

    class Discretize(torch.autograd.Function):
        """(X, U, s) -> (defect, penalty) through ciscvx_discretize; the backward
        pass is ciscvx_discretize_vjp with cotangents w = dL/ddefect and
        rho = dL/dpenalty (the adjoint kernel, not autograd tracing)."""

        @staticmethod
        def forward(ctx, X, U, s, model, n_sub, precision, layout):
            out = discretize(model, X, U, s, n_sub, precision, layout)
            ctx.save_for_backward(X, U, s)
            ctx.cfg = (model, n_sub, precision, layout)
            return out["defect"], out["penalty"]

        @staticmethod
        def backward(ctx, gdef, gpen):
            X, U, s = ctx.saved_tensors
            model, n_sub, precision, layout = ctx.cfg
            w = torch.zeros((s.shape[0], model.nxt), dtype=X.dtype, device=X.device) \
                if gdef is None else gdef.contiguous()
            rho = torch.zeros((s.shape[0], model.nc), dtype=X.dtype, device=X.device) \
                if gpen is None else gpen.contiguous()
            gX, gU, gs, _ = discretize_vjp(model, X, U, s, w, rho, n_sub, precision, layout,
                                           want_L=False)
            return gX, gU, gs, None, None, None, None

    return Discretize


_Discretize = None


def discretize_fn(model: Model, X, U, s, n_sub: int, precision: str = "fp64", layout: str = "node"):
    """Differentiable (defect, penalty) = F(X, U, s) (torch.autograd.Function)."""
    global _Discretize
    if _Discretize is None:
        _Discretize = _make_function()
    return _Discretize.apply(X, U, s, model, n_sub, precision, layout)


def _host_vec(v, n, name):
    if v is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
    if a.size != n:
        raise ValueError(f"{name} must hold {n} values")
    return a, a.ctypes.data_as(_dp)


class Socp:
    """ciscvx_socp: the SCP subproblem of one (model, N, layout) shape as a
    canonical SOCP (CSC structure on the host, values filled on the GPU for
    any number of instances).  Keyword parameters as ciscvx_socp_params; the
    scale/offset pairs are dicts {"x": (scale, offset), "u": ..., "s": ...,
    "phi": ..., "gam": ...} (each entry optional)."""

    def __init__(self, model: Model, N: int, layout: str = "node", *, w_px, w_ep, w_torque, s_min, s_max,
                 torque_max, x_init, x_final, scaling=None, phi_format: str = "dense"):
        lib = load()
        self.model, self.N, self.layout = model, int(N), layout
        sc = scaling or {}
        nx = 6 * model.nb
        keep = []

        def vec(v, n, name):
            a, p = _host_vec(v, n, name)
            keep.append(a)
            return p

        def pair(key, n):
            s_, o_ = sc.get(key, (None, None))
            return vec(s_, n, f"scale_{key}"), vec(o_, n, f"offset_{key}")

        sx, ox = pair("x", model.nxt)
        su, ou = pair("u", model.nu)
        sp, op = pair("phi", 2 * model.nc)
        sg, og = pair("gam", model.nc)
        ss, os_ = sc.get("s", (0.0, 0.0))
        prm = _SocpParams(float(w_px), float(w_ep), float(w_torque), float(s_min), float(s_max),
                          vec(torque_max, model.nj, "torque_max") if model.nj else None,
                          vec(x_init, nx, "x_init"), vec(x_final, nx, "x_final"), sx, ox, su, ou,
                          float(ss or 0.0), float(os_ or 0.0), sp, op, sg, og, FORMAT[phi_format])
        h = _vp()
        _check(lib.ciscvx_socp_create(model.handle, self.N, LAYOUT[layout], ctypes.byref(prm), ctypes.byref(h)))
        self._h = h
        d = _SocpDims()
        _check(lib.ciscvx_socp_get_dims(h, ctypes.byref(d)))
        self.dims = {f: getattr(d, f) for f, _ in d._fields_}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            load().ciscvx_socp_destroy(h)
            self._h = None

    def structure(self):
        """Host CSC index arrays of A, G and P, and P's values (numpy)."""
        d = self.dims
        i32 = lambda n: np.zeros(max(int(n), 1), dtype=np.int32)  # noqa: E731
        out = {"A_colptr": i32(d["n_var"] + 1), "A_rowind": i32(d["nnz_A"]),
               "G_colptr": i32(d["n_var"] + 1), "G_rowind": i32(d["nnz_G"]),
               "P_colptr": i32(d["n_var"] + 1), "P_rowind": i32(d["nnz_P"]),
               "P_values": np.zeros(max(int(d["nnz_P"]), 1))}
        ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))  # noqa: E731
        _check(load().ciscvx_socp_structure(self._h, ip(out["A_colptr"]), ip(out["A_rowind"]),
                                            ip(out["G_colptr"]), ip(out["G_rowind"]), ip(out["P_colptr"]),
                                            ip(out["P_rowind"]), out["P_values"].ctypes.data_as(_dp)))
        for k, n in (("A_rowind", d["nnz_A"]), ("G_rowind", d["nnz_G"]), ("P_rowind", d["nnz_P"]),
                     ("P_values", d["nnz_P"])):
            out[k] = out[k][:int(n)]
        return out

    def alloc_outputs(self, n_inst: int, device):
        import torch
        d = self.dims
        f = lambda n: torch.empty((n_inst, int(n)), dtype=torch.float64, device=device)  # noqa: E731
        return {"A_values": f(d["nnz_A"]), "b": f(d["n_eq"]), "G_values": f(d["nnz_G"]),
                "h": f(d["n_ineq"]), "c": f(d["n_var"]), "rho_A": f(d["n_eq"]), "rho_G": f(d["n_ineq"])}

    def fill(self, n_inst: int, inputs: dict, out: dict | None = None, precision: str = "fp64"):
        """ciscvx_socp_fill: inputs maps Xp, Xm, U, s, Phi, Gam, A, Bm, Bp, S, defect, g, Gvm, Gth,
        Gphi, Gpx, theta, dtheta, psi, dpsi to contiguous device tensors (instances concatenated)."""
        import torch
        if out is None:
            out = self.alloc_outputs(n_inst, inputs["Xp"].device)
        ptr = lambda k: _ptr(inputs.get(k))  # noqa: E731
        for k, t in inputs.items():
            if t is not None and not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise ValueError(f"{k} must be a contiguous CUDA tensor")
        ins = _SocpInputs(*[ptr(k) for k in _SOCP_IN], PRECISION[precision], *[ptr(k) for k in _SOCP_IN2])
        outs = _SocpOutputs(*[_ptr(out[k]) for k in _SOCP_OUT])
        _check(load().ciscvx_socp_fill(self._h, int(n_inst), ctypes.byref(ins), ctypes.byref(outs), _stream()))
        return out


class BatchPlan:
    """``ciscvx_batch_plan``: n instances, instance i using ``models[model_idx[i]]``
    with ``N[i]`` intervals and ``n_sub[i]`` substeps; arrays are packed back to
    back in instance order (see include/ciscvx.h)."""

    def __init__(self, models, model_idx, N, n_sub, precision="fp32_phi", layout="node",
                 tune: dict | None = None, out_format: str = "dense"):
        lib = load()
        self.models = list(models)
        self.model_idx = np.asarray(model_idx, dtype=np.int32)
        self.N = np.asarray(N, dtype=np.int32)
        self.n_sub = np.asarray(n_sub, dtype=np.int32)
        self.n_inst = len(self.model_idx)
        self.precision, self.layout, self.out_format = precision, layout, out_format
        hs = (_vp * len(self.models))(*[m.handle for m in self.models])
        ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))  # noqa: E731
        t = Tune(**tune) if tune else None
        h = _vp()
        _check(lib.ciscvx_batch_plan_create(hs, len(self.models), ip(self.model_idx), ip(self.N),
                                            ip(self.n_sub), self.n_inst, PRECISION[precision],
                                            LAYOUT[layout], FORMAT[out_format],
                                            ctypes.byref(t) if t else None,
                                            ctypes.byref(h)))
        self._h = h
        sz = _Sizes()
        _check(lib.ciscvx_batch_sizes_get(h, ctypes.byref(sz)))
        self.sizes = {k: getattr(sz, k) for k, _ in _Sizes._fields_}
        offs = []
        for i in range(self.n_inst):
            o = _Sizes()
            _check(lib.ciscvx_batch_offsets(h, i, ctypes.byref(o)))
            offs.append({k: getattr(o, k) for k, _ in _Sizes._fields_})
        self.offsets = offs

    @property
    def handle(self):
        return self._h

    def tune(self):
        t = Tune()
        _check(load().ciscvx_batch_get_tune(self._h, ctypes.byref(t)))
        return t.as_dict()

    def alloc_outputs(self, device):
        import torch
        pdt = torch.float64 if self.precision == "fp64" else torch.float32
        z = self.sizes
        return {
            "A": torch.empty(max(z["A"], 1), dtype=pdt, device=device),
            "Bm": torch.empty(max(z["B"], 1), dtype=pdt, device=device),
            "Bp": torch.empty(max(z["B"], 1), dtype=pdt, device=device),
            "S": torch.empty(max(z["S"], 1), dtype=pdt, device=device),
            "defect": torch.empty(max(z["defect"], 1), dtype=torch.float64, device=device),
            "penalty": torch.empty(max(z["penalty"], 1), dtype=torch.float64, device=device),
        }

    def _io(self, X, U, s, out):
        return _BatchIO(*[t.data_ptr() for t in (X, U, s, out["A"], out["Bm"], out["Bp"], out["S"],
                                                 out["defect"], out["penalty"])])

    def discretize(self, X, U, s, out=None):
        """ciscvx_batch_discretize on packed device tensors; returns the packed outputs."""
        if out is None:
            out = self.alloc_outputs(X.device)
        io = self._io(X, U, s, out)
        _check(load().ciscvx_batch_discretize(self._h, ctypes.byref(io), _stream()))
        return out

    def autotune(self, X, U, s, out=None):
        if out is None:
            out = self.alloc_outputs(X.device)
        io = self._io(X, U, s, out)
        t = Tune()
        _check(load().ciscvx_batch_autotune(self._h, ctypes.byref(io), _stream(), ctypes.byref(t)))
        return t.as_dict()

    def vjp_workspace_size(self):
        n = ctypes.c_size_t()
        _check(load().ciscvx_batch_vjp_workspace_size(self._h, ctypes.byref(n)))
        return n.value

    def vjp_workspace_sizes(self):
        """(min, full) bytes of VJP scratch (equal: see ciscvx_batch_vjp_workspace_sizes)."""
        lo, hi = ctypes.c_size_t(), ctypes.c_size_t()
        _check(load().ciscvx_batch_vjp_workspace_sizes(self._h, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def discretize_vjp(self, X, U, s, w, rho, workspace=None, want_L=True, out=None):
        """ciscvx_batch_discretize_vjp; returns dict gX, gU, gs, L (per instance).
        A given workspace of at least the minimum is used as it is (a larger
        one gives the coupled instances' adjoint larger chunks); without one
        (or with a smaller one) one of the minimum size is allocated."""
        import torch
        need = self.vjp_workspace_size()
        if workspace is None or workspace.numel() * workspace.element_size() < need:
            workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=X.device)
        if out is None:
            out = {"gX": torch.empty_like(X), "gU": torch.empty_like(U), "gs": torch.empty_like(s),
                   "L": torch.empty(self.n_inst, dtype=torch.float64, device=X.device) if want_L else None}
        io = _BatchVjpIO(*[None if t is None else t.data_ptr()
                           for t in (X, U, s, w, rho, out["gX"], out["gU"], out["gs"], out["L"])])
        _check(load().ciscvx_batch_discretize_vjp(self._h, ctypes.byref(io), _ptr(workspace),
                                                  workspace.numel() * workspace.element_size(),
                                                  _stream()))
        return out

    def _fused_args(self, X, U, s, w, rho, workspace, out, gout, want_L):
        import torch
        need = self.vjp_workspace_size()  # as discretize_vjp
        if workspace is None or workspace.numel() * workspace.element_size() < need:
            workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=X.device)
        if out is None:
            out = self.alloc_outputs(X.device)
        if gout is None:
            gout = {"gX": torch.empty_like(X), "gU": torch.empty_like(U), "gs": torch.empty_like(s),
                    "L": torch.empty(self.n_inst, dtype=torch.float64, device=X.device) if want_L else None}
        io = self._io(X, U, s, out)
        vio = _BatchVjpIO(*[None if t is None else t.data_ptr()
                            for t in (None, None, None, w, rho, gout["gX"], gout["gU"], gout["gs"], gout["L"])])
        return workspace, out, gout, io, vio

    def discretize_and_vjp(self, X, U, s, w, rho, workspace=None, out=None, gout=None, want_L=True):
        """ciscvx_batch_discretize_and_vjp: both outputs from one pass.  Returns (out, gout)."""
        workspace, out, gout, io, vio = self._fused_args(X, U, s, w, rho, workspace, out, gout, want_L)
        _check(load().ciscvx_batch_discretize_and_vjp(self._h, ctypes.byref(io), ctypes.byref(vio),
                                                      _ptr(workspace),
                                                      workspace.numel() * workspace.element_size(),
                                                      _stream()))
        return out, gout

    def autotune_fused(self, X, U, s, w, rho, workspace=None, out=None, gout=None):
        """ciscvx_batch_autotune_fused; returns the chosen launch shape."""
        workspace, out, gout, io, vio = self._fused_args(X, U, s, w, rho, workspace, out, gout, True)
        t = Tune()
        _check(load().ciscvx_batch_autotune_fused(self._h, ctypes.byref(io), ctypes.byref(vio),
                                                  _ptr(workspace),
                                                  workspace.numel() * workspace.element_size(),
                                                  _stream(), ctypes.byref(t)))
        return t.as_dict()

    def tune_fused(self):
        t = Tune()
        _check(load().ciscvx_batch_get_tune_fused(self._h, ctypes.byref(t)))
        return t.as_dict()

    def run_host(self, host_in, host_out, dev_in, dev_out, n_chunks=8, host_vjp=None, dev_vjp=None,
                 workspace=None):
        """ciscvx_batch_run_host: pipelined H2D -> linearize (-> VJP) -> D2H over chunks.

        host_in / dev_in: dicts X, U, s (host pinned / device tensors); host_out /
        dev_out: dicts A, Bm, Bp, S, defect, penalty; host_vjp / dev_vjp: dicts
        w, rho, gX, gU, gs, L (optional).  Asynchronous on the current stream."""
        p = lambda d, k: None if d is None or d.get(k) is None else d[k].data_ptr()  # noqa: E731
        hio = _BatchIO(*[p(host_in, "X"), p(host_in, "U"), p(host_in, "s")] +
                       [p(host_out, k) for k in ("A", "Bm", "Bp", "S", "defect", "penalty")])
        dio = _BatchIO(*[p(dev_in, "X"), p(dev_in, "U"), p(dev_in, "s")] +
                       [p(dev_out, k) for k in ("A", "Bm", "Bp", "S", "defect", "penalty")])
        hv = dv = None
        ws_ptr, ws_bytes = None, 0
        if host_vjp is not None:
            keys = ("X", "U", "s", "w", "rho", "gX", "gU", "gs", "L")
            hv = _BatchVjpIO(*[p(host_vjp, k) for k in keys])
            dv = _BatchVjpIO(*[p(dev_vjp, k) for k in keys])
            ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
        _check(load().ciscvx_batch_run_host(self._h, int(n_chunks), ctypes.byref(hio), ctypes.byref(dio),
                                            ctypes.byref(hv) if hv else None,
                                            ctypes.byref(dv) if dv else None, ws_ptr, ws_bytes,
                                            _stream()))

    def sync_status(self):
        _check(load().ciscvx_batch_sync_status(self._h, _stream()))

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ciscvx_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- packing helpers (host numpy) --
    def pack(self, arrays, key, total_key=None):
        """Packs per-instance numpy arrays into one flat array in instance order."""
        total = self.sizes[total_key or key]
        flat = np.empty(max(total, 1), dtype=np.float64)
        for i, a in enumerate(arrays):
            o = self.offsets[i][key]
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            flat[o:o + a.size] = a
        return flat

    def unpack(self, flat, key, i, shape):
        o = self.offsets[i][key]
        n = int(np.prod(shape))
        return np.asarray(flat[o:o + n]).reshape(shape)
