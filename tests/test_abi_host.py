"""Host-side checks of the C ABI library (no GPU): it builds, loads, exports every
symbol include/ciscvx.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_09993_gb300 import api, build
    build.build()
    return api.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "ciscvx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ciscvx_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2604_09993_gb300 import api
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(api.EXPORTS)


def test_version(lib):
    assert lib.ciscvx_version() == 9


def test_null_arguments_rejected(lib):
    from paper_2604_09993_gb300 import api
    h = ctypes.c_void_p()
    assert lib.ciscvx_model_create(None, ctypes.byref(h)) == api.EINVAL
    assert b"null" in lib.ciscvx_last_error()
    st = lib.ciscvx_discretize(None, 10, 4, 0, 0, None, None, None, None, None, None, None, None,
                               None, None, None, 0, None)
    assert st == api.EINVAL
    st = lib.ciscvx_discretize_vjp(None, 10, 4, 0, 0, None, None, None, None, None, None, None,
                                   None, None, None, 0, None)
    assert st == api.EINVAL
    assert lib.ciscvx_sync_status(None, None) == api.EINVAL
    n = ctypes.c_size_t()
    assert lib.ciscvx_workspace_size(None, 1, 10, 0, ctypes.byref(n)) == api.EINVAL
    assert lib.ciscvx_model_dims(None, None, None, None) == api.EINVAL
    prm = api._NodeParams(1e-3, None)
    assert lib.ciscvx_node_linearize(None, 4, None, None, None, None, ctypes.byref(prm), None,
                                     None, None, None, None, None, None, None) == api.EINVAL
    assert lib.ciscvx_discretize_compact(None, 10, 4, 0, 0, None, None, None, None, None, None,
                                         None, None, None, None, None, 0, None) == api.EINVAL
    lo, hi = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.ciscvx_discretize_workspace_size(None, 0, 10, 4, 0, 0, ctypes.byref(lo),
                                                ctypes.byref(hi)) == api.EINVAL
    assert lib.ciscvx_psi_rows(None, None) == api.EINVAL
    assert lib.ciscvx_psi_linearize(None, 4, None, None, 0.1, 1e-4, None, None, None) == api.EINVAL
    h = ctypes.c_void_p()
    assert lib.ciscvx_socp_create(None, 4, 0, None, ctypes.byref(h)) == api.EINVAL
    assert lib.ciscvx_socp_get_dims(None, None) == api.EINVAL
    assert lib.ciscvx_socp_structure(None, None, None, None, None, None, None, None) == api.EINVAL
    assert lib.ciscvx_socp_fill(None, 1, None, None, None) == api.EINVAL
    lib.ciscvx_socp_destroy(None)


def _desc(api, nb=2, joints=((0, 1),), contacts=((1,),), mass=1.0):
    bodies = (api._Body * nb)(*[api._Body(mass, 0.1) for _ in range(nb)])
    js = (api._Joint * max(len(joints), 1))(*[
        api._Joint(p, c, (ctypes.c_double * 2)(0.0, -0.1), (ctypes.c_double * 2)(0.0, 0.1))
        for p, c in joints])
    cs = (api._Contact * max(len(contacts), 1))(*[
        api._Contact(b[0], (ctypes.c_double * 2)(0.0, -0.1), 1.0) for b in contacts])
    d = api._Desc(nb, len(joints), len(contacts), bodies, js, cs, 9.81)
    return d, (bodies, js, cs)


@pytest.mark.parametrize("case", ["bad_parent", "self_joint", "bad_contact", "neg_mass",
                                  "two_contacts", "too_many_links", "zero_links",
                                  "bad_joint_force_model", "bad_scheme", "nan_terrain",
                                  "eliminated_closed_loop"])
def test_invalid_models_rejected_before_cuda(lib, case):
    from paper_2604_09993_gb300 import api
    kw = {}
    want = api.EINVAL
    if case == "bad_parent":
        kw = dict(joints=((5, 1),))
    elif case == "self_joint":
        kw = dict(joints=((1, 1),))
    elif case == "bad_contact":
        kw = dict(contacts=((7,),))
    elif case == "neg_mass":
        kw = dict(mass=-1.0)
    elif case == "two_contacts":
        kw = dict(contacts=((1,), (1,)))
        want = api.EUNSUPPORTED
    elif case == "too_many_links":
        kw = dict(nb=33, joints=(), contacts=())
        want = api.EUNSUPPORTED
    elif case == "zero_links":
        kw = dict(nb=0, joints=(), contacts=())
    elif case == "eliminated_closed_loop":  # link 2 hangs from two joints: not a forest
        kw = dict(nb=3, joints=((0, 2), (1, 2)), contacts=((2,),))
        want = api.EUNSUPPORTED
    d, keep = _desc(api, **kw)
    if case == "bad_joint_force_model":
        d.joint_forces = 2
    elif case == "bad_scheme":
        d.scheme = 7
    elif case == "nan_terrain":
        d.terrain_amp = float("nan")
    elif case == "eliminated_closed_loop":
        d.joint_forces = 1
    h = ctypes.c_void_p()
    assert lib.ciscvx_model_create(ctypes.byref(d), ctypes.byref(h)) == want
    assert h.value is None
    assert lib.ciscvx_last_error() != b""
