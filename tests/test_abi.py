"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/fs.h declares, and rejects bad requests before making
any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2306_04322_gb300 import build as B
from paper_2306_04322_gb300 import fs as F
from paper_2306_04322_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return F.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:FS_API\s+)?(?:const\s+)?\w+\s*\*?\s*(fs_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "fs_plan_create" in names and "fs_step" in names and len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_only_the_c_abi_is_exported(L):
    """Hidden visibility: the library exports the declared entry points and no
    C++ symbol (template instantiations and their function-local statics stay
    private, so a second build of the library in the same process, such as
    the bounds-checked one, shares nothing with this one)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if l.split()[-2:-1] in (["T"], ["u"], ["V"], ["W"])]
    # weak instantiations of the C++ standard library's own templates keep the
    # visibility its headers give them; none of them holds state of this library
    ours = sorted(x for x in syms if not x.startswith(("_ZNSt", "_ZSt", "_ZNKSt")))
    assert ours == declared_functions(), ours


def test_version(L):
    assert "sm_103a" in F.fs_version()


def good_params(**kw):
    pr = I.Problem(n=(64, 64), p=1)
    pr.dt = 5 * I.fd_stable_dt(pr)
    P = F.make_params(pr, "f64")
    for k, v in kw.items():
        setattr(P, k, v)
    return P


@pytest.mark.parametrize("field,value,status", [
    ("ndim", 1, F.FS_ERR_INVALID_ARG),
    ("p", 5, F.FS_ERR_INVALID_ARG),
    ("p", -1, F.FS_ERR_INVALID_ARG),
    ("dt", 0.0, F.FS_ERR_INVALID_ARG),
    ("dt", float("nan"), F.FS_ERR_INVALID_ARG),
    ("M", -1.0, F.FS_ERR_INVALID_ARG),
    ("precision", 7, F.FS_ERR_INVALID_ARG),
    ("lap", 3, F.FS_ERR_INVALID_ARG),
    ("scheme", 2, F.FS_ERR_INVALID_ARG),
])
def test_invalid_params_rejected_without_cuda(L, field, value, status):
    P = good_params(**{field: value})
    h = ctypes.c_void_p(123)
    assert L.fs_plan_create(ctypes.byref(P), None, ctypes.byref(h)) == status
    assert h.value is None
    assert L.fs_last_error(None)


@pytest.mark.parametrize("n", [(48, 64), (64, 4), (4096, 64), (64, 12)])
def test_unsupported_sizes(L, n):
    P = good_params()
    P.n[0], P.n[1] = n
    h = ctypes.c_void_p()
    assert L.fs_plan_create(ctypes.byref(P), None, ctypes.byref(h)) == F.FS_ERR_UNSUPPORTED
    assert b"power of two" in L.fs_last_error(None)


def test_bad_dx_and_null_pointers(L):
    P = good_params()
    P.dx[1] = 0.0
    h = ctypes.c_void_p()
    assert L.fs_plan_create(ctypes.byref(P), None, ctypes.byref(h)) == F.FS_ERR_INVALID_ARG
    assert L.fs_plan_create(None, None, ctypes.byref(h)) == F.FS_ERR_INVALID_ARG
    P = good_params()
    assert L.fs_plan_create(ctypes.byref(P), None, None) == F.FS_ERR_INVALID_ARG
    assert L.fs_step(None, 1) == F.FS_ERR_INVALID_ARG
    assert L.fs_set_fields(None, None) == F.FS_ERR_INVALID_ARG
    assert L.fs_destroy(None) == F.FS_OK


def test_batch_must_share_precision_and_p(L):
    a, b = good_params(), good_params(p=2)
    arr = (F.fs_params * 2)(a, b)
    h = ctypes.c_void_p()
    assert L.fs_batch_create(arr, 2, None, ctypes.byref(h)) == F.FS_ERR_INVALID_ARG
    assert L.fs_batch_create(arr, 0, None, ctypes.byref(h)) == F.FS_ERR_INVALID_ARG


def test_allocation_failure_reported_as_oom(L):
    """An allocator hook that fails: the plan reports FS_ERR_OOM, frees what it
    took, and touches no CUDA call before the workspace exists."""
    calls = {"alloc": 0, "free": 0}

    @F.ALLOC_FN
    def bad_alloc(nbytes, ctx):
        calls["alloc"] += 1
        return None

    @F.FREE_FN
    def bad_free(ptr, ctx):
        calls["free"] += 1

    P = good_params()
    h = ctypes.c_void_p()
    st = L.fs_plan_create_ex(ctypes.byref(P), None, bad_alloc, bad_free, None, ctypes.byref(h))
    assert st == F.FS_ERR_OOM
    assert calls["alloc"] >= 1 and h.value is None
    assert b"allocation" in L.fs_last_error(None)


def test_3d_axis_limits(L):
    """2D plans take axes up to 2048; 3D plans stop at 1024 along x and 512
    along y and z."""
    P = good_params()
    P.ndim = 3
    P.n[0], P.n[1], P.n[2] = 2048, 64, 64
    P.dx[2] = 1.0
    h = ctypes.c_void_p()
    assert L.fs_plan_create(ctypes.byref(P), None, ctypes.byref(h)) == F.FS_ERR_UNSUPPORTED
    assert b"3D grids" in L.fs_last_error(None)
    P.n[0], P.n[1] = 64, 1024
    assert L.fs_plan_create(ctypes.byref(P), None, ctypes.byref(h)) == F.FS_ERR_UNSUPPORTED


@pytest.mark.parametrize("kw,rank,nranks,status", [
    ({}, 0, 3, F.FS_ERR_UNSUPPORTED),            # not a power of two
    ({}, 2, 2, F.FS_ERR_INVALID_ARG),            # rank out of range
    ({}, -1, 2, F.FS_ERR_INVALID_ARG),
    ({}, 0, 16, F.FS_ERR_UNSUPPORTED),           # 64 / 16 < 8 rows per rank
    ({"precision": F.FS_F32_TC_TF32}, 0, 2, F.FS_ERR_UNSUPPORTED),
    ({"scheme": F.FS_SCHEME_EXPLICIT_FD}, 0, 2, F.FS_ERR_UNSUPPORTED),
    ({"ndim": 3}, 0, 2, F.FS_ERR_UNSUPPORTED),
    ({"dt": -1.0}, 0, 2, F.FS_ERR_INVALID_ARG),  # refused by the row plan's validation
])
def test_slab_requests_rejected_without_cuda(L, kw, rank, nranks, status):
    """fs_slab_create validates before any CUDA call (include/fs_slab.h)."""
    P = good_params(**kw)
    if kw.get("ndim") == 3:
        P.n[2], P.dx[2] = 64, 1.0
    h = ctypes.c_void_p(123)
    assert L.fs_slab_create(ctypes.byref(P), rank, nranks, None, ctypes.byref(h)) == status
    assert h.value is None
    assert L.fs_slab_last_error(None)


def test_slab_null_handles(L):
    h = ctypes.c_void_p()
    assert L.fs_slab_create(None, 0, 1, None, ctypes.byref(h)) == F.FS_ERR_INVALID_ARG
    P = good_params()
    assert L.fs_slab_create(ctypes.byref(P), 0, 1, None, None) == F.FS_ERR_INVALID_ARG
    for fn in ("fs_slab_row_pass", "fs_slab_col_pass", "fs_slab_sync"):
        assert getattr(L, fn)(None) == F.FS_ERR_INVALID_ARG
    assert L.fs_slab_info_get(None, None) == F.FS_ERR_INVALID_ARG
    assert L.fs_slab_destroy(None) == F.FS_OK
