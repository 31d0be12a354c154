"""Python binding of the C ABI in include/fs.h and include/fs_slab.h (ctypes;
argument marshalling only).

The module-level functions carry the C names (fs_plan_create, fs_set_fields,
fs_step, fs_get_fields, fs_destroy, ...) and take torch tensors or raw
pointers; every step of the computation runs in libfs_gb300.so.  `Plan` is a
small convenience wrapper over the same calls.  There is no fallback: if the
library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FS_OK, FS_ERR_INVALID_ARG, FS_ERR_UNSUPPORTED, FS_ERR_OOM, FS_ERR_CUDA, FS_ERR_NONFINITE, \
    FS_ERR_TIMEOUT, FS_ERR_STATE = range(8)
FS_F64, FS_F32, FS_F32_TC_TF32, FS_F32_TC_BF16X3 = range(4)
FS_LAP_SPECTRAL, FS_LAP_FD2, FS_LAP_FD4 = range(3)
FS_SCHEME_SEMI_IMPLICIT_FS, FS_SCHEME_EXPLICIT_FD = range(2)

PRECISIONS = {"f64": FS_F64, "f32": FS_F32, "tf32": FS_F32_TC_TF32, "bf16x3": FS_F32_TC_BF16X3}
STATUS_NAMES = {0: "FS_OK", 1: "FS_ERR_INVALID_ARG", 2: "FS_ERR_UNSUPPORTED", 3: "FS_ERR_OOM",
                4: "FS_ERR_CUDA", 5: "FS_ERR_NONFINITE", 6: "FS_ERR_TIMEOUT", 7: "FS_ERR_STATE"}


class FSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fs_params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("p", ctypes.c_int), ("M", ctypes.c_double), ("L", ctypes.c_double),
                ("kappa_c", ctypes.c_double), ("kappa_eta", ctypes.c_double),
                ("rho2", ctypes.c_double), ("c_alpha", ctypes.c_double), ("c_beta", ctypes.c_double),
                ("w", ctypes.c_double), ("alpha", ctypes.c_double), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("lap", ctypes.c_int), ("scheme", ctypes.c_int)]


class fs_slab_info(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("nranks", ctypes.c_int), ("rows", ctypes.c_int), ("cols", ctypes.c_int),
                ("slots_fwd", ctypes.c_int), ("slots_back", ctypes.c_int), ("elem_bytes", ctypes.c_size_t),
                ("block_elems", ctypes.c_size_t), ("send", ctypes.c_void_p), ("recv", ctypes.c_void_p),
                ("colspec", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_vpp = ctypes.POINTER(ctypes.c_void_p)


def library_path() -> str:
    return _build.LIB


def bind(path: str):
    """Load a build of the library at `path` and declare the C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(fs_params)
    plan = ctypes.c_void_p
    sig = {
        "fs_plan_create": [P, ctypes.c_void_p, ctypes.POINTER(plan)],
        "fs_plan_create_ex": [P, ctypes.c_void_p, ALLOC_FN, FREE_FN, ctypes.c_void_p, ctypes.POINTER(plan)],
        "fs_batch_create": [P, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(plan)],
        "fs_set_fields": [plan, _vpp],
        "fs_step": [plan, ctypes.c_int64],
        "fs_step_async": [plan, ctypes.c_int64],
        "fs_sync": [plan],
        "fs_get_fields": [plan, _vpp],
        "fs_set_params": [plan, P],
        "fs_set_stream": [plan, ctypes.c_void_p],
        "fs_free_energy": [plan, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "fs_step_adjoint": [plan, _vpp, _vpp, _vpp, ctypes.POINTER(ctypes.c_double)],
        "fs_step_profiled": [plan, ctypes.c_int64],
        "fs_profile_read": [plan, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                            ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "fs_batch_schedule": [plan] + [ctypes.POINTER(ctypes.c_int64)] * 4 + [ctypes.POINTER(ctypes.c_int)] * 2,
        "fs_workspace_bytes": [plan, ctypes.POINTER(ctypes.c_size_t)],
        "fs_last_launch_count": [plan, ctypes.POINTER(ctypes.c_int64)],
        "fs_destroy": [plan],
        "fs_step2d_static": [P, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p],
        "fs_test_short_wait": [plan, ctypes.c_int],
        "fs_set_pass_forms": [plan, ctypes.c_int, ctypes.c_int],
        "fs_measure_fp64_rate": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)],
        "fs_slab_create": [P, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
        "fs_slab_info_get": [ctypes.c_void_p, ctypes.POINTER(fs_slab_info)],
        "fs_slab_set_fields": [ctypes.c_void_p, _vpp, ctypes.POINTER(ctypes.c_double)],
        "fs_slab_set_c_sum": [ctypes.c_void_p, ctypes.c_double],
        "fs_slab_row_pass": [ctypes.c_void_p],
        "fs_slab_col_pass": [ctypes.c_void_p],
        "fs_slab_get_fields": [ctypes.c_void_p, _vpp],
        "fs_slab_sync": [ctypes.c_void_p],
        "fs_slab_destroy": [ctypes.c_void_p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.fs_last_error.argtypes = [plan]
    L.fs_last_error.restype = ctypes.c_char_p
    L.fs_slab_last_error.argtypes = [ctypes.c_void_p]
    L.fs_slab_last_error.restype = ctypes.c_char_p
    L.fs_version.argtypes = []
    L.fs_version.restype = ctypes.c_char_p
    return L


def lib(build_if_missing: bool = False):
    """Load libfs_gb300.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = library_path()
    if not os.path.exists(path):
        raise FileNotFoundError(f"libfs_gb300.so is not built ({path}); run __graft_entry__.build()")
    _lib = bind(path)
    return _lib


def _check(status: int, plan=None):
    if status != FS_OK:
        msg = lib().fs_last_error(plan)
        raise FSError(status, msg.decode() if msg else "")


def make_params(prob, precision="f64", scheme: int = FS_SCHEME_SEMI_IMPLICIT_FS) -> fs_params:
    """fs_params from an inputs.Problem (or any object with the same fields)."""
    P = fs_params()
    P.ndim = len(prob.n)
    for d in range(3):
        P.n[d] = prob.n[d] if d < P.ndim else 1
        P.dx[d] = prob.dx[d] if d < P.ndim else 1.0
    P.p = prob.p
    for k in ("M", "L", "kappa_c", "kappa_eta", "rho2", "c_alpha", "c_beta", "w", "alpha", "dt"):
        setattr(P, k, float(getattr(prob, k)))
    P.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    P.lap = int(getattr(prob, "lap", 0))
    P.scheme = int(scheme)
    return P


def _ptr(x) -> int:
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("field tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("field arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])
    return ctypes.cast(arr, _vpp), arr


def _current_stream():
    import torch
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


# ---- C names -----------------------------------------------------------------

def fs_plan_create(params: fs_params, stream=None):
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(lib().fs_plan_create(ctypes.byref(params), s, ctypes.byref(h)))
    return h


def fs_batch_create(params_list, stream=None):
    arr = (fs_params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(lib().fs_batch_create(arr, len(params_list), s, ctypes.byref(h)))
    return h


def fs_set_fields(plan, fields):
    pp, keep = _ptr_array(fields)
    _check(lib().fs_set_fields(plan, pp), plan)


def fs_step(plan, nsteps: int):
    _check(lib().fs_step(plan, int(nsteps)), plan)


def fs_step_async(plan, nsteps: int):
    _check(lib().fs_step_async(plan, int(nsteps)), plan)


def fs_sync(plan):
    _check(lib().fs_sync(plan), plan)


def fs_get_fields(plan, out):
    pp, keep = _ptr_array(out)
    _check(lib().fs_get_fields(plan, pp), plan)


def fs_set_params(plan, params: fs_params):
    _check(lib().fs_set_params(plan, ctypes.byref(params)), plan)


def fs_set_stream(plan, stream):
    _check(lib().fs_set_stream(plan, ctypes.c_void_p(stream)), plan)


def fs_free_energy(plan, nparts: int):
    F = ctypes.c_double()
    parts = (ctypes.c_double * nparts)()
    _check(lib().fs_free_energy(plan, ctypes.byref(F), parts), plan)
    return F.value, list(parts)


def fs_step_adjoint(plan, u, lam_in, lam_out, with_grad: bool = True):
    pu, k1 = _ptr_array(u)
    pi, k2 = _ptr_array(lam_in)
    po, k3 = _ptr_array(lam_out)
    g = (ctypes.c_double * 4)(0.0, 0.0, 0.0, 0.0)
    _check(lib().fs_step_adjoint(plan, pu, pi, po, g if with_grad else None), plan)
    return list(g)


def fs_step_profiled(plan, nsteps: int):
    _check(lib().fs_step_profiled(plan, int(nsteps)), plan)


def fs_profile_read(plan, npass_max: int = 8):
    """Per-pass-kind (milliseconds, launches) since the last read."""
    ms = (ctypes.c_double * npass_max)()
    cnt = (ctypes.c_int64 * npass_max)()
    n = ctypes.c_int()
    _check(lib().fs_profile_read(plan, ms, cnt, npass_max, ctypes.byref(n)), plan)
    return list(ms[:n.value]), list(cnt[:n.value])


def fs_batch_schedule(plan):
    """(row grid, column grid, row items, column items, row form, column form)
    of a batched plan, as chosen by the autotuner."""
    v = [ctypes.c_int64() for _ in range(4)]
    f = [ctypes.c_int() for _ in range(2)]
    _check(lib().fs_batch_schedule(plan, *[ctypes.byref(x) for x in v + f]), plan)
    return tuple(x.value for x in v + f)


def fs_set_pass_forms(plan, row_form: int, col_form: int):
    """Kernel forms of the passes: 0 default, 1 half-length / tile, 2 warp per line."""
    _check(lib().fs_set_pass_forms(plan, int(row_form), int(col_form)), plan)


def fs_test_short_wait(plan, enable):
    """Test hook: 1 (or True) cuts the first bounded device wait of every pass
    short, 2 the grid barriers of the fused step, 0 (False) restores both."""
    _check(lib().fs_test_short_wait(plan, int(enable)), plan)


def fs_measure_fp64_rate(stream=None):
    """(DFMA, DADD) thread-instructions per second of the current device."""
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().fs_measure_fp64_rate(s, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fs_workspace_bytes(plan) -> int:
    b = ctypes.c_size_t()
    _check(lib().fs_workspace_bytes(plan, ctypes.byref(b)), plan)
    return b.value


def fs_last_launch_count(plan) -> int:
    b = ctypes.c_int64()
    _check(lib().fs_last_launch_count(plan, ctypes.byref(b)), plan)
    return b.value


def fs_destroy(plan):
    _check(lib().fs_destroy(plan))


def fs_step2d_static(params: fs_params, fields, nsteps: int, stream=None) -> int:
    """Allocation-free 2D step on one contiguous device array of all fields;
    returns the status code (no exception, the call sets no error text)."""
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    return lib().fs_step2d_static(ctypes.byref(params), ctypes.c_void_p(_ptr(fields)), int(nsteps), s)


# ---- slab decomposition (include/fs_slab.h) -----------------------------------

def _check_slab(status: int, slab=None):
    if status != FS_OK:
        msg = lib().fs_slab_last_error(slab)
        raise FSError(status, msg.decode() if msg else "")


def fs_slab_create(params: fs_params, rank: int, nranks: int, stream=None):
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check_slab(lib().fs_slab_create(ctypes.byref(params), int(rank), int(nranks), s, ctypes.byref(h)))
    return h


def fs_slab_info_get(slab) -> fs_slab_info:
    info = fs_slab_info()
    _check_slab(lib().fs_slab_info_get(slab, ctypes.byref(info)), slab)
    return info


def fs_slab_set_fields(slab, fields) -> float:
    """Returns the FP64 sum of this rank's c values."""
    arr, keep = _ptr_array(fields)
    total = ctypes.c_double()
    _check_slab(lib().fs_slab_set_fields(slab, arr, ctypes.byref(total)), slab)
    return total.value


def fs_slab_set_c_sum(slab, c_sum_total: float):
    _check_slab(lib().fs_slab_set_c_sum(slab, float(c_sum_total)), slab)


def fs_slab_row_pass(slab):
    _check_slab(lib().fs_slab_row_pass(slab), slab)


def fs_slab_col_pass(slab):
    _check_slab(lib().fs_slab_col_pass(slab), slab)


def fs_slab_get_fields(slab, out):
    arr, keep = _ptr_array(out)
    _check_slab(lib().fs_slab_get_fields(slab, arr), slab)


def fs_slab_sync(slab):
    _check_slab(lib().fs_slab_sync(slab), slab)


def fs_slab_destroy(slab):
    _check_slab(lib().fs_slab_destroy(slab))


def fs_version() -> str:
    return lib().fs_version().decode()


# ---- convenience wrapper ------------------------------------------------------

class Plan:
    """One simulation (or a batch) on the current CUDA device and stream."""

    def __init__(self, prob, precision="f64", scheme: int = FS_SCHEME_SEMI_IMPLICIT_FS, stream=None):
        import torch
        self.batch = isinstance(prob, (list, tuple))
        probs = list(prob) if self.batch else [prob]
        self.probs = probs
        self.precision = precision
        self.nf = probs[0].nf
        self.dtype = torch.float64 if precision in ("f64", FS_F64) else torch.float32
        params = [make_params(p, precision, scheme) for p in probs]
        self.h = fs_batch_create(params, stream) if self.batch else fs_plan_create(params[0], stream)

    def set_fields(self, fields):
        """fields: per member, a tensor of shape (nf, *shape) (or list of nf tensors)."""
        flat = self._flatten(fields)
        fs_set_fields(self.h, flat)

    def _flatten(self, fields):
        members = fields if self.batch else [fields]
        flat = []
        for m in members:
            for f in range(self.nf):
                t = m[f]
                if t.dtype != self.dtype:
                    raise TypeError(f"field dtype {t.dtype} does not match plan dtype {self.dtype}")
                flat.append(t)
        return flat

    def step(self, n: int = 1):
        fs_step(self.h, n)

    def step_async(self, n: int = 1):
        fs_step_async(self.h, n)

    def sync(self):
        fs_sync(self.h)

    def get_fields(self, out=None, device="cuda"):
        import torch
        if out is None:
            out = [torch.empty((self.nf,) + p.shape, dtype=self.dtype, device=device) for p in self.probs]
            if not self.batch:
                out = out[0]
        fs_get_fields(self.h, self._flatten(out))
        return out

    def free_energy(self):
        return fs_free_energy(self.h, 2 + self.probs[0].p)

    def step_adjoint(self, u, lam_in, lam_out):
        return fs_step_adjoint(self.h, [u[f] for f in range(self.nf)], [lam_in[f] for f in range(self.nf)],
                               [lam_out[f] for f in range(self.nf)])

    def set_params(self, prob):
        fs_set_params(self.h, make_params(prob, self.precision))
        self.probs = [prob]

    @property
    def workspace_bytes(self) -> int:
        return fs_workspace_bytes(self.h)

    @property
    def last_launch_count(self) -> int:
        return fs_last_launch_count(self.h)

    def close(self):
        if self.h is not None and self.h.value:
            fs_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
