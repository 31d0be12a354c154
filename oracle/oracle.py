"""ctypes front end of the FP64 CPU oracle (fs_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg load this module; the product path never does.  It marshals
numpy arrays into the C functions and nothing else: every number it returns is
computed in fs_oracle.cpp, which follows the paper's equations and Algorithm 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fs_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfs_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no FMA contraction, OpenMP over lines)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrParams(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("p", ctypes.c_int), ("M", ctypes.c_double), ("L", ctypes.c_double),
                ("kappa_c", ctypes.c_double), ("kappa_eta", ctypes.c_double),
                ("rho2", ctypes.c_double), ("c_alpha", ctypes.c_double),
                ("c_beta", ctypes.c_double), ("w", ctypes.c_double), ("alpha", ctypes.c_double),
                ("dt", ctypes.c_double), ("lap", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OrParams)
        sig = {
            "or_fchem_point": (ctypes.c_double, [pp, ctypes.c_double, dp]),
            "or_dfchem_point": (None, [pp, ctypes.c_double, dp, dp]),
            "or_d2fchem_point": (None, [pp, ctypes.c_double, dp, dp]),
            "or_fft": (None, [dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
            "or_k2": (None, [pp, dp]),
            "or_derivatives": (None, [pp, dp, dp]),
            "or_step": (ctypes.c_double, [pp, dp, ctypes.c_int]),
            "or_free_energy": (ctypes.c_double, [pp, dp, dp]),
            "or_fd_step": (None, [pp, dp, ctypes.c_int]),
            "or_adjoint_step": (None, [pp, dp, dp, dp, dp]),
            "or_num_threads": (ctypes.c_int, []),
            "or_set_num_threads": (None, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def params(prob) -> OrParams:
    """Oracle parameter struct from an inputs.Problem."""
    P = OrParams()
    P.ndim = prob.ndim
    for d in range(3):
        P.n[d] = prob.n[d] if d < prob.ndim else 1
        P.dx[d] = prob.dx[d] if d < prob.ndim else 1.0
    P.p = prob.p
    for k in ("M", "L", "kappa_c", "kappa_eta", "rho2", "c_alpha", "c_beta", "w", "alpha", "dt"):
        setattr(P, k, float(getattr(prob, k)))
    P.lap = int(prob.lap)
    return P


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def fft(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT of a complex array along every axis (numpy axis order)."""
    z = np.ascontiguousarray(a, dtype=np.complex128).copy()
    dims = list(reversed(z.shape))  # x fastest
    n = (ctypes.c_int * 3)(*(dims + [1] * (3 - len(dims))))
    lib().or_fft(z.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 len(dims), n, sign)
    return z


def k2(prob) -> np.ndarray:
    out = np.empty(prob.shape)
    P = params(prob)
    lib().or_k2(ctypes.byref(P), _dp(out))
    return out


def derivatives(prob, fields) -> np.ndarray:
    f = _f64(fields)
    out = np.empty_like(f)
    P = params(prob)
    lib().or_derivatives(ctypes.byref(P), _dp(f), _dp(out))
    return out


def step(prob, fields, nsteps: int = 1):
    """Algorithm 1, nsteps steps; returns (new fields, worst imag/real ratio)."""
    f = _f64(fields).copy()
    P = params(prob)
    worst = lib().or_step(ctypes.byref(P), _dp(f), int(nsteps))
    return f, worst


def free_energy(prob, fields, parts: bool = False):
    f = _f64(fields)
    P = params(prob)
    pt = np.zeros(2 + prob.p)
    F = lib().or_free_energy(ctypes.byref(P), _dp(f), _dp(pt))
    return (F, pt) if parts else F


def fd_step(prob, fields, nsteps: int = 1) -> np.ndarray:
    f = _f64(fields).copy()
    P = params(prob)
    lib().or_fd_step(ctypes.byref(P), _dp(f), int(nsteps))
    return f


def adjoint_step(prob, u, lam):
    """lam_out = J(u)^T lam and the step's parameter sensitivities
    (d/dM, d/dL, d/dkappa_c, d/dkappa_eta) of <lam, step(u)>."""
    uu, ll = _f64(u), _f64(lam)
    out = np.empty_like(uu)
    g = np.zeros(4)
    P = params(prob)
    lib().or_adjoint_step(ctypes.byref(P), _dp(uu), _dp(ll), _dp(out), _dp(g))
    return out, g


def fchem_point(prob, c: float, eta) -> float:
    e = _f64(np.atleast_1d(eta))
    P = params(prob)
    return lib().or_fchem_point(ctypes.byref(P), float(c), _dp(e))


def dfchem_point(prob, c: float, eta) -> np.ndarray:
    e = _f64(np.atleast_1d(eta))
    out = np.empty(1 + prob.p)
    P = params(prob)
    lib().or_dfchem_point(ctypes.byref(P), float(c), _dp(e), _dp(out))
    return out


def d2fchem_point(prob, c: float, eta) -> np.ndarray:
    e = _f64(np.atleast_1d(eta))
    out = np.empty((1 + prob.p) * (1 + prob.p))
    P = params(prob)
    lib().or_d2fchem_point(ctypes.byref(P), float(c), _dp(e), _dp(out))
    return out.reshape(1 + prob.p, 1 + prob.p)


def set_threads(n: int) -> int:
    lib().or_set_num_threads(int(n))
    return lib().or_num_threads()
