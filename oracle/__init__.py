"""CPU oracle for the MSD-AFQMC hot path: a ctypes binding of msd_oracle.c.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the library never does. It shares no code with the
CUDA path. See msd_oracle.c for the definitions it follows (the paper's naive
per-determinant approach, Sec. II B, with the Sec. II A single-determinant
overlap, Green's function and generalized-Wick energy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmsd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(path: str):
    """Load a compiled oracle and declare its entry points."""
    lib = ctypes.CDLL(path)
    dp = ctypes.c_void_p
    ci = ctypes.c_int
    lib.oracle_det.argtypes = [ci, ci, ci, dp, dp, dp, ctypes.c_double, ci, dp,
                               dp, dp, dp, dp, dp]
    lib.oracle_det.restype = ci
    lib.oracle_msd.argtypes = [ci, ci, ci, ci, dp, dp, dp, dp, ctypes.c_double, ci, dp,
                               ci, dp, dp, dp, dp, dp, dp, dp, dp, ci]
    lib.oracle_msd.restype = ci
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def det_terms(M, occ_a, occ_b, h1, e0, L, phi_a, phi_b, want_g=False):
    """O_I, E_I (and G_I, shape (2, M, M), if want_g) of one determinant pair
    against one walker. Raises ZeroDivisionError if O_I is exactly zero."""
    lib = _load()
    occ_a = _c(occ_a, np.int32); occ_b = _c(occ_b, np.int32)
    h1 = _c(h1, np.float64); L = _c(L, np.float64)
    phi_a = _c(phi_a, np.complex128); phi_b = _c(phi_b, np.complex128)
    o = np.zeros(1, np.complex128); e = np.zeros(1, np.complex128)
    g = np.zeros((2, M, M), np.complex128) if want_g else None
    rc = lib.oracle_det(M, occ_a.size, occ_b.size, _p(occ_a), _p(occ_b), _p(h1), float(e0),
                        L.shape[0], _p(L), _p(phi_a), _p(phi_b), _p(o), _p(e), _p(g))
    if rc < 0:
        raise MemoryError("oracle_det: allocation failed")
    if rc > 0:
        raise ZeroDivisionError("oracle_det: the determinant overlap is exactly zero")
    return (o[0], e[0], g) if want_g else (o[0], e[0])


def msd(system, phi_a, phi_b, *, energy=True, vbias=True, green=False,
        per_det=False, n_threads=0):
    """Trial-level quantities for every walker.

    Returns a dict with 'ovlp' (n_w,), and as requested 'e_loc' (n_w,),
    'vbias' (n_w, n_chol), 'G_T' (n_w, 2, M, M), 'det_ovlp' and 'det_e'
    (n_w, n_det)."""
    lib = _load()
    s = system
    M = s.M
    coeff = _c(s.coeff, np.float64)
    occ_a = _c(s.occ_a, np.int32); occ_b = _c(s.occ_b, np.int32)
    h1 = _c(s.h1, np.float64); L = _c(s.L, np.float64)
    phi_a = _c(phi_a, np.complex128); phi_b = _c(phi_b, np.complex128)
    n_w = phi_a.shape[0]
    n_det = coeff.shape[0]
    out = {"ovlp": np.zeros(n_w, np.complex128)}
    if energy:
        out["e_loc"] = np.zeros(n_w, np.complex128)
    if vbias:
        out["vbias"] = np.zeros((n_w, L.shape[0]), np.complex128)
    if green:
        out["G_T"] = np.zeros((n_w, 2, M, M), np.complex128)
    if per_det:
        out["det_ovlp"] = np.zeros((n_w, n_det), np.complex128)
        if energy:
            out["det_e"] = np.zeros((n_w, n_det), np.complex128)
    rc = lib.oracle_msd(M, s.n_alpha, s.n_beta, n_det, _p(coeff), _p(occ_a), _p(occ_b),
                        _p(h1), float(s.e0), L.shape[0], _p(L), n_w, _p(phi_a), _p(phi_b),
                        _p(out["ovlp"]), _p(out.get("e_loc")), _p(out.get("vbias")),
                        _p(out.get("G_T")), _p(out.get("det_ovlp")), _p(out.get("det_e")),
                        int(n_threads))
    if rc < 0:
        raise MemoryError("oracle_msd: allocation failed")
    if rc > 0:
        raise ZeroDivisionError(f"oracle_msd: walker {rc - 1} has an exactly zero "
                                "determinant overlap")
    return out
