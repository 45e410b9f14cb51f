"""ctypes wrapper of the compiled oracle (oracle/c/oracle.c).  Test infrastructure.

build() compiles it with gcc (-O2 -fopenmp, no machine-specific flags, so the
same source builds on x86_64 and aarch64).  The functions mirror
oracle/dirac.py and oracle/msolve.py and are pinned against them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "oracle.c")
_LIB = os.path.join(_HERE, "c", "liboracle.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", _LIB, _SRC])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.orc_dslash.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int, ctypes.c_int]
        L.orc_h2.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int]
        L.orc_multishift.argtypes = [P, P, ctypes.c_double, P, P, ctypes.c_int, ctypes.c_int, P,
                                     ctypes.c_double, ctypes.c_int, P, P]
        L.orc_multishift.restype = ctypes.c_int
        L.orc_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _i4(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def threads():
    return lib().orc_threads()


def apply_dw(U, psi, dims, kappa, bc=(1, 1, 1, 1), g5out=False):
    V = int(np.prod(dims))
    p = _c(psi)
    B = 1 if p.ndim == 3 else p.shape[-1]
    out = np.empty_like(p)
    Uc = _c(U)
    d, b = _i4(dims), _i4(bc)
    lib().orc_dslash(d.ctypes.data, b.ctypes.data, kappa, Uc.ctypes.data, p.ctypes.data, out.ctypes.data, B,
                     int(g5out))
    assert out.shape[0] == V
    return out


def apply_h2(U, psi, dims, kappa, bc=(1, 1, 1, 1)):
    p = _c(psi)
    B = 1 if p.ndim == 3 else p.shape[-1]
    out = np.empty_like(p)
    Uc = _c(U)
    d, b = _i4(dims), _i4(bc)
    lib().orc_h2(d.ctypes.data, b.ctypes.data, kappa, Uc.ctypes.data, p.ctypes.data, out.ctypes.data, B)
    return out


def multishift_cg(U, dims, kappa, b, shifts, tol, bc=(1, 1, 1, 1), max_iter=100000):
    """b: [V,4,3,B].  Returns (x[n,V,4,3,B], iterations, resid[n,B])."""
    bb = _c(b)
    B = bb.shape[-1]
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    n = sh.size
    x = np.empty((n,) + bb.shape, dtype=np.complex128)
    res = np.empty((n, B))
    Uc = _c(U)
    d, bcv = _i4(dims), _i4(bc)
    k = lib().orc_multishift(d.ctypes.data, bcv.ctypes.data, kappa, Uc.ctypes.data, bb.ctypes.data, B, n,
                             sh.ctypes.data, tol, max_iter, x.ctypes.data, res.ctypes.data)
    if k < 0:
        raise RuntimeError("oracle multishift CG did not converge")
    return x, k, res
