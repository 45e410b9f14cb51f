"""Compiled helper of the input generators (synth/c/stout.c), built with gcc."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "stout.c")
LIB = os.path.join(HERE, "c", "libsynth.so")
_lib = None


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        _lib.synth_stout.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int]
        _lib.synth_stout.restype = None
    return _lib


def stout(U, dims, rho, steps):
    """The stout steps of gauge.stout_smooth, in C (OpenMP); returns a new array."""
    out = np.ascontiguousarray(U, dtype=np.complex128).copy()
    d = (ctypes.c_int * 4)(*dims)
    lib().synth_stout(out.ctypes.data, d, float(rho), int(steps))
    return out
