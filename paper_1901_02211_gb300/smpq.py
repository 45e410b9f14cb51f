"""Python binding of libsmpq (include/smpq.h): argument marshalling only.

Every function keeps the C name and forwards to the CUDA library; all compute
runs in the library's kernels.  Arrays may be numpy (host, on_device=0) or
torch CUDA tensors (device, on_device=1); complex128 arrays are passed as the
interleaved doubles the ABI expects.  If the compiled library is missing, the
import fails: there is no other implementation behind these names.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

SMPQ_OK = 0
SMPQ_EINVAL = -1
SMPQ_ENOMEM = -2
SMPQ_ECUDA = -3
SMPQ_ENOCONV = -4
SMPQ_EBREAKDOWN = -5
SMPQ_ETIMEOUT = -6
SMPQ_ENOTSU3 = -7
SMPQ_ESTATE = -8
SMPQ_FP64 = 0
SMPQ_FP32 = 1
SMPQ_MIXED = 2
SMPQ_FP16N = 3
SMPQ_BF16N = 4

_NAMES = {v: k for k, v in globals().items() if k.startswith("SMPQ_E") or k == "SMPQ_OK"}


class SmpqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "?"), code, msg))
        self.code = code


class smpq_options(ctypes.Structure):
    _fields_ = [
        ("kappa", ctypes.c_double),
        ("npoles", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("reliable_delta", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("rhs_block", ctypes.c_int),
        ("iters_per_check", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("switch_residual", ctypes.c_double),
        ("autotune", ctypes.c_int),
        ("full_support", ctypes.c_int),
        ("true_residual", ctypes.c_int),
        ("tune_cache", ctypes.c_char_p),
        ("staging", ctypes.c_int),
    ]


class smpq_stats(ctypes.Structure):
    _fields_ = [
        ("n_rhs", ctypes.c_int),
        ("n_classes", ctypes.c_int),
        ("n_batches", ctypes.c_int),
        ("max_iterations", ctypes.c_int),
        ("total_iterations", ctypes.c_longlong),
        ("reliable_updates", ctypes.c_int),
        ("max_resid", ctypes.c_double),
        ("max_im_q", ctypes.c_double),
        ("Q", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("total_ms", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
        ("dslash_ms", ctypes.c_double),
        ("dslash_launches", ctypes.c_longlong),
        ("update_ms", ctypes.c_double),
        ("update_launches", ctypes.c_longlong),
        ("dslash_hi_ms", ctypes.c_double),
        ("dslash_hi_launches", ctypes.c_longlong),
        ("update_hi_ms", ctypes.c_double),
        ("update_hi_launches", ctypes.c_longlong),
        ("rhs_tile", ctypes.c_int),
        ("q_round_dev", ctypes.c_double),
        ("true_resid", ctypes.c_double),
        ("tiles_per_block_hi", ctypes.c_int),
        ("tiles_per_block_lo", ctypes.c_int),
        ("cols_per_thread", ctypes.c_int),
        ("shape_from_cache", ctypes.c_int),
        ("staged", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = [
    "smpq_options_default", "smpq_create", "smpq_destroy", "smpq_last_error", "smpq_set_options",
    "smpq_load_gauge", "smpq_set_spectrum", "smpq_measure_spectrum", "smpq_zolotarev", "smpq_get_zolotarev",
    "smpq_build_sources", "smpq_colour_sites", "smpq_dslash", "smpq_apply_dov", "smpq_compute_qx",
    "smpq_compute_qx_classes", "smpq_dslash_noalloc", "smpq_trace_dwinv", "smpq_compute_qx_batch",
    "smpq_low_modes", "smpq_get_low_modes", "smpq_clear_low_modes", "smpq_time_dslash", "smpq_context_info",
    "smpq_alu_peak", "smpq_tune_cache_lookup", "smpq_tune_cache_store",
]

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libsmpq.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libsmpq.so not built; run paper_1901_02211_gb300._build.build()")
    L = ctypes.CDLL(_build.LIB)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    PI, PD = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "smpq_options_default": [ctypes.POINTER(smpq_options)],
        "smpq_create": [ctypes.POINTER(P), I, P, ctypes.POINTER(smpq_options)],
        "smpq_destroy": [P],
        "smpq_set_options": [P, ctypes.POINTER(smpq_options)],
        "smpq_load_gauge": [P, PI, P, I],
        "smpq_set_spectrum": [P, D, D],
        "smpq_measure_spectrum": [P, I, PD, PD],
        "smpq_zolotarev": [I, D, D, PD, P, P, PD],
        "smpq_get_zolotarev": [P, PD, P, P, PD],
        "smpq_build_sources": [P, I, I, PI],
        "smpq_colour_sites": [PI, I, I, P, PI],
        "smpq_dslash": [P, P, P, I, I, I, I],
        "smpq_dslash_noalloc": [P, P, P, I, I, I],
        "smpq_time_dslash": [P, I, I, I, I, PD, PD],
        "smpq_apply_dov": [P, P, P, I, I],
        "smpq_compute_qx": [P, P, P, I, PD, ctypes.POINTER(smpq_stats)],
        "smpq_compute_qx_classes": [P, PI, I, P, P, I, ctypes.POINTER(smpq_stats)],
        "smpq_trace_dwinv": [P, P, P, I, PD, ctypes.POINTER(smpq_stats)],
        "smpq_compute_qx_batch": [P, I, P, P, I, PD, ctypes.POINTER(smpq_stats)],
        "smpq_low_modes": [P, I, I, D, I, P, P, PI],
        "smpq_get_low_modes": [P, P, P, PI],
        "smpq_clear_low_modes": [P],
        "smpq_context_info": [P, PI, PI],
        "smpq_alu_peak": [I, I, PD],
        "smpq_tune_cache_lookup": [ctypes.c_char_p, ctypes.c_char_p, PI, I, I, PI],
        "smpq_tune_cache_store": [ctypes.c_char_p, ctypes.c_char_p, PI, I, I, PI, D],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = I
    L.smpq_last_error.argtypes = [P]
    L.smpq_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc, ctx=None):
    if rc != SMPQ_OK:
        msg = load().smpq_last_error(ctx).decode() if ctx else ""
        raise SmpqError(rc, msg)


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def smpq_context_info(ctx):
    """(dims, device) of a context; dims are zeros before a gauge field is loaded."""
    d = (ctypes.c_int * 4)()
    dev = ctypes.c_int()
    _check(load().smpq_context_info(ctx, d, ctypes.byref(dev)), ctx)
    return tuple(d), dev.value


ALU_FP32, ALU_FP32X2, ALU_FP64 = 0, 1, 2


def smpq_alu_peak(device=0, kind=ALU_FP32X2):
    """Measured lane operations (multiply-adds) per second of the GPU: kind
    ALU_FP32 (scalar FFMA), ALU_FP32X2 (packed two-lane FFMA2) or ALU_FP64."""
    v = ctypes.c_double()
    _check(load().smpq_alu_peak(device, kind, ctypes.byref(v)))
    return v.value


def smpq_tune_cache_lookup(path, device, dims, B, precision):
    """The cached launch shape (bc, tpb_hi, tpb_lo, nr, staged) or None."""
    d = (ctypes.c_int * 4)(*dims)
    sh = (ctypes.c_int * 5)()
    rc = load().smpq_tune_cache_lookup(os.fsencode(path), device.encode(), d, B, precision, sh)
    if rc == SMPQ_ESTATE:
        return None
    _check(rc)
    return tuple(sh)


def smpq_tune_cache_store(path, device, dims, B, precision, shape, ms):
    d = (ctypes.c_int * 4)(*dims)
    if len(shape) != 5:
        raise ValueError("a launch shape has 5 entries (bc, tpb_hi, tpb_lo, nr, staged)")
    sh = (ctypes.c_int * 5)(*shape)
    _check(load().smpq_tune_cache_store(os.fsencode(path), device.encode(), d, B, precision, sh, ms))


def _check_buf(ctx, a, count, kind, what):
    """Refuse, before any launch, a buffer the kernels could overrun or could
    not reach: it must hold `count` elements of `kind` ("complex128" or
    "float64") and, as device memory, sit on the context's GPU."""
    dims, dev = smpq_context_info(ctx)
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(kind):
            raise ValueError("%s: dtype %s, expected %s" % (what, a.dtype, kind))
        n = a.size
    elif hasattr(a, "data_ptr"):
        import torch
        want = torch.complex128 if kind == "complex128" else torch.float64
        if a.dtype != want:
            raise ValueError("%s: dtype %s, expected %s" % (what, a.dtype, want))
        if a.is_cuda and a.device.index != dev:
            raise ValueError("%s: on cuda:%d, the context runs on cuda:%d" % (what, a.device.index, dev))
        n = a.numel()
    else:
        raise TypeError("%s: expected a numpy array or a torch tensor" % what)
    if n < count:
        raise ValueError("%s: %d elements, the call reads or writes %d" % (what, n, count))


def _volume(ctx):
    dims, _ = smpq_context_info(ctx)
    V = int(np.prod(dims))
    if V == 0:
        raise SmpqError(SMPQ_ESTATE, "no gauge field loaded")
    return V


# ----------------------------------------------------------------------------- thin wrappers (same names)


def smpq_options_default():
    o = smpq_options()
    _check(load().smpq_options_default(ctypes.byref(o)))
    return o


def smpq_create(device=0, stream=None, options=None):
    ctx = ctypes.c_void_p()
    o = options if options is not None else smpq_options_default()
    _check(load().smpq_create(ctypes.byref(ctx), device, stream, ctypes.byref(o)))
    return ctx


def smpq_destroy(ctx):
    _check(load().smpq_destroy(ctx))


def smpq_last_error(ctx):
    return load().smpq_last_error(ctx).decode()


def smpq_set_options(ctx, options):
    _check(load().smpq_set_options(ctx, ctypes.byref(options)), ctx)


def smpq_load_gauge(ctx, dims, links):
    d = (ctypes.c_int * 4)(*dims)
    _check_buf(ctx, links, int(np.prod(dims)) * 36, "complex128", "links")
    p, dev = _ptr(links)
    _check(load().smpq_load_gauge(ctx, d, p, dev), ctx)


def smpq_set_spectrum(ctx, lmin2, lmax2):
    _check(load().smpq_set_spectrum(ctx, lmin2, lmax2), ctx)


def smpq_measure_spectrum(ctx, iters=200):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(load().smpq_measure_spectrum(ctx, iters, ctypes.byref(lo), ctypes.byref(hi)), ctx)
    return lo.value, hi.value


def smpq_low_modes(ctx, k, block=0, tol=0.0, max_iter=0):
    """(evals[k+1] signed, ordered by |lambda|; residual norms[k+1]; filter steps)."""
    ev = np.zeros(k + 1)
    res = np.zeros(k + 1)
    it = ctypes.c_int()
    _check(load().smpq_low_modes(ctx, k, block, tol, max_iter, ev.ctypes.data, res.ctypes.data, ctypes.byref(it)),
           ctx)
    return ev, res, it.value


def smpq_get_low_modes(ctx, V):
    """(evals[k], evecs complex[V, 4, 3, k]) of the modes in use (k may be 0)."""
    k = ctypes.c_int()
    _check(load().smpq_get_low_modes(ctx, None, None, ctypes.byref(k)), ctx)
    ev = np.zeros(k.value)
    vec = np.zeros((V, 4, 3, k.value), dtype=np.complex128)
    if k.value:
        _check(load().smpq_get_low_modes(ctx, vec.ctypes.data, ev.ctypes.data, ctypes.byref(k)), ctx)
    return ev, vec


def smpq_clear_low_modes(ctx):
    _check(load().smpq_clear_low_modes(ctx), ctx)


def smpq_zolotarev(npoles, a, b):
    c0, delta = ctypes.c_double(), ctypes.c_double()
    c = np.zeros(npoles)
    q = np.zeros(npoles)
    _check(load().smpq_zolotarev(npoles, a, b, ctypes.byref(c0), c.ctypes.data, q.ctypes.data, ctypes.byref(delta)))
    return c0.value, c, q, delta.value


def smpq_get_zolotarev(ctx, npoles):
    c0, delta = ctypes.c_double(), ctypes.c_double()
    c = np.zeros(npoles)
    q = np.zeros(npoles)
    _check(load().smpq_get_zolotarev(ctx, ctypes.byref(c0), c.ctypes.data, q.ctypes.data, ctypes.byref(delta)), ctx)
    return c0.value, c, q, delta.value


def smpq_build_sources(ctx, r, mode):
    n = ctypes.c_int()
    _check(load().smpq_build_sources(ctx, r, mode, ctypes.byref(n)), ctx)
    return n.value


def smpq_colour_sites(dims, r, mode):
    d = (ctypes.c_int * 4)(*dims)
    V = int(np.prod(dims))
    col = np.zeros(V, dtype=np.int32)
    n = ctypes.c_int()
    _check(load().smpq_colour_sites(d, r, mode, col.ctypes.data, ctypes.byref(n)))
    return col, n.value


def _check_fields(ctx, inp, out, B):
    n = _volume(ctx) * 12 * B
    _check_buf(ctx, inp, n, "complex128", "in")
    _check_buf(ctx, out, n, "complex128", "out")


def _check_sites(ctx, a, b, names):
    V = _volume(ctx)
    _check_buf(ctx, a, V, "float64", names[0])
    _check_buf(ctx, b, V, "float64", names[1])


def smpq_dslash(ctx, inp, out, B, dagger=False, precision=SMPQ_FP64):
    _check_fields(ctx, inp, out, B)
    pi, di = _ptr(inp)
    po, do = _ptr(out)
    if di != do:
        raise ValueError("in and out must both be host or both be device buffers")
    _check(load().smpq_dslash(ctx, pi, po, B, int(dagger), precision, di), ctx)


def smpq_time_dslash(ctx, B, dagger=False, precision=SMPQ_FP32, reps=10):
    """Average ms of one stand-alone D_W launch on B scratch columns, and the
    algorithmic bytes of that launch: returns (ms, bytes)."""
    ms, nbytes = ctypes.c_double(), ctypes.c_double()
    _check(load().smpq_time_dslash(ctx, B, int(dagger), precision, reps, ctypes.byref(ms), ctypes.byref(nbytes)),
           ctx)
    return ms.value, nbytes.value


def smpq_dslash_noalloc(ctx, inp, out, B, dagger=False, precision=SMPQ_FP64):
    """Allocation-free D_W for callers that cannot allocate device memory:
    `inp` and `out` must be device buffers (torch CUDA tensors)."""
    _check_fields(ctx, inp, out, B)
    pi, di = _ptr(inp)
    po, do = _ptr(out)
    if not (di and do):
        raise ValueError("smpq_dslash_noalloc takes device buffers only")
    _check(load().smpq_dslash_noalloc(ctx, pi, po, B, int(dagger), precision), ctx)


def smpq_apply_dov(ctx, inp, out, B):
    _check_fields(ctx, inp, out, B)
    pi, di = _ptr(inp)
    po, do = _ptr(out)
    if di != do:
        raise ValueError("in and out must both be host or both be device buffers")
    _check(load().smpq_apply_dov(ctx, pi, po, B, di), ctx)


def smpq_compute_qx(ctx, q_re, q_im):
    _check_sites(ctx, q_re, q_im, ("q_re", "q_im"))
    pr, dr = _ptr(q_re)
    pm, dm = _ptr(q_im)
    if dr != dm:
        raise ValueError("q_re and q_im must both be host or both be device buffers")
    Q = ctypes.c_double()
    st = smpq_stats()
    _check(load().smpq_compute_qx(ctx, pr, pm, dr, ctypes.byref(Q), ctypes.byref(st)), ctx)
    return Q.value, st.as_dict()


def smpq_compute_qx_classes(ctx, classes, q_re, q_im):
    cl = np.ascontiguousarray(classes, dtype=np.int32)
    _check_sites(ctx, q_re, q_im, ("q_re", "q_im"))
    pr, dr = _ptr(q_re)
    pm, dm = _ptr(q_im)
    st = smpq_stats()
    _check(load().smpq_compute_qx_classes(ctx, cl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cl.size, pr, pm, dr,
                                          ctypes.byref(st)), ctx)
    return st.as_dict()


def smpq_trace_dwinv(ctx, t_re, t_im):
    _check_sites(ctx, t_re, t_im, ("t_re", "t_im"))
    pr, dr = _ptr(t_re)
    pm, dm = _ptr(t_im)
    if dr != dm:
        raise ValueError("t_re and t_im must both be host or both be device buffers")
    T = ctypes.c_double()
    st = smpq_stats()
    _check(load().smpq_trace_dwinv(ctx, pr, pm, dr, ctypes.byref(T), ctypes.byref(st)), ctx)
    return T.value, st.as_dict()


def smpq_compute_qx_batch(ctxs, q_re, q_im):
    """Uneven batch over several contexts; q_re/q_im: lists of per-lattice buffers."""
    n = len(ctxs)
    for c, a, b in zip(ctxs, q_re, q_im):
        _check_sites(c, a, b, ("q_re", "q_im"))
    pr = [_ptr(a) for a in q_re]
    pm = [_ptr(a) for a in q_im]
    dev = {d for _, d in pr + pm}
    if len(dev) != 1:
        raise ValueError("all buffers must be host or all device")
    C = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    R = (ctypes.c_void_p * n)(*[p for p, _ in pr])
    M = (ctypes.c_void_p * n)(*[p for p, _ in pm])
    Q = (ctypes.c_double * n)()
    st = (smpq_stats * n)()
    rc = load().smpq_compute_qx_batch(C, n, R, M, dev.pop(), Q, st)
    if rc != SMPQ_OK:
        raise SmpqError(rc, "uneven batch failed")
    return list(Q), [x.as_dict() for x in st]
