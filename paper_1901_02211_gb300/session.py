"""Convenience wrapper over the C ABI (one context = one GPU, one stream)."""
from __future__ import annotations

import numpy as np

from . import smpq as S


class Session:
    """Owns one smpq context.  Options are smpq_options field names, e.g.
    Session(precision=S.SMPQ_FP32, tol=1e-10, rhs_block=0)."""

    def __init__(self, device=0, stream=None, **options):
        o = S.smpq_options_default()
        for k, v in options.items():
            if k == "bc":
                o.bc[:] = list(v)
            elif k == "tune_cache":
                o.tune_cache = None if v is None else str(v).encode()
            else:
                setattr(o, k, v)
        self.options = o
        self.ctx = S.smpq_create(device, stream, o)
        self.dims = None

    def close(self):
        if self.ctx is not None:
            S.smpq_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **options):
        for k, v in options.items():
            if k == "bc":
                self.options.bc[:] = list(v)
            elif k == "tune_cache":
                self.options.tune_cache = None if v is None else str(v).encode()
            else:
                setattr(self.options, k, v)
        S.smpq_set_options(self.ctx, self.options)

    def load_gauge(self, dims, U):
        U = np.ascontiguousarray(U, dtype=np.complex128) if isinstance(U, np.ndarray) else U
        S.smpq_load_gauge(self.ctx, dims, U)
        self.dims = tuple(dims)
        self.V = int(np.prod(dims))

    def set_spectrum(self, lmin2, lmax2):
        S.smpq_set_spectrum(self.ctx, lmin2, lmax2)

    def measure_spectrum(self, iters=200):
        return S.smpq_measure_spectrum(self.ctx, iters)

    def low_modes(self, k, block=0, tol=0.0, max_iter=0):
        """Treat the k lowest modes of H_W exactly from now on; returns
        (evals[k+1], residuals[k+1], filter steps)."""
        return S.smpq_low_modes(self.ctx, k, block, tol, max_iter)

    def get_low_modes(self):
        return S.smpq_get_low_modes(self.ctx, self.V)

    def clear_low_modes(self):
        S.smpq_clear_low_modes(self.ctx)

    def zolotarev(self):
        return S.smpq_get_zolotarev(self.ctx, self.options.npoles)

    def build_sources(self, r, mode=0):
        return S.smpq_build_sources(self.ctx, r, mode)

    def dslash(self, psi, dagger=False, precision=S.SMPQ_FP64):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        B = 1 if psi.ndim == 3 else psi.shape[-1]
        out = np.empty_like(psi)
        S.smpq_dslash(self.ctx, psi, out, B, dagger, precision)
        return out

    def apply_dov(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        B = 1 if psi.ndim == 3 else psi.shape[-1]
        out = np.empty_like(psi)
        S.smpq_apply_dov(self.ctx, psi, out, B)
        return out

    def compute_qx(self, classes=None, device=False):
        """Return (q complex[V], Q, stats).  device=True returns torch CUDA tensors."""
        if device:
            import torch
            q_re = torch.zeros(self.V, dtype=torch.float64, device="cuda")
            q_im = torch.zeros(self.V, dtype=torch.float64, device="cuda")
        else:
            q_re = np.zeros(self.V)
            q_im = np.zeros(self.V)
        if classes is None:
            Q, st = S.smpq_compute_qx(self.ctx, q_re, q_im)
        else:
            st = S.smpq_compute_qx_classes(self.ctx, classes, q_re, q_im)
            Q = st["Q"]
        if device:
            import torch
            return torch.complex(q_re, q_im), Q, st
        return q_re + 1j * q_im, Q, st

    def trace_dwinv(self):
        """SMP estimate of diag D_W^{-1}: (t complex[V], Tr, stats)."""
        t_re = np.zeros(self.V)
        t_im = np.zeros(self.V)
        T, st = S.smpq_trace_dwinv(self.ctx, t_re, t_im)
        return t_re + 1j * t_im, T, st
