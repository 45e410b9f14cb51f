"""Shifted solves (D_W^dag D_W + q_i) x_i = b of Eqs. 6-8 (Sec. 2.1).

The paper solves M_i v_i = b, M_i = (D_W^dag D_W + q_i)/c_i, by CG for every
source.  All shifts share one Krylov space, so one multi-shift CG (Frommer et
al. 1995; Jegerlehner, hep-lat/9612014) yields every x_i = (A + q_i)^{-1} b at
the cost of the smallest shift; c_i is applied afterwards (c_i v_i-form of Eq. 6
is x_i * c_i).  Written out from the CG recurrences:

  base system (A + s0) x = b, s0 = min_i q_i, relative shifts sig_i = q_i - s0;
  alpha_k = <r_k, r_k> / <p_k, (A + s0) p_k>,   r_{k+1} = r_k - alpha_k (A + s0) p_k,
  beta_k = <r_{k+1}, r_{k+1}> / <r_k, r_k>,    p_{k+1} = r_{k+1} + beta_k p_k;
  shifted residuals stay collinear, r^i_k = zeta^i_k r_k, with
  zeta^i_{k+1} = zeta^i_k zeta^i_{k-1} alpha_{k-1} /
                 (alpha_k beta_{k-1} (zeta^i_{k-1} - zeta^i_k)
                  + zeta^i_{k-1} alpha_{k-1} (1 + sig_i alpha_k)),
  alpha^i_k = alpha_k zeta^i_{k+1}/zeta^i_k,  beta^i_k = beta_k (zeta^i_{k+1}/zeta^i_k)^2,
  x^i += alpha^i_k p^i_k,  p^i_{k+1} = zeta^i_{k+1} r_{k+1} + beta^i_k p^i_k,
  starting from zeta_0 = zeta_{-1} = 1, alpha_{-1} = 1, beta_{-1} = 0, p^i_0 = b.
Shift i of column j stops updating once |zeta^i| ||r|| <= tol ||b||.

Vectors are 2-D arrays [N, B]: B independent right-hand sides, each with its own
scalars (the columns never mix).
"""
from __future__ import annotations

import numpy as np


def _dot(u, v):
    return np.einsum("nb,nb->b", u.conj(), v)


def cg(apply_A, b, shift, tol, max_iter=10000):
    """Plain CG for (A + shift) x = b, columns independent.  Returns (x, iters)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = b.copy()
    rr = _dot(r, r).real
    bb = rr.copy()
    active = rr > tol * tol * bb
    k = 0
    while active.any() and k < max_iter:
        Ap = apply_A(p) + shift * p
        pAp = _dot(p, Ap).real
        alpha = np.where(active, rr / np.where(active, pAp, 1.0), 0.0)
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = _dot(r, r).real
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        p = np.where(active, r + beta * p, p)
        rr = np.where(active, rr_new, rr)
        active = active & (rr > tol * tol * bb)
        k += 1
    return x, k


def multishift_cg(apply_A, b, shifts, tol, max_iter=10000):
    """Multi-shift CG.  b: [N, B]; shifts: [n] (any order, all > -lambda_min(A)).

    Returns (x[n, N, B] in the order of `shifts`, iterations, info) where info
    holds the final recursive residual ratios |zeta| ||r|| / ||b|| per shift.
    """
    shifts = np.asarray(shifts, dtype=np.float64)
    n = shifts.size
    N, B = b.shape
    s0 = shifts.min()
    sig = shifts - s0
    x = np.zeros((n, N, B), dtype=b.dtype)
    ps = np.repeat(b[None], n, axis=0)
    r = b.copy()
    p = b.copy()
    rr = _dot(r, r).real
    bb = rr.copy()
    zeta = np.ones((n, B))
    zeta_prev = np.ones((n, B))
    alpha_prev = np.ones(B)
    beta_prev = np.zeros(B)
    tol2 = tol * tol
    active = np.repeat((rr > tol2 * bb)[None], n, axis=0)  # per (shift, column)
    k = 0
    while active.any() and k < max_iter:
        col = active.any(axis=0)
        Ap = apply_A(p) + s0 * p
        pAp = _dot(p, Ap).real
        alpha = rr / np.where(col, pAp, 1.0)
        den = alpha[None] * beta_prev[None] * (zeta_prev - zeta) + zeta_prev * alpha_prev[None] * (
            1.0 + sig[:, None] * alpha[None]
        )
        zeta_new = np.where(active, zeta * zeta_prev * alpha_prev[None] / np.where(active, den, 1.0), zeta)
        alpha_s = np.where(active, alpha[None] * zeta_new / np.where(active, zeta, 1.0), 0.0)
        x = x + alpha_s[:, None, :] * ps
        r_new = np.where(col, r - alpha * Ap, r)
        rr_new = _dot(r_new, r_new).real
        beta = np.where(col, rr_new / rr, 0.0)
        beta_s = beta[None] * (zeta_new / zeta) ** 2
        ps = np.where(active[:, None, :], zeta_new[:, None, :] * r_new[None] + beta_s[:, None, :] * ps, ps)
        p = np.where(col, r_new + beta * p, p)
        r = r_new
        zeta_prev = np.where(active, zeta, zeta_prev)
        zeta = zeta_new
        alpha_prev = np.where(col, alpha, alpha_prev)
        beta_prev = np.where(col, beta, beta_prev)
        rr = np.where(col, rr_new, rr)
        active = active & (zeta**2 * rr[None] > tol2 * bb[None])
        k += 1
    info = dict(resid=np.sqrt(zeta**2 * rr[None] / bb[None]), converged=not active.any())
    return x, k, info


def true_residuals(apply_A, b, shifts, x):
    """||b - (A + q_i) x_i|| / ||b|| per shift and column (FP64)."""
    out = np.empty((len(shifts), b.shape[1]))
    bn = np.sqrt(_dot(b, b).real)
    for i, q in enumerate(shifts):
        r = b - apply_A(x[i]) - q * x[i]
        out[i] = np.sqrt(_dot(r, r).real) / bn
    return out
