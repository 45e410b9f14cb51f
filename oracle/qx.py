"""Topological charge density by point sources and by SMP sources (Eqs. 3-5, 15-16).

  gamma_5 D_ov = gamma_5 + eps(H_W) = gamma_5 + gamma_5 D_W R(H_W^2)          (Eqs. 3-4)
  q(x)  = 1/2 sum_{alpha,a} <psi(x,alpha,a)| gamma_5 D_ov |psi(x,alpha,a)>   (Eq. 5)
  q^SMP(x) = 1/2 sum_{alpha,a} <psi(x,alpha,a)| gamma_5 D_ov |phi_P(S(x),alpha,a)>  (Eq. 16,
             with D~_ov = gamma_5 D_ov / 2)

For a source b, y = R(H^2) b = c0 b + sum_i c_i x_i with x_i = (H^2 + q_i)^{-1} b
(Eqs. 6-8), z = D_W y, and gamma_5 D_ov b = gamma_5 (b + z).  The gamma_5 b part
contributes 1/2 * 3 * tr(gamma_5) = 0 to every site, so
  q(x) = 1/2 sum_{alpha,a} (gamma_5 z_{alpha,a})(x, alpha, a).
SMP estimates are complex per site (off-diagonal terms); Q = sum_x q(x) is real
up to rounding.
"""
from __future__ import annotations

import numpy as np

from . import dirac, msolve, native, probing


def smp_qx(U, dims, kappa, zolo, colour, n_colours, tol=1e-13, bc=(1, 1, 1, 1),
           colours=None, batch_colours=8, max_iter=100000, backend="c"):
    """Complex q^SMP(x) for every site whose colour is in `colours` (default: all).

    zolo = (c0, c[n], q[n]).  Returns (q[V] complex, stats) with q = 0 on sites
    whose colour was not processed.  backend "c" runs the solver and D_W in the
    compiled oracle (oracle/c/oracle.c), "numpy" in oracle/dirac.py + msolve.py.
    """
    c0, c, q = zolo
    V = int(np.prod(dims))
    if colours is None:
        colours = range(n_colours)
    colours = list(colours)
    out = np.zeros(V, dtype=np.complex128)
    iters = []
    worst = 0.0
    def A(v):
        return dirac.apply_h2(U, v.reshape(V, 4, 3, -1), dims, kappa, bc).reshape(12 * V, -1)
    for start in range(0, len(colours), batch_colours):
        cls = colours[start:start + batch_colours]
        b = probing.smp_sources(colour, cls)
        B = b.shape[-1]
        if backend == "numpy":
            xs, k, info = msolve.multishift_cg(A, b.reshape(12 * V, B), q, tol, max_iter)
            res = info["resid"]
        else:
            xs, k, res = native.multishift_cg(U, dims, kappa, b, q, tol, bc, max_iter)
            xs = xs.reshape(len(q), 12 * V, B)
        iters.append(k)
        worst = max(worst, float(res.max()))
        y = c0 * b.reshape(12 * V, B) + np.einsum("i,inb->nb", c, xs)
        if backend == "numpy":
            z = dirac.apply_dw(U, y.reshape(V, 4, 3, B), dims, kappa, bc)
        else:
            z = native.apply_dw(U, y.reshape(V, 4, 3, B), dims, kappa, bc)
        g5z = dirac.apply_g5(z)
        for j, cl in enumerate(cls):
            sites = np.nonzero(colour == cl)[0]
            acc = np.zeros(len(sites), dtype=np.complex128)
            for alpha in range(4):
                for a in range(3):
                    acc += g5z[sites, alpha, a, 12 * j + 3 * alpha + a]
            out[sites] = 0.5 * acc
    return out, dict(iterations=iters, max_recursive_resid=worst)


def point_qx(U, dims, kappa, zolo, tol=1e-13, bc=(1, 1, 1, 1), sites=None, batch_sites=8, backend="c"):
    """Exact q(x) (Eq. 5) from the 12 point sources of each listed site (default all)."""
    V = int(np.prod(dims))
    colour = np.arange(V)
    if sites is None:
        sites = range(V)
    return smp_qx(U, dims, kappa, zolo, colour, V, tol, bc, colours=list(sites),
                  batch_colours=batch_sites, backend=backend)


def total_charge(q):
    """Q = sum_x q(x) in site order (real part), and max |Im q(x)|."""
    return float(np.sum(q.real)), float(np.max(np.abs(q.imag))) if q.size else 0.0


# ----------------------------------------------------------------------------- dense forms (4^4 pins)


def dense_g5dov(U, dims, kappa, zolo, bc=(1, 1, 1, 1)):
    """Dense gamma_5 D_ov = gamma_5 + H R(H^2) (same rational as the solver path)."""
    c0, c, q = zolo
    Dw = dirac.dense_dw(U, dims, kappa, bc)
    V = int(np.prod(dims))
    g5 = np.kron(np.eye(V), np.kron(dirac.GAMMA5, np.eye(3)))
    H = g5 @ Dw
    lam, W = np.linalg.eigh(H)
    f = lam * (c0 + np.sum(c[None, :] / (lam[:, None] ** 2 + q[None, :]), axis=1))
    return g5 + (W * f[None, :]) @ W.conj().T, lam, W


def dense_smp_qx(M, colour):
    """q^SMP(x) = 1/2 sum_{y in S(x)} sum_{alpha,a} M[(x,alpha,a), (y,alpha,a)] (Eq. 16)."""
    V = colour.shape[0]
    Mr = M.reshape(V, 12, V, 12)
    diag12 = np.einsum("xiyi->xy", Mr)
    same = colour[:, None] == colour[None, :]
    return 0.5 * np.sum(np.where(same, diag12, 0.0), axis=1)


# ----------------------------------------------------------------------------- trace of D_W^{-1} (Sec. 4 outlook)


def smp_trace_dwinv(U, dims, kappa, colour, n_colours, tol=1e-13, bc=(1, 1, 1, 1), colours=None, batch_colours=8,
                    max_iter=100000):
    """SMP estimate t(x) = sum_{alpha,a} <psi(x,alpha,a)| D_W^{-1} |phi_P(S(x),alpha,a)>.

    D_W^{-1} b is computed as (D_W^dag D_W)^{-1} D_W^dag b (CG on the normal
    equations; D_W^dag = gamma_5 D_W gamma_5).  Returns (t[V] complex, stats).
    """
    V = int(np.prod(dims))
    if colours is None:
        colours = range(n_colours)
    colours = list(colours)
    out = np.zeros(V, dtype=np.complex128)
    iters = []
    for start in range(0, len(colours), batch_colours):
        cls = colours[start:start + batch_colours]
        b = probing.smp_sources(colour, cls)
        bd = dirac.apply_g5(native.apply_dw(U, dirac.apply_g5(b), dims, kappa, bc))
        xs, k, res = native.multishift_cg(U, dims, kappa, bd, [0.0], tol, bc, max_iter)
        iters.append(k)
        x = xs[0]
        for j, cl in enumerate(cls):
            sites = np.nonzero(colour == cl)[0]
            acc = np.zeros(len(sites), dtype=np.complex128)
            for alpha in range(4):
                for a in range(3):
                    acc += x[sites, alpha, a, 12 * j + 3 * alpha + a]
            out[sites] = acc
    return out, dict(iterations=iters)


def dense_smp_trace(Minv, colour):
    """t^SMP(x) = sum_{y in S(x)} sum_{alpha,a} Minv[(x,alpha,a), (y,alpha,a)]."""
    return 2.0 * dense_smp_qx(Minv, colour)
