"""Spectral bounds of H_W^2 = D_W^dag D_W (setup for the interval of Eq. 4).

The paper does not say how the Zolotarev interval is chosen.  Here the extreme
eigenvalues of H_W^2 are computed with ARPACK (scipy eigsh) on the operator, or
with a dense eigen-decomposition for small lattices, and widened by fixed
margins: [a, b] = [lo * lambda_min^2, hi * lambda_max^2].
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh

from . import dirac, native

MARGIN_LO = 0.98
MARGIN_HI = 1.02


def h2_extremes(U, dims, kappa, bc=(1, 1, 1, 1), tol=1e-10, backend="c"):
    """(lambda_min^2, lambda_max^2) of H_W^2 via eigsh on the matrix-free operator
    (applied by the compiled oracle, or by oracle/dirac.py with backend="numpy")."""
    V = int(np.prod(dims))
    n = 12 * V
    h2 = native.apply_h2 if backend == "c" else dirac.apply_h2

    def mv(v):
        return h2(U, v.reshape(V, 4, 3), dims, kappa, bc).reshape(n)

    op = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    lmax = eigsh(op, k=1, which="LA", tol=tol, return_eigenvectors=False)[0]
    # smallest eigenvalue of H^2 = largest of (lmax*1.01 - H^2)
    s = 1.01 * lmax
    op2 = LinearOperator((n, n), matvec=lambda v: s * v - mv(v), dtype=np.complex128)
    lmin = s - eigsh(op2, k=1, which="LA", tol=tol, return_eigenvectors=False)[0]
    return float(lmin), float(lmax)


def zolotarev_interval(lmin2, lmax2):
    return MARGIN_LO * lmin2, MARGIN_HI * lmax2
