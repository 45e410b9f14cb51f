"""Low modes of H_W = gamma_5 D_W projected out of the sign function.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper evaluates eps(H_W) with the Zolotarev rational on the whole spectrum
(Eq. 4) and, at the end of Sec. 3, compares the SMP cost with low modes of the
overlap operator.  Treating the lowest eigenmodes of H_W exactly is the
standard way overlap codes shorten the Zolotarev interval; it is not in the
paper.  With the k eigenpairs (lambda_j, v_j) of smallest |lambda|,

  eps(H) = sum_{j<k} sign(lambda_j) v_j v_j^dag + H R(H^2) P_perp,
  P_perp = 1 - sum_{j<k} v_j v_j^dag,

and R is the Zolotarev rational on [a, b] with a below lambda_{k+1}^2, the
smallest eigenvalue of H^2 on the complement.  For an SMP source b the solves
run on b_perp = P_perp b; y = R(H^2) b_perp = c0 b_perp + sum_i c_i x_i and

  eps(H) b = gamma_5 D_W y + sum_j sign(lambda_j) v_j (v_j^dag b),

so q^SMP(x) (Eq. 16) gains the low-mode term 1/2 sum_{alpha,a} sum_j
sign(lambda_j) v_j(x, alpha, a) (v_j^dag b_{alpha,a}) next to the usual
contraction of gamma_5 D_W y.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh

from . import dirac, msolve, native, probing


def dense_h(U, dims, kappa, bc=(1, 1, 1, 1)):
    """Dense H_W = gamma_5 D_W (12V x 12V)."""
    V = int(np.prod(dims))
    g5 = np.kron(np.eye(V), np.kron(dirac.GAMMA5, np.eye(3)))
    return g5 @ dirac.dense_dw(U, dims, kappa, bc)


def low_modes_dense(U, dims, kappa, k, bc=(1, 1, 1, 1)):
    """The k + 1 eigenpairs of H_W of smallest |lambda| from the dense
    eigen-decomposition, ordered by |lambda|: (lambda[k+1], V[12V, k+1])."""
    lam, W = np.linalg.eigh(dense_h(U, dims, kappa, bc))
    order = np.argsort(np.abs(lam), kind="stable")[: k + 1]
    return lam[order], W[:, order]


def low_modes(U, dims, kappa, k, bc=(1, 1, 1, 1), tol=1e-12, lmax2=8.0):
    """The k + 1 eigenpairs of H_W of smallest |lambda| without the dense matrix.

    ARPACK (scipy eigsh) finds the k + 1 lowest eigenvectors of H^2 as the
    highest of lmax2 - H^2 (H^2 applied by the compiled oracle); H is then
    diagonalised inside that subspace (Rayleigh-Ritz), which fixes the signs.
    Returns (lambda[k+1] ordered by |lambda|, V[12V, k+1])."""
    V = int(np.prod(dims))
    n = 12 * V

    def h2(v):
        return native.apply_h2(U, v.reshape(V, 4, 3), dims, kappa, bc).reshape(n)

    op = LinearOperator((n, n), matvec=lambda v: lmax2 * v - h2(v), dtype=np.complex128)
    _, X = eigsh(op, k=k + 1, which="LA", tol=tol, ncv=max(2 * (k + 1) + 1, 20))
    X, _ = np.linalg.qr(X)
    HX = np.stack([dirac.apply_h(U, X[:, j].reshape(V, 4, 3), dims, kappa, bc).reshape(n)
                   for j in range(X.shape[1])], axis=1)
    G = X.conj().T @ HX
    theta, Z = np.linalg.eigh(0.5 * (G + G.conj().T))
    order = np.argsort(np.abs(theta), kind="stable")
    return theta[order], (X @ Z)[:, order]


def dense_g5dov_projected(U, dims, kappa, zolo, k, bc=(1, 1, 1, 1)):
    """Dense gamma_5 D_ov with the k lowest modes of H_W exact:
    gamma_5 + W diag(f) W^dag, f = sign(lambda) on those k modes and
    lambda R(lambda^2) on the rest."""
    c0, c, q = zolo
    H = dense_h(U, dims, kappa, bc)
    lam, W = np.linalg.eigh(H)
    f = lam * (c0 + np.sum(c[None, :] / (lam[:, None] ** 2 + q[None, :]), axis=1))
    low = np.argsort(np.abs(lam), kind="stable")[:k]
    f[low] = np.sign(lam[low])
    V = int(np.prod(dims))
    g5 = np.kron(np.eye(V), np.kron(dirac.GAMMA5, np.eye(3)))
    return g5 + (W * f[None, :]) @ W.conj().T


def smp_qx_projected(U, dims, kappa, zolo, colour, n_colours, modes, tol=1e-13, bc=(1, 1, 1, 1),
                     colours=None, batch_colours=8, max_iter=100000, backend="c"):
    """q^SMP(x) (Eq. 16) with the low modes `modes = (lambda[k], V[12V, k])`
    treated exactly; returns (q[V] complex, stats) like qx.smp_qx."""
    c0, c, q = zolo
    lam, Vk = modes
    lam = np.asarray(lam)
    V = int(np.prod(dims))
    Vk = np.asarray(Vk).reshape(12 * V, len(lam))
    s = np.sign(lam)
    if colours is None:
        colours = range(n_colours)
    colours = list(colours)
    out = np.zeros(V, dtype=np.complex128)
    iters = []

    def A(v):
        return dirac.apply_h2(U, v.reshape(V, 4, 3, -1), dims, kappa, bc).reshape(12 * V, -1)

    for start in range(0, len(colours), batch_colours):
        cls = colours[start:start + batch_colours]
        b = probing.smp_sources(colour, cls).reshape(12 * V, -1)
        B = b.shape[-1]
        w = Vk.conj().T @ b  # v_j^dag b
        b_perp = b - Vk @ w
        if backend == "numpy":
            xs, k, _ = msolve.multishift_cg(A, b_perp, q, tol, max_iter)
        else:
            xs, k, _ = native.multishift_cg(U, dims, kappa, b_perp.reshape(V, 4, 3, B), q, tol, bc, max_iter)
            xs = xs.reshape(len(q), 12 * V, B)
        iters.append(k)
        y = c0 * b_perp + np.einsum("i,inb->nb", c, xs)
        z = native.apply_dw(U, y.reshape(V, 4, 3, B), dims, kappa, bc)
        eps_b = dirac.apply_g5(z).reshape(12 * V, B) + Vk @ (s[:, None] * w)
        eps_b = eps_b.reshape(V, 4, 3, B)
        for j, cl in enumerate(cls):
            sites = np.nonzero(colour == cl)[0]
            acc = np.zeros(len(sites), dtype=np.complex128)
            for alpha in range(4):
                for a in range(3):
                    acc += eps_b[sites, alpha, a, 12 * j + 3 * alpha + a]
            out[sites] = 0.5 * acc
    return out, dict(iterations=iters)
