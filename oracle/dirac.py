"""Wilson kernel of the overlap operator (Sec. 2.1, around Eq. 3 and Eq. 4).

Conventions (the paper fixes only kappa = 0.21 and kappa in (kappa_c, 0.25)):
  * Euclidean chiral basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] for
    k = 1, 2, 3, gamma_4 = [[0, 1], [1, 0]], so gamma_5 = gamma_1 gamma_2
    gamma_3 gamma_4 = diag(1, 1, -1, -1);
  * D_W psi(x) = psi(x) - kappa sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                       + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ];
  * bc[mu] = +1 (periodic) or -1 (antiperiodic) multiplies every hop that
    crosses the lattice boundary in direction mu.
Spinors are complex128 [V, 4, 3] or [V, 4, 3, B] (site, spin, colour[, rhs]).
"""
from __future__ import annotations

import numpy as np

_S = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)

GAMMA = np.stack(
    [np.block([[_Z2, -1j * _S[k]], [1j * _S[k], _Z2]]) for k in range(3)]
    + [np.block([[_Z2, _I2], [_I2, _Z2]])]
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)


def _hop_fwd(psi, dims, mu, bc):
    """psi(x + mu_hat), with the boundary phase on sites whose x_mu = n_mu - 1."""
    nx, ny, nz, nt = dims
    shp = psi.shape
    f = psi.reshape((nt, nz, ny, nx) + shp[1:])
    axis = 3 - mu
    g = np.roll(f, -1, axis=axis)
    if bc[mu] != 1:
        idx = [slice(None)] * g.ndim
        idx[axis] = dims[mu] - 1
        g = g.copy()
        g[tuple(idx)] *= bc[mu]
    return g.reshape(shp)


def _hop_bwd(psi, dims, mu, bc):
    """psi(x - mu_hat), with the boundary phase on sites whose x_mu = 0."""
    nx, ny, nz, nt = dims
    shp = psi.shape
    f = psi.reshape((nt, nz, ny, nx) + shp[1:])
    axis = 3 - mu
    g = np.roll(f, +1, axis=axis)
    if bc[mu] != 1:
        idx = [slice(None)] * g.ndim
        idx[axis] = 0
        g = g.copy()
        g[tuple(idx)] *= bc[mu]
    return g.reshape(shp)


def apply_dw(U, psi, dims, kappa, bc=(1, 1, 1, 1)):
    """D_W psi for psi[V,4,3] or psi[V,4,3,B]."""
    out = psi.copy()
    batched = psi.ndim == 4
    for mu in range(4):
        Umu = U[:, mu]
        # forward hop: (1 - gamma_mu) U_mu(x) psi(x + mu)
        pf = _hop_fwd(psi, dims, mu, bc)
        if batched:
            up = np.einsum("sab,sibn->sian", Umu, pf)
            out -= kappa * np.einsum("ij,sjan->sian", ONE4 - GAMMA[mu], up)
        else:
            up = np.einsum("sab,sib->sia", Umu, pf)
            out -= kappa * np.einsum("ij,sja->sia", ONE4 - GAMMA[mu], up)
        # backward hop: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
        Ub = _hop_bwd(Umu, dims, mu, (1, 1, 1, 1))
        pb = _hop_bwd(psi, dims, mu, bc)
        if batched:
            dn = np.einsum("sba,sibn->sian", Ub.conj(), pb)
            out -= kappa * np.einsum("ij,sjan->sian", ONE4 + GAMMA[mu], dn)
        else:
            dn = np.einsum("sba,sib->sia", Ub.conj(), pb)
            out -= kappa * np.einsum("ij,sja->sia", ONE4 + GAMMA[mu], dn)
    return out


def apply_g5(psi):
    """gamma_5 acting on the spin index."""
    if psi.ndim == 4:
        return np.einsum("ij,sjan->sian", GAMMA5, psi)
    return np.einsum("ij,sja->sia", GAMMA5, psi)


def apply_h(U, psi, dims, kappa, bc=(1, 1, 1, 1)):
    """H_W = gamma_5 D_W (Hermitian; the argument of the sign function in Eq. 3)."""
    return apply_g5(apply_dw(U, psi, dims, kappa, bc))


def apply_h2(U, psi, dims, kappa, bc=(1, 1, 1, 1)):
    """H_W^2 = D_W^dag D_W = gamma_5 D_W gamma_5 D_W (the matrix of Eq. 4)."""
    return apply_h(U, apply_h(U, psi, dims, kappa, bc), dims, kappa, bc)


def dense_dw(U, dims, kappa, bc=(1, 1, 1, 1)):
    """Dense 12V x 12V matrix of D_W, index (site, spin, colour) row-major.

    Built column by column from apply_dw on unit vectors (the matrix is the
    operator's definition written out; used on 4^4 only).
    """
    V = int(np.prod(dims))
    n = 12 * V
    eye = np.zeros((V, 4, 3, n), dtype=np.complex128)
    eye.reshape(n, n)[np.arange(n), np.arange(n)] = 1.0
    cols = apply_dw(U, eye, dims, kappa, bc)
    return cols.reshape(n, n)
