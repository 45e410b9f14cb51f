"""Pins of the oracle's low-mode projection (oracle/lowmodes.py): the exact
treatment of the lowest eigenmodes of H_W in eps(H_W) (Eq. 4), on the 4^4 flux
configuration, against the dense eigen-decomposition."""
import numpy as np
import pytest

from conftest import KAPPA, NPOLES
from oracle import lowmodes, probing, qx, zolotarev

K4 = 8  # 4^4 flux: |lambda|^2 jumps from 0.0225 (8th mode) to 0.0434 (9th)


@pytest.fixture(scope="module")
def proj4(flux4, dense4):
    lam = dense4["lam"]
    l2 = np.sort(lam ** 2)
    a, b = 0.98 * l2[K4], 1.02 * l2[-1]
    c0, c, q, delta = zolotarev.zolotarev(NPOLES, a, b)
    modes = lowmodes.low_modes_dense(flux4["U"], flux4["dims"], KAPPA, K4)
    return dict(zolo=(c0, c, q), delta=delta, a=a, modes=modes)


def test_dense_low_modes_are_the_smallest(dense4, proj4):
    lam, W = proj4["modes"]
    assert len(lam) == K4 + 1
    ref = np.sort(np.abs(dense4["lam"]))[: K4 + 1]
    assert np.allclose(np.abs(lam), ref, atol=1e-13)
    H = dense4["H"]
    assert np.abs(H @ W - W * lam[None, :]).max() <= 1e-12
    assert np.abs(W.conj().T @ W - np.eye(K4 + 1)).max() <= 1e-12


def test_matrix_free_low_modes_match_dense(flux4, dense4, proj4):
    """ARPACK on H^2 + Rayleigh-Ritz with H gives the same eigenvalues and the
    same projector onto the low space as the dense eigen-decomposition."""
    lam, W = lowmodes.low_modes(flux4["U"], flux4["dims"], KAPPA, K4, tol=1e-13)
    lam_d, W_d = proj4["modes"]
    assert np.abs(lam[:K4] - lam_d[:K4]).max() <= 1e-10
    P = W[:, :K4] @ W[:, :K4].conj().T
    P_d = W_d[:, :K4] @ W_d[:, :K4].conj().T
    assert np.abs(P - P_d).max() <= 1e-8


@pytest.mark.parametrize("r,mode,ncls", [(2, 0, 4), (2, 1, 3)])
def test_projected_smp_vs_dense(flux4, proj4, r, mode, ncls):
    """q^SMP(x) with the 8 lowest modes exact equals 1/2 sum_{y in S(x)} of the
    diagonal blocks of gamma_5 + W diag(f) W^dag with f = sign(lambda) on the
    low modes and lambda R(lambda^2) (Zolotarev on the shortened interval)
    elsewhere."""
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, r, mode)
    cls = list(range(0, n, max(1, n // ncls)))[:ncls]
    lam, W = proj4["modes"]
    q, st = lowmodes.smp_qx_projected(U, dims, KAPPA, proj4["zolo"], colour, n, (lam[:K4], W[:, :K4]),
                                      colours=cls, batch_colours=ncls)
    ref = qx.dense_smp_qx(lowmodes.dense_g5dov_projected(U, dims, KAPPA, proj4["zolo"], K4), colour)
    mask = np.isin(colour, cls)
    assert np.abs(q[mask] - ref[mask]).max() <= 1e-10


def test_projection_needs_the_low_term(flux4, dense4, proj4):
    """The low-mode term moves q^SMP(x) by up to ~4e-3 per site: the pin above
    fails if the term is dropped or its sign flipped.  (With 14 poles the
    rational stays within ~1e-10 of sign(lambda) even at the low modes below
    the shortened interval, so what the projection gains is the shorter Krylov
    spectrum, not accuracy.)"""
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, 2, 0)
    lam, W = dense4["lam"], dense4["W"]
    low = np.argsort(np.abs(lam), kind="stable")[:K4]
    term = (W[:, low] * np.sign(lam[low])[None, :]) @ W[:, low].conj().T
    M = lowmodes.dense_g5dov_projected(U, dims, KAPPA, proj4["zolo"], K4)
    ref = qx.dense_smp_qx(M, colour)
    without = qx.dense_smp_qx(M - term, colour)
    assert np.abs(ref - without).max() > 1e-3


def test_projected_exact_trace_is_the_index(dense4, proj4, flux4):
    """Q = 1/2 tr eps(H) with the low modes exact: the low modes add
    1/2 sum sign(lambda), the rest the rational; the index is met within
    6 V delta of the shortened interval, whose delta is smaller."""
    lam = dense4["lam"]
    low = np.argsort(np.abs(lam), kind="stable")[:K4]
    c0, c, q = proj4["zolo"]
    f = lam * zolotarev.rational(lam ** 2, c0, c, q)
    f[low] = np.sign(lam[low])
    Q = 0.5 * f.sum()
    assert abs(Q - flux4["Q_closed"]) <= 6 * 256 * proj4["delta"] + 1e-10
    _, _, _, delta_full = zolotarev.zolotarev(NPOLES, 0.98 * (lam ** 2).min(), 1.02 * (lam ** 2).max())
    assert proj4["delta"] < delta_full


def test_no_modes_is_the_unprojected_estimate(flux4, zolo4):
    """k = 0: b_perp = b and no low term, so the projected path is qx.smp_qx."""
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, 2, 0)
    zolo = (zolo4["c0"], zolo4["c"], zolo4["q"])
    empty = (np.zeros(0), np.zeros((12 * 256, 0), dtype=np.complex128))
    a, _ = lowmodes.smp_qx_projected(U, dims, KAPPA, zolo, colour, n, empty, colours=[0, 3], batch_colours=2)
    b, _ = qx.smp_qx(U, dims, KAPPA, zolo, colour, n, colours=[0, 3], batch_colours=2)
    assert np.abs(a - b).max() <= 1e-14
