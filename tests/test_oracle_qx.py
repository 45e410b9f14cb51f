"""Pins of the oracle's q(x) by point sources (Eq. 5) and SMP sources (Eq. 16)."""
import numpy as np
import pytest

from conftest import KAPPA, NPOLES
from oracle import probing, qx, zolotarev


def _zolo(z):
    return (z["c0"], z["c"], z["q"])


def test_exact_q_point_sources_vs_dense(flux4, g5dov4, zolo4):
    """q(x) = 1/2 tr_dc(gamma_5 D_ov)(x, x) from 12 point sources per site (Eq. 5)."""
    U, dims = flux4["U"], flux4["dims"]
    sites = [0, 1, 37, 128, 255]
    q, st = qx.point_qx(U, dims, KAPPA, _zolo(zolo4), sites=sites, batch_sites=5)
    ref = qx.dense_smp_qx(g5dov4, np.arange(256))
    assert np.abs(q[sites] - ref[sites]).max() <= 1e-10
    assert np.abs(ref.imag).max() <= 1e-14  # diagonal of a Hermitian matrix


def test_dense_exact_trace_is_integer(dense4, zolo4, g5dov4, flux4):
    """Q = 1/2 sum_lambda lambda R(lambda^2) equals the closed-form index within 6 V delta."""
    lam = dense4["lam"]
    f = lam * zolotarev.rational(lam ** 2, zolo4["c0"], zolo4["c"], zolo4["q"])
    Q = 0.5 * f.sum()
    bound = 6 * 256 * zolo4["delta"] + 1e-10
    assert abs(Q - round(Q)) <= bound
    assert round(Q) == flux4["Q_closed"] == 1
    # (n_+ - n_-)/2 from the eigenvalue signs
    assert ((lam > 0).sum() - (lam < 0).sum()) // 2 == 1
    Qd = qx.dense_smp_qx(g5dov4, np.arange(256)).real.sum()
    assert abs(Qd - Q) <= 1e-10


@pytest.mark.parametrize("r,mode,ncls", [(2, 0, 4), (2, 1, 4), (2, 2, 3), (4, 2, 4)])
def test_smp_vs_dense(flux4, g5dov4, zolo4, r, mode, ncls):
    """q^SMP(x) = 1/2 sum_{y in S(x)} sum_{alpha,a} (gamma_5 D_ov)(x alpha a; y alpha a)
    from the dense matrix: an exact pin of the probing error (Eq. 16)."""
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, r, mode)
    cls = list(range(0, n, max(1, n // ncls)))[:ncls]
    q, st = qx.smp_qx(U, dims, KAPPA, _zolo(zolo4), colour, n, colours=cls, batch_colours=ncls)
    ref = qx.dense_smp_qx(g5dov4, colour)
    mask = np.isin(colour, cls)
    assert np.abs(q[mask] - ref[mask]).max() <= 1e-10
    assert np.abs(ref[mask].imag).max() > 1e-8  # SMP estimates are complex per site


def test_smp_full_charge_real(flux4, g5dov4):
    """Summed over all sites the imaginary parts cancel (Hermitian gamma_5 D_ov)."""
    colour, n = probing.color_sites(flux4["dims"], 2, 0)
    ref = qx.dense_smp_qx(g5dov4, colour)
    assert abs(ref.imag.sum()) <= 1e-12
    assert abs(ref.real.sum() - 1.0) < 0.5  # the probing bias of r_min = 2 on 4^4 is O(0.1)


def test_single_site_sets_are_point_sources():
    """Scheme with r = lattice extent: every set is one site (Sec. 2.1 vs 2.2)."""
    dims = (4, 4, 4, 8)
    colour, n = probing.color_sites(dims, dims, 0)
    assert n == int(np.prod(dims))
    assert np.array_equal(colour, np.arange(n))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_unit_links_q_vanishes(mode):
    """Free field: gamma_5 D_ov contains only 1 and gamma_mu structures, so
    tr_spin(gamma_5 ...) = 0 for every q(x) and q^SMP(x)."""
    dims = (4, 4, 4, 4)
    U = np.zeros((256, 4, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    c0, c, q, _ = zolotarev.zolotarev(NPOLES, 0.2, 7.5)
    colour, n = probing.color_sites(dims, 2, mode)
    out, st = qx.smp_qx(U, dims, KAPPA, (c0, c, q), colour, n, colours=[0, 1], batch_colours=2)
    assert np.abs(out).max() <= 1e-12
