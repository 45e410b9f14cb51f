"""Pins of the Zolotarev rational sign function (Eq. 4)."""
import numpy as np
import pytest

from oracle import zolotarev


def _alternation(n, a, b, npts=200001):
    """Extrema of e(x) = 1 - sqrt(x) R(x) between consecutive sign changes."""
    c0, c, q, delta = zolotarev.zolotarev(n, a, b)
    x = np.exp(np.linspace(np.log(a), np.log(b), npts))
    e = 1 - np.sqrt(x) * zolotarev.rational(x, c0, c, q)
    sgn = np.sign(e)
    cuts = np.flatnonzero(sgn[1:] != sgn[:-1]) + 1
    segs = np.split(e, cuts)
    ext = np.array([s[np.argmax(np.abs(s))] for s in segs])
    return ext, delta, e


@pytest.mark.parametrize("n,a,b", [(6, 0.1, 7.0), (8, 0.02, 7.5), (10, 1e-3, 8.0), (14, 1e-4, 10.0)])
def test_equioscillation(n, a, b):
    """Chebyshev alternation: 2n+2 extrema of equal |e| = delta with alternating
    sign characterise the type-(n, n) best relative approximation."""
    ext, delta, e = _alternation(n, a, b)
    assert len(ext) == 2 * n + 2
    assert np.all(np.sign(ext[1:]) != np.sign(ext[:-1]))
    assert np.allclose(np.abs(ext), delta, rtol=1e-4)
    assert np.abs(e).max() <= delta * (1 + 1e-6) + 1e-13  # + evaluation rounding


@pytest.mark.parametrize("n,a,b", [(14, 0.02, 7.0), (14, 1e-3, 8.0), (6, 0.5, 2.0)])
def test_coefficients_positive_and_sorted(n, a, b):
    c0, c, q, delta = zolotarev.zolotarev(n, a, b)
    assert c0 > 0 and np.all(c > 0) and np.all(q > 0)
    assert np.all(np.diff(q) > 0)
    assert len(c) == n and len(q) == n


def test_error_decreases_with_poles():
    ds = [zolotarev.zolotarev(n, 1e-3, 1.0)[3] for n in range(4, 15)]
    assert np.all(np.diff(np.log(ds)) < -0.5)


def test_scale_invariance():
    """R for [s a, s b] equals R for [a, b] evaluated at x/s, divided by sqrt(s)."""
    a, b, s = 0.03, 6.0, 3.7
    c0, c, q, _ = zolotarev.zolotarev(14, a, b)
    C0, C, Q, _ = zolotarev.zolotarev(14, s * a, s * b)
    x = np.linspace(s * a, s * b, 101)
    assert np.allclose(zolotarev.rational(x, C0, C, Q), zolotarev.rational(x / s, c0, c, q) / np.sqrt(s),
                       rtol=1e-12)
