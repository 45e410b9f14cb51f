"""Pins of the oracle's SMP trace of D_W^{-1} against the dense inverse on 4^4."""
import numpy as np
import pytest

from conftest import KAPPA
from oracle import probing, qx


@pytest.fixture(scope="module")
def dwinv(dense4):
    return np.linalg.inv(dense4["Dw"])


@pytest.mark.parametrize("r,mode,ncls", [(4, 0, 3), (2, 0, 2), (2, 1, 2)])
def test_trace_dwinv_vs_dense(flux4, dwinv, r, mode, ncls):
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, r, mode)
    cls = list(range(ncls))
    t, st = qx.smp_trace_dwinv(U, dims, KAPPA, colour, n, colours=cls, batch_colours=ncls)
    ref = qx.dense_smp_trace(dwinv, colour)
    mask = np.isin(colour, cls)
    assert np.abs(t[mask] - ref[mask]).max() <= 1e-10


def test_trace_dwinv_is_real(dwinv):
    """gamma_5-hermiticity: tr D_W^{-1} = conj(tr D_W^{-1})."""
    assert abs(np.trace(dwinv).imag) <= 1e-10 * abs(np.trace(dwinv))
