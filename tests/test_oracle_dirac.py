"""Pins of the oracle's Wilson kernel (Sec. 2.1, around Eq. 3; Eq. 4)."""
import itertools

import numpy as np
import pytest

from conftest import KAPPA
from oracle import dirac, native
from synth import gauge_transform, haar_su3, make_config, random_spinor, site_coords


def _ip(a, b):
    return np.vdot(a.ravel(), b.ravel())


def test_gamma_algebra():
    G = dirac.GAMMA
    for mu, nu in itertools.product(range(4), range(4)):
        ac = G[mu] @ G[nu] + G[nu] @ G[mu]
        assert np.allclose(ac, 2 * (mu == nu) * np.eye(4))
        assert np.allclose(G[mu], G[mu].conj().T)
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_gamma5_hermiticity(flux4, bc, impl):
    """<chi, g5 D_W g5 psi> = <D_W chi, psi>  (D_W^dag = g5 D_W g5, used in Eq. 4)."""
    U, dims = flux4["U"], flux4["dims"]
    rng = np.random.default_rng(7)
    chi, psi = random_spinor(rng, 256), random_spinor(rng, 256)
    dw = dirac.apply_dw if impl == "numpy" else native.apply_dw
    lhs = _ip(chi, dirac.apply_g5(dw(U, dirac.apply_g5(psi), dims, KAPPA, bc)))
    rhs = _ip(dw(U, chi, dims, KAPPA, bc), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_free_field_plane_wave(bc, impl):
    """U = 1: D_W e^{ipx} u = (1 - 2k sum cos p + 2ik sum gamma_mu sin p) e^{ipx} u."""
    dims = (4, 4, 6, 8)
    V = int(np.prod(dims))
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    xyzt = site_coords(dims)
    rng = np.random.default_rng(3)
    dw = dirac.apply_dw if impl == "numpy" else native.apply_dw
    for trial in range(3):
        n = rng.integers(0, 8, size=4)
        p = np.array([(2 * n[mu] + (0 if bc[mu] == 1 else 1)) * np.pi / dims[mu] for mu in range(4)])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (xyzt @ p))
        psi = phase[:, None, None] * u[None]
        M = (1 - 2 * KAPPA * np.cos(p).sum()) * np.eye(4) + 2j * KAPPA * sum(
            dirac.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (M @ u)[None]
        got = dw(U, psi, dims, KAPPA, bc)
        assert np.abs(got - expect).max() <= 1e-13


@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_gauge_covariance(impl):
    """D_W[U^g] (g psi) = g D_W[U] psi, U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    cfg = make_config("flux4x8", gauge=False)
    U, dims = cfg["U"], cfg["dims"]
    V = int(np.prod(dims))
    rng = np.random.default_rng(11)
    g = haar_su3(rng, V)
    Ug = gauge_transform(U, g, dims)
    psi = random_spinor(rng, V)
    gpsi = np.einsum("sab,sib->sia", g, psi)
    dw = dirac.apply_dw if impl == "numpy" else native.apply_dw
    lhs = dw(Ug, gpsi, dims, KAPPA)
    rhs = np.einsum("sab,sib->sia", g, dw(U, psi, dims, KAPPA))
    assert np.abs(lhs - rhs).max() <= 1e-13


def test_c_matches_numpy_batched(flux4):
    U, dims = flux4["U"], flux4["dims"]
    rng = np.random.default_rng(5)
    psi = random_spinor(rng, 256, 7)
    for bc in [(1, 1, 1, 1), (-1, 1, 1, -1)]:
        a = dirac.apply_dw(U, psi, dims, KAPPA, bc)
        b = native.apply_dw(U, psi, dims, KAPPA, bc)
        assert np.abs(a - b).max() <= 1e-13
        a = dirac.apply_h2(U, psi, dims, KAPPA, bc)
        b = native.apply_h2(U, psi, dims, KAPPA, bc)
        assert np.abs(a - b).max() <= 1e-12


def test_dense_matches_operator(flux4, dense4):
    U, dims = flux4["U"], flux4["dims"]
    rng = np.random.default_rng(2)
    psi = random_spinor(rng, 256)
    got = (dense4["Dw"] @ psi.reshape(-1)).reshape(256, 4, 3)
    assert np.abs(got - dirac.apply_dw(U, psi, dims, KAPPA)).max() <= 1e-13
    H = dense4["H"]
    assert np.abs(H - H.conj().T).max() <= 1e-14
