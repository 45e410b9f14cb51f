"""Sanity of the seeded input generators (not the method)."""
import numpy as np

from synth import (apply_noise, flux_field, gauge_transform, haar_su3, make_config, site_coords,
                   site_index, stout_smooth)


def _su3_err(U):
    M = U.reshape(-1, 3, 3)
    un = np.abs(np.einsum("nab,ncb->nac", M, M.conj()) - np.eye(3)).max()
    det = np.abs(np.linalg.det(M) - 1).max()
    return un, det


def test_generators_are_su3():
    rng = np.random.default_rng(0)
    assert max(_su3_err(haar_su3(rng, 1000))) < 1e-13
    cfg = make_config("flux4")
    assert max(_su3_err(cfg["U"])) < 1e-13
    assert max(_su3_err(stout_smooth(cfg["U"], cfg["dims"], 0.1, 2))) < 1e-12


def _plaq(U, dims, mu, nu):
    xyzt = site_coords(dims)
    e = np.eye(4, dtype=np.int64)
    xm = site_index(xyzt + e[mu], dims)
    xn = site_index(xyzt + e[nu], dims)
    return np.einsum("sab,sbc,sdc,sed->sae", U[:, mu], U[xm, nu], U[xn, mu].conj(), U[:, nu].conj())


def test_flux_plaquettes_constant():
    dims = (4, 6, 4, 8)
    k = 2
    U = flux_field(dims, k)
    p12 = _plaq(U, dims, 0, 1)
    p34 = _plaq(U, dims, 2, 3)
    phi12 = 2 * np.pi * np.array([k, -k, 0]) / (4 * 6)
    phi34 = 2 * np.pi * np.array([1, 0, -1]) / (4 * 8)
    assert np.allclose(np.diagonal(p12, axis1=1, axis2=2), np.exp(1j * phi12)[None])
    assert np.allclose(np.diagonal(p34, axis1=1, axis2=2), np.exp(1j * phi34)[None])
    assert np.allclose(_plaq(U, dims, 0, 2), np.eye(3))


def test_gauge_transform_keeps_plaquette_trace():
    cfg = make_config("flux4x8", gauge=False)
    U, dims = cfg["U"], cfg["dims"]
    g = haar_su3(np.random.default_rng(4), U.shape[0])
    Ug = gauge_transform(U, g, dims)
    for mu, nu in [(0, 1), (1, 3), (2, 3)]:
        a = np.einsum("saa->s", _plaq(U, dims, mu, nu))
        b = np.einsum("saa->s", _plaq(Ug, dims, mu, nu))
        assert np.abs(a - b).max() < 1e-12


def test_seeded_reproducible():
    a = make_config("flux4")["U"]
    b = make_config("flux4")["U"]
    assert np.array_equal(a, b)
    rng = np.random.default_rng(1)
    n = apply_noise(flux_field((4, 4, 4, 4), 1), rng, 0.05)
    assert np.abs(n - flux_field((4, 4, 4, 4), 1)).max() < 0.5


def test_stout_c_matches_numpy():
    """The compiled stout smoothing (used for the large rough configurations)
    equals the numpy recipe and keeps the links in SU(3)."""
    from synth import gauge, native
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    U = gauge.haar_su3(np.random.default_rng(7), 4 * V).reshape(V, 4, 3, 3)
    a = gauge.stout_smooth(U, dims, 0.1, 3)
    b = native.stout(U, dims, 0.1, 3)
    assert np.abs(a - b).max() <= 1e-13
    uu = np.einsum("smab,smcb->smac", b, b.conj())
    assert np.abs(uu - np.eye(3)).max() <= 1e-13
    assert np.abs(np.linalg.det(b) - 1).max() <= 1e-13
    # smoothing raises the average plaquette of the rough Haar field
    def plaq(W):
        p = 0.0
        for mu in range(4):
            for nu in range(mu + 1, 4):
                P = np.einsum("sab,sbc,sdc,sed->sae", W[:, mu], gauge._roll(W[:, nu], dims, mu, +1),
                              gauge._roll(W[:, mu], dims, nu, +1).conj(), W[:, nu].conj())
                p += np.einsum("saa->s", P).real.mean() / 3
        return p / 6
    assert plaq(b) > plaq(U) + 0.1


def test_third_link_row_is_conj_cross_of_the_first_two():
    """SU(3) rows: row 2 = conj(row 0 x row 1), the identity behind storing two
    rows of every link (reconstruct-12) in the half-precision D_W."""
    for name in ("flux4", "flux4x8"):
        U = make_config(name)["U"]
        assert np.abs(np.conj(np.cross(U[..., 0, :], U[..., 1, :])) - U[..., 2, :]).max() < 1e-13
