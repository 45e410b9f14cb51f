"""Seeded gauge-field and spinor generators (inputs only).

Conventions shared with every consumer:
  * lattice dims = (nx, ny, nz, nt); site index s = x + nx*(y + ny*(z + nz*t)),
    x fastest;
  * a gauge field is a complex128 array U[V, 4, 3, 3] with U[s, mu] the SU(3)
    link from s to s + mu_hat (mu = 0..3 for x, y, z, t), row-major colour
    indices;
  * a spinor is complex128 psi[V, 4, 3] (site, spin, colour), optionally with a
    trailing right-hand-side axis psi[V, 4, 3, B].

The paper measures on Iwasaki pure-gauge ensembles (Sec. 3, Table 1) that are not
available here; the configurations below stand in for them.  Their recipes:

  * quantised-flux background: for colour c with integer fluxes (n12_c, n34_c),
    constant U(1) field strength 2*pi*n12_c/(nx*ny) in the x-y plane and
    2*pi*n34_c/(nz*nt) in the z-t plane, with the twist on the last row so
    every plaquette of the plane carries the same phase.  The colour-traceless
    choice (k, 1), (-k, 0), (0, -1) keeps det U = 1 exactly and has a
    continuum index sum_c n12_c n34_c = k;
  * noise: U <- exp(i eps H) U with H = sum_a xi_a lambda_a (Gell-Mann matrices),
    xi_a ~ N(0, 1), exponentiated exactly through the eigen-decomposition of H;
  * random gauge transform: g(x) Haar-distributed in SU(3) (QR of a complex
    Ginibre matrix with the phase fix of Mezzadri 2007, then det^(1/3) removed),
    U_mu(x) <- g(x) U_mu(x) g(x + mu_hat)^dagger;
  * stout-style smoothing (Morningstar-Peardon step, rho, simultaneous update).
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------- lattice bookkeeping


def site_coords(dims):
    """Return int64 array [V, 4] of (x, y, z, t) for every site index."""
    nx, ny, nz, nt = dims
    s = np.arange(nx * ny * nz * nt, dtype=np.int64)
    x = s % nx
    y = (s // nx) % ny
    z = (s // (nx * ny)) % nz
    t = s // (nx * ny * nz)
    return np.stack([x, y, z, t], axis=1)


def site_index(coords, dims):
    """Site index of (x, y, z, t) with periodic wrap."""
    nx, ny, nz, nt = dims
    c = np.asarray(coords, dtype=np.int64)
    x = c[..., 0] % nx
    y = c[..., 1] % ny
    z = c[..., 2] % nz
    t = c[..., 3] % nt
    return x + nx * (y + ny * (z + nz * t))


def _roll(field, dims, mu, step):
    """field(x + step*mu_hat) for a field with a leading site axis (periodic)."""
    nx, ny, nz, nt = dims
    shp = field.shape
    f = field.reshape((nt, nz, ny, nx) + shp[1:])
    axis = 3 - mu
    return np.roll(f, -step, axis=axis).reshape(shp)


# ----------------------------------------------------------------------------- SU(3) helpers

_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1] = -1j
_GELL_MANN[1][1, 0] = 1j
_GELL_MANN[2][0, 0] = 1
_GELL_MANN[2][1, 1] = -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2] = -1j
_GELL_MANN[4][2, 0] = 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2] = -1j
_GELL_MANN[6][2, 1] = 1j
_GELL_MANN[7][0, 0] = _GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
_GELL_MANN[7][2, 2] = -2 / np.sqrt(3)


def _expi_hermitian(h):
    """exp(i h) for a stack of Hermitian 3x3 matrices, via eigh (exact up to rounding)."""
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), v.conj())


def su3_noise(rng, n, eps):
    """n matrices exp(i eps sum_a xi_a lambda_a) with xi_a ~ N(0, 1)."""
    xi = rng.standard_normal((n, 8))
    h = np.einsum("na,aij->nij", xi, _GELL_MANN)
    return _expi_hermitian(eps * h)


def haar_su3(rng, n):
    """n Haar-random SU(3) matrices (Mezzadri's QR recipe, then det^(1/3) removed)."""
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


# ----------------------------------------------------------------------------- gauge fields


def flux_field(dims, k):
    """Quantised-flux U(1)^2-in-SU(3) field with colour fluxes (k,1), (-k,0), (0,-1).

    Returns U[V, 4, 3, 3] (diagonal links, det = 1 exactly in exact arithmetic).
    """
    nx, ny, nz, nt = dims
    V = nx * ny * nz * nt
    n12 = np.array([k, -k, 0], dtype=np.float64)
    n34 = np.array([1, 0, -1], dtype=np.float64)
    xyzt = site_coords(dims)
    x, y, z, t = (xyzt[:, i].astype(np.float64) for i in range(4))
    phi12 = 2 * np.pi * n12 / (nx * ny)
    phi34 = 2 * np.pi * n34 / (nz * nt)
    ph = np.zeros((V, 4, 3))
    ph[:, 0, :] = -phi12[None, :] * y[:, None]
    ph[:, 1, :] = np.where((xyzt[:, 1] == ny - 1)[:, None], phi12[None, :] * ny * x[:, None], 0.0)
    ph[:, 2, :] = -phi34[None, :] * t[:, None]
    ph[:, 3, :] = np.where((xyzt[:, 3] == nt - 1)[:, None], phi34[None, :] * nt * z[:, None], 0.0)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    for c in range(3):
        U[:, :, c, c] = np.exp(1j * ph[:, :, c])
    return U


def apply_noise(U, rng, eps):
    """U <- exp(i eps H) U on every link."""
    V = U.shape[0]
    n = su3_noise(rng, V * 4, eps).reshape(V, 4, 3, 3)
    return np.einsum("smab,smbc->smac", n, U)


def random_gauge(rng, V):
    return haar_su3(rng, V)


def gauge_transform(U, g, dims):
    """U_mu(x) -> g(x) U_mu(x) g(x + mu_hat)^dagger."""
    out = np.empty_like(U)
    for mu in range(4):
        gf = _roll(g, dims, mu, +1)
        out[:, mu] = np.einsum("sab,sbc,sdc->sad", g, U[:, mu], gf.conj())
    return out


def stout_smooth(U, dims, rho, steps):
    """`steps` stout-style smoothing steps with parameter rho, all links at once."""
    for _ in range(steps):
        C = np.zeros_like(U)
        for mu in range(4):
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = U[:, nu]
                Umu_xnu = _roll(U[:, mu], dims, nu, +1)
                Unu_xmu = _roll(U[:, nu], dims, mu, +1)
                up = np.einsum("sab,sbc,sdc->sad", Unu, Umu_xnu, Unu_xmu.conj())
                Unu_m = _roll(U[:, nu], dims, nu, -1)
                Umu_m = _roll(U[:, mu], dims, nu, -1)
                Unu_mpm = _roll(_roll(U[:, nu], dims, nu, -1), dims, mu, +1)
                dn = np.einsum("sba,sbc,scd->sad", Unu_m.conj(), Umu_m, Unu_mpm)
                C[:, mu] += rho * (up + dn)
        Om = np.einsum("smab,smcb->smac", C, U.conj())
        A = Om.conj().transpose(0, 1, 3, 2) - Om
        tr = np.einsum("smaa->sm", A)
        Qm = 0.5j * A - (1j / 6.0) * tr[:, :, None, None] * np.eye(3)
        U = np.einsum("smab,smbc->smac", _expi_hermitian(Qm), U)
    return U


def random_spinor(rng, V, nrhs=None):
    shape = (V, 4, 3) if nrhs is None else (V, 4, 3, nrhs)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


# ----------------------------------------------------------------------------- named workloads

# Seeded synthetic configurations shaped like the paper's lattices (Sec. 3, Table 1).
CONFIGS = {
    "flux4": dict(dims=(4, 4, 4, 4), k=1, eps=0.05, seed_noise=1002, seed_gauge=1001),
    "flux8x16": dict(dims=(8, 8, 8, 16), k=2, eps=0.10, seed_noise=2002, seed_gauge=2001),
    "flux16x32": dict(dims=(16, 16, 16, 32), k=-1, eps=0.15, seed_noise=3002, seed_gauge=3001),
    "flux12x24": dict(dims=(12, 12, 12, 24), k=2, eps=0.10, seed_noise=4004, seed_gauge=4003),
    "flux8x16_b": dict(dims=(8, 8, 8, 16), k=1, eps=0.10, seed_noise=4002, seed_gauge=4001),
    "flux16x32_b": dict(dims=(16, 16, 16, 32), k=3, eps=0.10, seed_noise=4006, seed_gauge=4005),
    # small variants used by the fast tests
    "flux4_k0": dict(dims=(4, 4, 4, 4), k=0, eps=0.05, seed_noise=1012, seed_gauge=1011),
    "flux4x8": dict(dims=(4, 4, 4, 8), k=1, eps=0.05, seed_noise=1022, seed_gauge=1021),
    # seeded Haar-random links smoothed by 20 stout steps (rho = 0.1): a rough
    # background with no closed-form charge, the largest lattice of the set
    "stout32x64": dict(dims=(32, 32, 32, 64), stout=(0.1, 20), seed=5001),
    "stout8x16": dict(dims=(8, 8, 8, 16), stout=(0.1, 20), seed=5011),
}


def make_config(name, gauge=True):
    """Build a named synthetic configuration.

    Returns dict(dims, U, Q_closed, name).  `gauge=False` skips the random gauge
    transform (useful for gauge-covariance tests).
    """
    p = CONFIGS[name]
    dims = tuple(p["dims"])
    V = int(np.prod(dims))
    if "stout" in p:
        from . import native
        rho, steps = p["stout"]
        U = haar_su3(np.random.default_rng(p["seed"]), 4 * V).reshape(V, 4, 3, 3)
        return dict(dims=dims, U=native.stout(U, dims, rho, steps), Q_closed=None, name=name)
    U = flux_field(dims, p["k"])
    U = apply_noise(U, np.random.default_rng(p["seed_noise"]), p["eps"])
    if gauge:
        g = random_gauge(np.random.default_rng(p["seed_gauge"]), V)
        U = gauge_transform(U, g, dims)
    return dict(dims=dims, U=U, Q_closed=p["k"], name=name)
