"""Symmetric multi-probing colouring and sources (Sec. 2.2; Eqs. 15, 18-19; Tables 1-2).

Scheme P(m_x, m_y, m_z, m_t, mode) on L(n_x, n_y, n_z, n_t): m_mu sites of one
colour along direction mu, i.e. same-colour sites every r_mu = n_mu / m_mu sites.

  mode 0 (Normal):  colour(x) = (x_mu mod r_mu)_mu; prod(r_mu) colours, m_x m_y m_z m_t
                    sites per set, r_min = r.
  mode 1 (Split):   each Normal set is split like a checkerboard on its own coarse
                    lattice, colour = (Normal colour, sum_mu floor(x_mu / r_mu) mod 2);
                    2 prod(r_mu) colours of half the size, r_min = sqrt(2) r.  The
                    checkerboard only closes around the torus when every m_mu is even.
  mode 2 (Combine): a Normal set is merged with its translate by (r/2, r/2, r/2, r/2);
                    prod(r_mu)/2 colours of twice the size, r_min = r; r_mu even.

Colour numbering (the paper leaves it free; it only fixes the summation order):
  mode 0: c = sum_mu b_mu prod_{nu<mu} r_nu with b_mu = x_mu mod r_mu (x fastest);
  mode 1: c = 2 * c_mode0 + parity;
  mode 2: with h_mu = r_mu / 2, e_mu = b_mu mod h_mu and d_mu = floor(b_mu / h_mu),
          the pair {d, 1 - d} is represented by the member with d_x = 0:
          c = 8 * (sum_mu e_mu prod_{nu<mu} h_nu) + (d_y + 2 d_z + 4 d_t) after that flip.
"""
from __future__ import annotations

import itertools

import numpy as np

from synth.gauge import site_coords


def _rvec(dims, r):
    rv = np.array([r] * 4 if np.isscalar(r) else list(r), dtype=np.int64)
    return rv


def validate(dims, r, mode):
    """Raise ValueError when scheme (r, mode) does not tile the lattice."""
    rv = _rvec(dims, r)
    dims = np.asarray(dims)
    if mode not in (0, 1, 2):
        raise ValueError("mode must be 0, 1 or 2")
    if np.any(rv < 1) or np.any(dims % rv != 0):
        raise ValueError("r must divide every lattice extent")
    if mode == 1 and np.any((dims // rv) % 2 != 0):
        raise ValueError("split mode needs an even number of same-colour sites per direction")
    if mode == 2 and np.any(rv % 2 != 0):
        raise ValueError("combine mode needs even r")
    return rv


def color_sites(dims, r, mode):
    """Return (colour[V] int64, n_colours)."""
    rv = validate(dims, r, mode)
    xyzt = site_coords(dims)
    b = xyzt % rv[None, :]
    stride = np.array([1, rv[0], rv[0] * rv[1], rv[0] * rv[1] * rv[2]])
    if mode == 0:
        return (b * stride[None]).sum(1), int(np.prod(rv))
    if mode == 1:
        c0 = (b * stride[None]).sum(1)
        par = (xyzt // rv[None, :]).sum(1) % 2
        return 2 * c0 + par, int(2 * np.prod(rv))
    h = rv // 2
    e = b % h[None, :]
    d = b // h[None, :]
    d = np.where(d[:, :1] == 1, 1 - d, d)
    hstride = np.array([1, h[0], h[0] * h[1], h[0] * h[1] * h[2]])
    return 8 * (e * hstride[None]).sum(1) + d[:, 1] + 2 * d[:, 2] + 4 * d[:, 3], int(np.prod(rv)) // 2


def n_smp_sources(dims, m, mode):
    """N^SMP = 12 N_p for symmetric scheme (m, mode) (Table 2)."""
    r = np.asarray(dims) // np.asarray([m] * 4 if np.isscalar(m) else m)
    _, n = color_sites(tuple(dims), tuple(int(v) for v in r), mode)
    return 12 * n


def _min_image_d2(dims, a, b):
    dims = np.asarray(dims)
    d = np.abs(a - b)
    d = np.minimum(d, dims - d)
    return (d * d).sum(-1)


def r_min_bruteforce(dims, colour, all_pairs=False):
    """Smallest minimum-image Euclidean distance between two sites of one colour (Eq. 18).

    Brute force: from the first member of every colour to every other member of
    that colour (all_pairs=True: over every pair).  Returns (r_min, neighbours)
    with `neighbours` the number of same-colour sites at distance r_min from
    site 0.
    """
    xyzt = site_coords(dims)
    best = np.inf
    order = np.argsort(colour, kind="stable")
    cs = colour[order]
    bounds = np.flatnonzero(np.diff(cs)) + 1
    for grp in np.split(order, bounds):
        pts = xyzt[grp]
        if len(pts) < 2:
            continue
        if all_pairs:
            d2 = _min_image_d2(dims, pts[:, None, :], pts[None, :, :])
            d2[np.arange(len(pts)), np.arange(len(pts))] = 1 << 60
        else:
            d2 = _min_image_d2(dims, pts[:1], pts[1:])
        best = min(best, d2.min())
    pts = xyzt[colour == colour[0]]
    d2 = _min_image_d2(dims, pts[0][None], pts)
    return float(np.sqrt(best)), int(np.sum(d2 == best))


def smp_sources(colour, classes):
    """SMP sources of Eq. 15 for the listed colours: b[V, 4, 3, 12*len(classes)].

    Column 12*j + 3*alpha + a is sum_{y in S_j} psi(y, alpha, a).
    """
    V = colour.shape[0]
    classes = list(classes)
    b = np.zeros((V, 4, 3, 12 * len(classes)), dtype=np.complex128)
    for j, c in enumerate(classes):
        sites = np.nonzero(colour == c)[0]
        for alpha, a in itertools.product(range(4), range(3)):
            b[sites, alpha, a, 12 * j + 3 * alpha + a] = 1.0
    return b
