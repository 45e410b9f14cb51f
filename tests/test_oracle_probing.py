"""Pins of the symmetric colouring (Sec. 2.2, Eqs. 18-19) against Tables 1 and 2."""
import math
import os

import numpy as np
import pytest

from oracle import probing

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("row", _rows(), ids=lambda r: "%d^4-(%d,%d)" % r[:3])
def test_table2_counts(row):
    """N^SMP and N^SMP / N^PT of Table 2; set sizes of Sec. 2.2."""
    n, m, mode, ra, rs, nsmp, den = row
    dims = (n, n, n, n)
    assert probing.n_smp_sources(dims, m, mode) == nsmp
    assert nsmp * den == 12 * n ** 4
    colour, ncls = probing.color_sites(dims, n // m, mode)
    sizes = np.bincount(colour, minlength=ncls)
    expect = {0: m ** 4, 1: m ** 4 // 2, 2: 2 * m ** 4}[mode]
    assert np.all(sizes == expect)


@pytest.mark.parametrize("row", [r for r in _rows() if r[0] <= 16], ids=lambda r: "%d^4-(%d,%d)" % r[:3])
def test_table1_rmin(row):
    """r_min of Table 1 by brute force over same-colour sites (Eq. 18)."""
    n, m, mode, ra, rs, nsmp, den = row
    dims = (n, n, n, n)
    colour, ncls = probing.color_sites(dims, n // m, mode)
    rmin, nn = probing.r_min_bruteforce(dims, colour, all_pairs=(n <= 12 and m <= 6))
    assert rmin == pytest.approx(ra * math.sqrt(2) ** rs, rel=1e-12)


@pytest.mark.parametrize("mode,expect", [(0, 8), (1, 24), (2, 24)])
def test_nearest_neighbour_counts(mode, expect):
    """8 nearest same-colour neighbours in Normal mode, 24 in Split mode (Sec. 3);
    Combine mode: 8 axial + 16 diagonal (r/2,r/2,r/2,r/2) offsets."""
    dims = (16, 16, 16, 16)
    colour, n = probing.color_sites(dims, 4, mode)
    _, nn = probing.r_min_bruteforce(dims, colour)
    assert nn == expect


def test_rmin_formula_non_cubic():
    """Eq. 19 on L(n_s, n_s, n_s, n_t): r_min = r (modes 0, 2), sqrt(2) r (mode 1)."""
    dims = (8, 8, 8, 16)
    for r, mode, want in [(2, 0, 2), (4, 0, 4), (2, 1, 2 * math.sqrt(2)), (4, 2, 4), (2, 2, 2)]:
        colour, n = probing.color_sites(dims, r, mode)
        assert probing.r_min_bruteforce(dims, colour)[0] == pytest.approx(want)


def test_partition_and_validation():
    dims = (8, 8, 8, 16)
    for r, mode in [(2, 0), (4, 0), (2, 1), (2, 2), (4, 2), (8, 0)]:
        colour, n = probing.color_sites(dims, r, mode)
        assert colour.min() == 0 and colour.max() == n - 1
        assert len(np.unique(colour)) == n  # every colour used, each site exactly one colour
    with pytest.raises(ValueError):
        probing.color_sites(dims, 3, 0)  # r must divide n_mu (Eq. 19 remark)
    with pytest.raises(ValueError):
        probing.color_sites(dims, 8, 1)  # m_x = 1 cannot be checkerboarded
    with pytest.raises(ValueError):
        probing.color_sites((6, 6, 6, 6), 3, 2)  # combine mode needs even r
    with pytest.raises(ValueError):
        probing.color_sites(dims, 2, 3)


def test_sources_sum_point_sources():
    dims = (4, 4, 4, 4)
    colour, n = probing.color_sites(dims, 2, 0)
    b = probing.smp_sources(colour, [3])
    assert b.shape == (256, 4, 3, 12)
    assert np.all(b.sum(axis=(1, 2)) == (colour == 3)[:, None])
    for col in range(12):
        alpha, a = divmod(col, 3)
        assert np.all(b[:, alpha, a, col] == (colour == 3))
