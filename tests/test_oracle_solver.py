"""Pins of the oracle's shifted solves (Eqs. 6-8) and of the sign function it builds (Eqs. 3-4)."""
import numpy as np

from conftest import KAPPA
from oracle import dirac, msolve, native, spectrum
from synth import random_spinor


def _A(U, dims):
    V = int(np.prod(dims))
    return lambda v: dirac.apply_h2(U, v.reshape(V, 4, 3, -1), dims, KAPPA).reshape(12 * V, -1)


def test_multishift_equals_single_shift_cg(flux4, zolo4):
    """Every x_i of one multi-shift solve equals an independent CG on (A + q_i) x = b."""
    U, dims = flux4["U"], flux4["dims"]
    A = _A(U, dims)
    rng = np.random.default_rng(21)
    b = random_spinor(rng, 256, 2).reshape(3072, 2)
    q = zolo4["q"]
    xs, k, info = msolve.multishift_cg(A, b, q, 1e-13)
    assert info["converged"]
    for i in [0, 3, 7, 13]:
        xi, _ = msolve.cg(A, b, q[i], 1e-13)
        assert np.abs(xs[i] - xi).max() <= 1e-11 * np.abs(xi).max()
    tr = msolve.true_residuals(A, b, q, xs)
    assert tr.max() <= 1e-12


def test_c_multishift_matches_numpy(flux4, zolo4):
    U, dims = flux4["U"], flux4["dims"]
    rng = np.random.default_rng(22)
    b = random_spinor(rng, 256, 3)
    q = zolo4["q"]
    xa, ka, info = msolve.multishift_cg(_A(U, dims), b.reshape(3072, 3), q, 1e-12)
    xb, kb, res = native.multishift_cg(U, dims, KAPPA, b, q, 1e-12)
    assert abs(ka - kb) <= 1  # the stopping test may flip on rounding at the threshold
    assert np.abs(xa - xb.reshape(14, 3072, 3)).max() <= 1e-11
    assert info["resid"].max() <= 1e-12 and res.max() <= 1e-12


def _eps_apply(U, dims, zolo, v):
    """eps(H) v = H R(H^2) v through the solver path (Eq. 4)."""
    V = int(np.prod(dims))
    xs, k, res = native.multishift_cg(U, dims, KAPPA, v, zolo["q"], 1e-13)
    y = zolo["c0"] * v + np.einsum("i,i...->...", zolo["c"], xs)
    return dirac.apply_g5(native.apply_dw(U, y, dims, KAPPA)).reshape(V, 4, 3, -1)


def test_sign_function_against_dense(flux4, dense4, zolo4):
    """eps(H)v equals W diag(lam R(lam^2)) W^dag v, and sign(H) v within delta."""
    U, dims = flux4["U"], flux4["dims"]
    rng = np.random.default_rng(23)
    v = random_spinor(rng, 256, 2)
    got = _eps_apply(U, dims, zolo4, v).reshape(3072, 2)
    lam, W = dense4["lam"], dense4["W"]
    f = lam * (zolo4["c0"] + np.sum(zolo4["c"][None, :] / (lam[:, None] ** 2 + zolo4["q"][None, :]), axis=1))
    vv = v.reshape(3072, 2)
    ref = W @ (f[:, None] * (W.conj().T @ vv))
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    sgn = W @ (np.sign(lam)[:, None] * (W.conj().T @ vv))
    assert np.linalg.norm(got - sgn) <= (zolo4["delta"] + 1e-11) * np.linalg.norm(vv)
    # the rational on the spectrum is within delta of sign(lambda)
    assert np.abs(f - np.sign(lam)).max() <= zolo4["delta"] * (1 + 1e-6) + 1e-14


def test_eps_squared_is_one(flux4, zolo4):
    U, dims = flux4["U"], flux4["dims"]
    rng = np.random.default_rng(24)
    v = random_spinor(rng, 256, 1)
    e2 = _eps_apply(U, dims, zolo4, _eps_apply(U, dims, zolo4, v))
    assert np.linalg.norm(e2 - v) <= (2 * zolo4["delta"] + 1e-10) * np.linalg.norm(v)


def test_ginsparg_wilson(g5dov4, dense4, zolo4):
    """D = 1 + g5 eps: D + D^dag = D^dag D up to O(delta)."""
    D = dense4["g5"] @ g5dov4
    lhs = D + D.conj().T
    rhs = D.conj().T @ D
    assert np.abs(lhs - rhs).max() <= 4 * zolo4["delta"] + 1e-12


def test_spectrum_eigsh_matches_dense(flux4, dense4):
    U, dims = flux4["U"], flux4["dims"]
    lmin, lmax = spectrum.h2_extremes(U, dims, KAPPA)
    l2 = dense4["lam"] ** 2
    assert abs(lmin - l2.min()) <= 1e-8 * l2.max()
    assert abs(lmax - l2.max()) <= 1e-8 * l2.max()
