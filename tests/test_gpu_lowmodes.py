"""GPU parity of the low-mode projection (the lowest eigenmodes of H_W treated
exactly in eps(H_W), Eq. 4) against the FP64 oracle (oracle/lowmodes.py).

Tolerances: eigenvalues 1e-9, projector onto the low space 1e-8 (the GPU
eigen-solver stops at ||H v - lambda v|| <= 1e-11); q(x) within 1e-8 per site
as for the unprojected path.
"""
import json
import os

import numpy as np
import pytest

from conftest import KAPPA, NPOLES
from oracle import lowmodes, probing, qx, zolotarev
from synth import make_config, random_spinor

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "spectra.json")
K4 = 8    # 4^4 flux: |lambda|^2 jumps from 0.0225 to 0.0434 after the 8th mode
K8 = 20   # 8^3 x 16 flux: from 0.0327 to 0.0403 after the 20th


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02211_gb300 import smpq
    smpq.load()
    return smpq


def _lmax2(name):
    with open(GOLD) as f:
        return json.load(f)[name]["lmax2"]


@pytest.fixture(scope="module")
def dense_modes4(flux4):
    lam, W = lowmodes.low_modes_dense(flux4["U"], flux4["dims"], KAPPA, K4)
    a, b = 0.98 * lam[K4] ** 2, 1.02 * _lmax2("flux4")
    c0, c, q, _ = zolotarev.zolotarev(NPOLES, a, b)
    return dict(lam=lam, W=W, a=a, b=b, zolo=(c0, c, q))


def _gpu_modes(S, s, k, full_interval):
    s.set_spectrum(*full_interval)
    ev, res, it = s.low_modes(k, tol=1e-11)
    return ev, res, it


def test_low_modes_4x4_vs_dense(S, flux4, dense_modes4, zolo4):
    from paper_1901_02211_gb300 import Session
    U, dims = flux4["U"], flux4["dims"]
    with Session(precision=S.SMPQ_FP64) as s:
        s.load_gauge(dims, U)
        ev, res, it = _gpu_modes(S, s, K4, (zolo4["a"], zolo4["b"]))
        lam_g, vec = s.get_low_modes()
    print("4^4 low modes: %d filter steps, max residual %.2e" % (it, res.max()))
    assert res.max() <= 1e-11
    assert np.abs(ev - dense_modes4["lam"]).max() <= 1e-9
    Vg = vec.reshape(-1, K4)
    assert np.abs(Vg.conj().T @ Vg - np.eye(K4)).max() <= 1e-12
    W = dense_modes4["W"][:, :K4]
    assert np.abs(Vg @ Vg.conj().T - W @ W.conj().T).max() <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("r,mode", [(2, 0), (2, 1)])
def test_projected_qx_4x4_vs_dense(S, flux4, dense_modes4, zolo4, prec, r, mode):
    """q^SMP(x) with the 8 lowest modes exact against the dense matrix
    gamma_5 + W diag(f) W^dag (f = sign on the low modes, lambda R(lambda^2)
    with the shortened interval elsewhere); the solves need fewer iterations
    than with the whole spectrum."""
    from paper_1901_02211_gb300 import Session
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, r, mode)
    ref = qx.dense_smp_qx(lowmodes.dense_g5dov_projected(U, dims, KAPPA, dense_modes4["zolo"], K4), colour)
    precision = S.SMPQ_FP64 if prec == "fp64" else S.SMPQ_MIXED
    with Session(precision=precision) as s:
        s.load_gauge(dims, U)
        s.build_sources(r, mode)
        s.set_spectrum(zolo4["a"], zolo4["b"])
        _, _, st_full = s.compute_qx()
        _gpu_modes(S, s, K4, (zolo4["a"], zolo4["b"]))
        s.set_spectrum(dense_modes4["a"], dense_modes4["b"])
        q, Q, st = s.compute_qx()
    err = np.abs(q - ref).max()
    print("4^4 r=%d mode %d %s projected: max |dq| = %.2e, iterations %d (whole spectrum: %d)" % (
        r, mode, prec, err, st["max_iterations"], st_full["max_iterations"]))
    assert err <= 1e-8
    assert abs(Q - ref.real.sum()) <= 1e-9
    assert st["max_iterations"] < st_full["max_iterations"]


def test_projected_apply_dov_4x4(S, flux4, dense_modes4, zolo4):
    """D_ov v = gamma_5 (gamma_5 + eps_proj(H)) v on random fields."""
    from paper_1901_02211_gb300 import Session
    U, dims = flux4["U"], flux4["dims"]
    M = lowmodes.dense_g5dov_projected(U, dims, KAPPA, dense_modes4["zolo"], K4)
    V = 256
    g5 = np.kron(np.eye(V), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    psi = random_spinor(np.random.default_rng(71), V, 3)
    with Session(precision=S.SMPQ_FP64) as s:
        s.load_gauge(dims, U)
        _gpu_modes(S, s, K4, (zolo4["a"], zolo4["b"]))
        s.set_spectrum(dense_modes4["a"], dense_modes4["b"])
        out = s.apply_dov(psi)
        s.clear_low_modes()
        assert s.get_low_modes()[0].size == 0
    ref = (g5 @ M) @ psi.reshape(12 * V, 3)
    assert np.abs(out.reshape(12 * V, 3) - ref).max() <= 1e-9


def test_projected_qx_8x16_sampled(S):
    """8^3 x 16 flux, the 20 lowest modes (ARPACK in the oracle, the filtered
    subspace iteration on the GPU), SMP r = 4 on sampled classes."""
    from paper_1901_02211_gb300 import Session
    cfg = make_config("flux8x16")
    U, dims = cfg["U"], cfg["dims"]
    lam, W = lowmodes.low_modes(U, dims, KAPPA, K8, tol=1e-12)
    lmax2 = _lmax2("flux8x16")
    a, b = 0.98 * lam[K8] ** 2, 1.02 * lmax2
    c0, c, q, _ = zolotarev.zolotarev(NPOLES, a, b)
    colour, n = probing.color_sites(dims, 4, 0)
    classes = [0, 77]
    ref, _ = lowmodes.smp_qx_projected(U, dims, KAPPA, (c0, c, q), colour, n, (lam[:K8], W[:, :K8]),
                                       colours=classes, batch_colours=2)
    with Session(precision=S.SMPQ_MIXED) as s:
        s.load_gauge(dims, U)
        s.build_sources(4, 0)
        ev, res, it = _gpu_modes(S, s, K8, (0.98 * 0.0252, 1.02 * lmax2))
        s.set_spectrum(a, b)
        qg, Q, st = s.compute_qx(classes=classes)
    mask = np.isin(colour, classes)
    err = np.abs(qg[mask] - ref[mask]).max()
    print("8^3x16 low modes: %d filter steps, |dlambda| %.2e; projected q max |dq| = %.2e, iterations %d" % (
        it, np.abs(ev - lam).max(), err, st["max_iterations"]))
    assert np.abs(ev - lam).max() <= 1e-9
    assert err <= 1e-8


def test_low_modes_errors(S, flux4, zolo4):
    """Out-of-order and invalid requests return status codes, not faults."""
    from paper_1901_02211_gb300 import Session
    U, dims = flux4["U"], flux4["dims"]
    with Session(precision=S.SMPQ_FP64) as s:
        s.load_gauge(dims, U)
        with pytest.raises(S.SmpqError) as e:
            s.low_modes(4)  # no spectral interval yet
        assert e.value.code == S.SMPQ_ESTATE
        s.set_spectrum(zolo4["a"], zolo4["b"])
        for k, block in ((0, 0), (44, 0), (4, 20), (4, 60)):
            with pytest.raises(S.SmpqError) as e:
                s.low_modes(k, block=block)
            assert e.value.code == S.SMPQ_EINVAL
        assert s.get_low_modes()[0].size == 0
        ev, res, it = s.low_modes(4, block=12, tol=1e-10)
        assert ev.size == 5 and res.max() <= 1e-10
        s.load_gauge(dims, U)  # a new gauge field drops the modes
        assert s.get_low_modes()[0].size == 0
