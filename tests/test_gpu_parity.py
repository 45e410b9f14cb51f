"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: q(x) within 1e-8 absolute per site and Q within 1e-9 for the FP64
path (the solver stops at relative residual 1e-10; the oracle at 1e-13);
D_W within 1e-13 (FP64) / 2e-6 relative (FP32 kernel).
"""
import json
import os

import numpy as np
import pytest

from conftest import KAPPA, NPOLES
from oracle import dirac, native, probing, qx, zolotarev
from synth import make_config, random_spinor

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "spectra.json")


def _spectra():
    with open(GOLD) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02211_gb300 import smpq
    smpq.load()
    return smpq


def _session(S, **kw):
    from paper_1901_02211_gb300 import Session
    return Session(**kw)


def _interval(name):
    sp = _spectra()[name]
    return 0.98 * sp["lmin2"], 1.02 * sp["lmax2"]


def _zolo(a, b):
    c0, c, q, d = zolotarev.zolotarev(NPOLES, a, b)
    return (c0, c, q), d


# ----------------------------------------------------------------------------- D_W


@pytest.mark.parametrize("name", ["flux4", "flux4x8", "flux8x16"])
@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
def test_dslash_fp64(S, name, bc):
    cfg = make_config(name)
    V = int(np.prod(cfg["dims"]))
    psi = random_spinor(np.random.default_rng(1), V, 3)
    with _session(S, bc=bc) as s:
        s.load_gauge(cfg["dims"], cfg["U"])
        for dag in (False, True):
            got = s.dslash(psi, dagger=dag)
            ref = native.apply_dw(cfg["U"], dirac.apply_g5(psi) if dag else psi, cfg["dims"], KAPPA, bc)
            if dag:
                ref = dirac.apply_g5(ref)
            assert np.abs(got - ref).max() <= 1e-13


def test_dslash_fp32(S):
    cfg = make_config("flux8x16")
    V = int(np.prod(cfg["dims"]))
    psi = random_spinor(np.random.default_rng(2), V, 2)
    with _session(S) as s:
        s.load_gauge(cfg["dims"], cfg["U"])
        got = s.dslash(psi, precision=S.SMPQ_FP32)
    ref = native.apply_dw(cfg["U"], psi, cfg["dims"], KAPPA)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


# Half-precision storage (SMPQ_FP16N / SMPQ_BF16N): FP16 or BF16 components
# scaled by one FP32 norm per site and right-hand side, links as FP16/BF16 rows
# 0 and 1 with row 2 = conj(row 0 x row 1), FP32 arithmetic.
# Largest rounding error of a stored value in [-1, 1]: half the spacing below 1.
HALF_UNIT = {"fp16": 2.0 ** -12, "bf16": 2.0 ** -9}
HALF_PREC = ("fp16n", "bf16n")


def _round_half(x, fmt):
    """float32 array -> nearest FP16 (numpy) or BF16 (torch on the CPU), as float64."""
    x = np.asarray(x, dtype=np.float32)
    if fmt == "fp16":
        return x.astype(np.float16).astype(np.float64)
    import torch
    return torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()


def _quantise_spinor(psi, fmt):
    """The field the half format holds for psi [V, 4, 3, B]: per (site, rhs) the
    FP32 norm n = max |re|, |im| of the 12 components, values n * half(v / n)."""
    V, B = psi.shape[0], psi.shape[-1]
    p = psi.reshape(V, 12, B)
    n = np.maximum(np.abs(p.real), np.abs(p.imag)).max(axis=1).astype(np.float32).astype(np.float64)
    d = np.where(n > 0, n, 1.0)[:, None, :]
    q = _round_half(p.real / d, fmt) + 1j * _round_half(p.imag / d, fmt)
    return (q * n[:, None, :]).reshape(psi.shape)


def _quantise_links(U, fmt):
    """Rows 0 and 1 rounded (FP32, then the half format), row 2 rebuilt as
    conj(row 0 x row 1) in FP64 (the unitary third row of an SU(3) matrix)."""
    Uq = np.empty_like(U)
    Uq[..., :2, :] = _round_half(U[..., :2, :].real, fmt) + 1j * _round_half(U[..., :2, :].imag, fmt)
    Uq[..., 2, :] = np.conj(np.cross(Uq[..., 0, :], Uq[..., 1, :]))
    return Uq


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("name,B,bc", [("flux4x8", 3, (1, 1, 1, -1)), ("flux8x16", 32, (1, 1, 1, 1)),
                                       ("flux8x16", 48, (1, 1, 1, -1))])
def test_dslash_half(S, fmt, name, B, bc):
    """D_W in the half format against the FP64 oracle D_W on the quantised field
    and links: the result differs only by its own rounding to the half format
    (<= HALF_UNIT of its (site, rhs) norm in every real and imaginary part) and
    FP32 arithmetic (< 1e-5 of that norm).
    B = 3 runs one-column tiles, B = 32 and 48 the 16-column tiles."""
    prec = S.SMPQ_FP16N if fmt == "fp16" else S.SMPQ_BF16N
    cfg = make_config(name)
    V = int(np.prod(cfg["dims"]))
    psi = random_spinor(np.random.default_rng(7), V, B)
    psi_q = _quantise_spinor(psi, fmt)
    U_q = _quantise_links(cfg["U"], fmt)
    with _session(S, bc=bc) as s:
        s.load_gauge(cfg["dims"], cfg["U"])
        for dag in (False, True):
            got = s.dslash(psi_q, dagger=dag, precision=prec)
            ref = native.apply_dw(U_q, dirac.apply_g5(psi_q) if dag else psi_q, cfg["dims"], KAPPA, bc)
            if dag:
                ref = dirac.apply_g5(ref)
            r12 = ref.reshape(V, 12, B)
            norm = np.maximum(np.abs(r12.real), np.abs(r12.imag)).max(axis=1)[:, None, :]
            d = got.reshape(V, 12, B) - r12
            err = np.maximum(np.abs(d.real), np.abs(d.imag)) / norm  # each real part is rounded on its own
            assert err.max() <= HALF_UNIT[fmt] * 1.001 + 1e-5, err.max()
            # against the unrounded field and links (the format's own error)
            full = native.apply_dw(cfg["U"], dirac.apply_g5(psi) if dag else psi, cfg["dims"], KAPPA, bc)
            if dag:
                full = dirac.apply_g5(full)
            rel = np.abs(got - full).max() / np.abs(full).max()
            print("\nD_W %s %s B=%d dagger=%d: max |err| / max |D_W psi| = %.3e (vs quantised inputs %.3e)"
                  % (fmt, name, B, dag, rel, err.max()))
            assert rel <= 16 * HALF_UNIT[fmt]


def test_time_dslash_every_format(S):
    cfg = make_config("flux4x8")
    V = int(np.prod(cfg["dims"]))
    with _session(S) as s:
        s.load_gauge(cfg["dims"], cfg["U"])
        for prec, spinor, link in ((S.SMPQ_FP64, 192, 144), (S.SMPQ_FP32, 96, 72), (S.SMPQ_FP16N, 52, 24),
                                   (S.SMPQ_BF16N, 52, 24)):
            for B in (12, 48):
                ms, nbytes = S.smpq_time_dslash(s.ctx, B, False, prec, 3)
                assert ms > 0
                assert nbytes == V * B * 2 * spinor + V * 4 * link
        with pytest.raises(S.SmpqError):
            S.smpq_time_dslash(s.ctx, 12, False, S.SMPQ_MIXED, 3)
        with pytest.raises(S.SmpqError):
            s.dslash(random_spinor(np.random.default_rng(1), V, 2), precision=S.SMPQ_MIXED)


# ----------------------------------------------------------------------------- D_ov, spectrum


def test_apply_dov_vs_dense(S, flux4, dense4, zolo4, g5dov4):
    U, dims = flux4["U"], flux4["dims"]
    v = random_spinor(np.random.default_rng(3), 256, 2)
    with _session(S) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(zolo4["a"], zolo4["b"])
        got = s.apply_dov(v)
    Dov = dense4["g5"] @ g5dov4
    ref = (Dov @ v.reshape(3072, 2)).reshape(256, 4, 3, 2)
    assert np.abs(got - ref).max() <= 1e-9


def test_measure_spectrum(S, flux4, dense4):
    with _session(S) as s:
        s.load_gauge(flux4["dims"], flux4["U"])
        lo, hi = s.measure_spectrum(300)
    l2 = dense4["lam"] ** 2
    assert l2.min() * (1 - 1e-9) <= lo <= l2.min() * (1 + 1e-4)
    assert l2.max() * (1 - 1e-4) <= hi <= l2.max() * (1 + 1e-9)


def test_zolotarev_of_context_matches_oracle(S, flux4, zolo4):
    with _session(S) as s:
        s.load_gauge(flux4["dims"], flux4["U"])
        s.set_spectrum(zolo4["a"], zolo4["b"])
        c0, c, q, d = s.zolotarev()
    assert np.allclose(c, zolo4["c"], rtol=1e-11) and np.allclose(q, zolo4["q"], rtol=1e-11)


# ----------------------------------------------------------------------------- q(x) on 4^4 against dense


@pytest.mark.parametrize("rhs_block", [1, 0])
@pytest.mark.parametrize("r,mode", [(2, 0), (2, 1), (2, 2), (4, 2)])
def test_qx_4x4_fp64_vs_dense(S, flux4, zolo4, g5dov4, r, mode, rhs_block):
    """Every colouring mode, batched and one source at a time (rhs_block = 1)."""
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, r, mode)
    ref = qx.dense_smp_qx(g5dov4, colour)
    with _session(S, rhs_block=rhs_block) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(zolo4["a"], zolo4["b"])
        assert s.build_sources(r, mode) == n
        q, Q, st = s.compute_qx()
    assert np.abs(q - ref).max() <= 1e-8
    assert abs(Q - ref.real.sum()) <= 1e-9
    assert st["max_resid"] <= 1e-10
    assert abs(st["max_im_q"] - np.abs(ref.imag).max()) <= 1e-8


def test_qx_8x16_mixed_enforced_base_residual(S):
    """true_residual = 2: the mixed path drives the base system to a true
    residual below tol after every shift has converged (one replacement, then
    a CG restart of the base shift); q(x) still meets the per-site bar."""
    cfg = make_config("flux8x16")
    U, dims = cfg["U"], cfg["dims"]
    a, b = _interval("flux8x16")
    zolo, delta = _zolo(a, b)
    colour, n = probing.color_sites(dims, 4, 0)
    classes = [0, 77, 255]
    ref, _ = qx.smp_qx(U, dims, KAPPA, zolo, colour, n, colours=classes, batch_colours=len(classes))
    with _session(S, precision=S.SMPQ_MIXED, true_residual=2) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(a, b)
        s.build_sources(4, 0)
        q, Q, st = s.compute_qx(classes=classes)
    mask = np.isin(colour, classes)
    err = np.abs(q[mask] - ref[mask]).max()
    print("8^3x16 r=4 mixed, base residual enforced: max |dq| = %.3e, |dQ| = %.3e, true residual %.2e, "
          "%d iterations" % (err, abs(Q - ref.real[mask].sum()), st["true_resid"], st["max_iterations"]))
    assert 0 <= st["true_resid"] <= 1.1e-10
    assert err <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("r,mode", [(2, 0), (2, 1)])
def test_qx_4x4_antiperiodic_vs_dense(S, flux4, r, mode, prec):
    """Antiperiodic fermion boundary in t (the other common convention): q^SMP
    against the dense gamma_5 D_ov built with the same boundary factors and
    its own spectrum."""
    U, dims = flux4["U"], flux4["dims"]
    bc = (1, 1, 1, -1)
    H = dirac.apply_g5(dirac.dense_dw(U, dims, KAPPA, bc).reshape(256, 4, 3, 3072)).reshape(3072, 3072)
    lam = np.linalg.eigvalsh(H)
    a, b = 0.98 * (lam ** 2).min(), 1.02 * (lam ** 2).max()
    zolo, delta = _zolo(a, b)
    ref = qx.dense_smp_qx(qx.dense_g5dov(U, dims, KAPPA, zolo, bc)[0], probing.color_sites(dims, r, mode)[0])
    precision = S.SMPQ_FP64 if prec == "fp64" else S.SMPQ_MIXED
    with _session(S, bc=bc, precision=precision) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(a, b)
        s.build_sources(r, mode)
        q, Q, st = s.compute_qx()
    err = np.abs(q - ref).max()
    print("4^4 antiperiodic r=%d mode %d %s: max |dq| = %.3e, Q = %.9f" % (r, mode, prec, err, Q))
    assert err <= 1e-8
    assert abs(Q - ref.real.sum()) <= 1e-9


@pytest.fixture(scope="module")
def flux4_light():
    """The 4^4 flux field with kappa = 0.08 (below the free critical 1/8): a
    well-conditioned H_W^2 (condition number about 20) for the storage formats
    whose rounding times the condition number of the kappa = 0.21 operator
    (about 360 on 4^4) leaves the reliable updates no contraction (BF16)."""
    from synth import make_config
    cfg = make_config("flux4")
    U, dims, kappa = cfg["U"], cfg["dims"], 0.08
    H = dirac.apply_g5(dirac.dense_dw(U, dims, kappa).reshape(256, 4, 3, 3072)).reshape(3072, 3072)
    lam = np.linalg.eigvalsh(H)
    a, b = 0.98 * (lam ** 2).min(), 1.02 * (lam ** 2).max()
    zolo, _ = _zolo(a, b)
    return dict(U=U, dims=dims, kappa=kappa, a=a, b=b, g5dov=qx.dense_g5dov(U, dims, kappa, zolo)[0])


@pytest.mark.parametrize("fmt", ["fp16n", "bf16n"])
def test_qx_4x4_half_one_source_at_a_time(S, flux4_light, fmt):
    """The half-storage solve with one source per batch (one-column tiles, the
    kernels of odd tile widths) against the dense matrix, at the format's
    floor (2 u per site, as the batched half-storage solves)."""
    U, dims = flux4_light["U"], flux4_light["dims"]
    colour, n = probing.color_sites(dims, 2, 0)
    ref = qx.dense_smp_qx(flux4_light["g5dov"], colour)
    precision = S.SMPQ_FP16N if fmt == "fp16n" else S.SMPQ_BF16N
    with _session(S, precision=precision, rhs_block=1, kappa=flux4_light["kappa"]) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(flux4_light["a"], flux4_light["b"])
        s.build_sources(2, 0)
        q, Q, st = s.compute_qx(classes=[0, 7])
    mask = np.isin(colour, [0, 7])
    err = np.abs(q[mask] - ref[mask]).max()
    scale = np.abs(ref[mask]).max()
    print("4^4 kappa 0.08 %s one source per batch: max |dq| = %.3e (max |q| %.3e), %d batches, %d iterations" % (
        fmt, err, scale, st["n_batches"], st["max_iterations"]))
    assert st["n_batches"] == 24 and st["rhs_tile"] == 1
    assert err <= 2 * HALF_UNIT[fmt[:4]]
    assert 0 <= st["true_resid"] <= 1e-10  # the last reliable update of the base system


def test_exact_trace_point_sources_4x4(S, flux4, zolo4, g5dov4):
    """r = n_mu: every set is one site, 3072 point sources (Eq. 5); Q = 1."""
    U, dims = flux4["U"], flux4["dims"]
    ref = qx.dense_smp_qx(g5dov4, np.arange(256))
    with _session(S) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(zolo4["a"], zolo4["b"])
        assert s.build_sources(4, 0) == 256
        q, Q, st = s.compute_qx()
    assert st["n_rhs"] == 3072
    assert np.abs(q - ref).max() <= 1e-8
    assert abs(Q - 1.0) <= 1e-8 + 6 * 256 * zolo4["delta"]
    assert st["max_im_q"] <= 1e-10


def test_unit_links_give_zero(S):
    dims = (4, 4, 4, 4)
    U = np.zeros((256, 4, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    with _session(S) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(0.2, 7.5)
        for mode in (0, 1, 2):
            s.build_sources(2, mode)
            q, Q, st = s.compute_qx()
            assert np.abs(q).max() <= 1e-11


# ----------------------------------------------------------------------------- 8^3 x 16 against the oracle (sampled classes)


def mixed_resid_bar(theta):
    """Bar on the base system's true residual after a mixed solve that switched
    to FP32 at ||r|| = theta ||b|| with no later replacement: 256 u_32 theta
    (u_32 = 2^-24) above the 1e-10 tolerance."""
    return 256 * 2.0 ** -24 * theta + 1e-10



@pytest.mark.parametrize("r,classes", [(2, [0, 9]), (4, [0, 77, 255])])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed1e-4", "mixed1e-3", "mixed7e-3", "mixed1e-2", "mixed3e-2", "fp16n",
                                  "bf16n"])
def test_qx_8x16_sampled(S, r, classes, prec):
    cfg = make_config("flux8x16")
    U, dims = cfg["U"], cfg["dims"]
    a, b = _interval("flux8x16")
    zolo, delta = _zolo(a, b)
    colour, n = probing.color_sites(dims, r, 0)
    ref, _ = qx.smp_qx(U, dims, KAPPA, zolo, colour, n, colours=classes, batch_colours=len(classes))
    precision = S.SMPQ_MIXED if prec.startswith("mixed") else {
        "fp64": S.SMPQ_FP64, "fp32": S.SMPQ_FP32, "fp16n": S.SMPQ_FP16N, "bf16n": S.SMPQ_BF16N}[prec]
    switch = float(prec[5:]) if prec.startswith("mixed") else 1e-3
    with _session(S, precision=precision, switch_residual=switch, true_residual=1) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(a, b)
        s.build_sources(r, 0)
        q, Q, st = s.compute_qx(classes=classes)
    mask = np.isin(colour, classes)
    err = np.abs(q[mask] - ref[mask]).max()
    print("8^3x16 r=%d %s: max |dq| = %.3e, iterations %d, reliable updates %d, true residual %.2e, "
          "recursive %.2e, %.2f launches per iteration" % (
              r, prec, err, st["max_iterations"], st["reliable_updates"], st["true_resid"], st["max_resid"],
              st["kernel_launches"] / st["max_iterations"]))
    # the base system's residual recomputed with FP64 accuracy after the solve:
    # the FP64, FP32 and half paths stop at the 1e-10 tolerance (FP32 and half
    # through their residual replacements); the mixed path's FP32 phase has no
    # replacement: it starts at ||r|| = theta ||b|| and its FP32 operator moves
    # the iterated residual away from the true one by about u_32 theta times a
    # growth factor (measured 50-70 on these lattices, bar 256)
    assert 0 <= st["true_resid"] <= (mixed_resid_bar(switch) if prec.startswith("mixed") else 1.1e-10)
    # FP64 and the FP64-then-FP32 path meet the 1e-8 per-site bar; the FP32
    # path with FP64 reliable updates has the FP32 floor of its shifted systems.
    # The per-site error of the mixed path grows with the switch point (about
    # 1e-8 theta).  The 1e-9 bar on the sum over the sampled sites holds up to
    # 7e-3 here; at 1e-2 and 3e-2 the bar is looser (informational).  Over the
    # whole lattice the drift of the FP32 phase adds up coherently, which is
    # why the default switch is 1e-3 (bench.py compares the whole-lattice Q
    # with the FP64 path)
    # The half-storage paths (FP16 / BF16 D_W input and output with per-site
    # norms, FP64 reliable updates) have the same kind of floor at the format's
    # rounding u (2^-12, 2^-9): held to 2 u per site, Q not checked.
    if prec in HALF_PREC:
        u = HALF_UNIT[prec[:4]]
        print("    |Q - Q_oracle| = %.3e (%d sites), per-site bound 2 u = %.2e" % (
            abs(Q - ref.real[mask].sum()), mask.sum(), 2 * u))
        assert err <= 2 * u
        return
    tol = 1e-5 if prec == "fp32" else 1e-8
    assert err <= tol
    qtol = {"fp32": 1e-4, "mixed1e-2": 3e-9, "mixed3e-2": 1e-7}.get(prec, 1e-9)
    assert abs(Q - ref.real[mask].sum()) <= qtol


# ----------------------------------------------------------------------------- star support against the whole lattice


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_support_ablation_4x4(S, flux4, zolo4, g5dov4, prec):
    """The shifted directions kept on every site (full_support) give the same
    q^SMP(x) as the star support: their recurrences never couple sites, so the
    restriction is exact (only rounding differs)."""
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, 2, 0)
    ref = qx.dense_smp_qx(g5dov4, colour)
    precision = S.SMPQ_FP64 if prec == "fp64" else S.SMPQ_MIXED
    out = {}
    for full in (0, 1):  # a fixed launch shape: the two runs differ only in the support
        with _session(S, precision=precision, full_support=full, autotune=0) as s:
            s.load_gauge(dims, U)
            s.set_spectrum(zolo4["a"], zolo4["b"])
            s.build_sources(2, 0)
            out[full] = s.compute_qx()[0]
    assert np.abs(out[1] - out[0]).max() <= 1e-12
    assert np.abs(out[1] - ref).max() <= 1e-8


# ----------------------------------------------------------------------------- host/device buffers, determinism, errors


def test_device_buffers_and_determinism(S, flux4, zolo4):
    with _session(S) as s:
        s.load_gauge(flux4["dims"], flux4["U"])
        s.set_spectrum(zolo4["a"], zolo4["b"])
        s.build_sources(2, 0)
        q1, Q1, _ = s.compute_qx()
        q2, Q2, _ = s.compute_qx()
        qd, Qd, _ = s.compute_qx(device=True)
    assert np.array_equal(q1, q2) and Q1 == Q2
    assert np.array_equal(qd.cpu().numpy(), q1) and Qd == Q1


def test_error_codes(S, flux4):
    from paper_1901_02211_gb300 import smpq
    with _session(S) as s:
        with pytest.raises(smpq.SmpqError) as e:
            s.build_sources(2, 0)
        assert e.value.code == smpq.SMPQ_ESTATE
        bad = flux4["U"].copy()
        bad[3, 1] *= 1.01
        with pytest.raises(smpq.SmpqError) as e:
            s.load_gauge(flux4["dims"], bad)
        assert e.value.code == smpq.SMPQ_ENOTSU3
        s.load_gauge(flux4["dims"], flux4["U"])
        with pytest.raises(smpq.SmpqError) as e:
            s.build_sources(3, 0)
        assert e.value.code == smpq.SMPQ_EINVAL
        s.build_sources(2, 0)
        with pytest.raises(smpq.SmpqError) as e:
            s.compute_qx()
        assert e.value.code == smpq.SMPQ_ESTATE  # no spectrum yet
        s.set_spectrum(0.02, 7.0)
        s.set_options(max_iter=5, iters_per_check=5)
        with pytest.raises(smpq.SmpqError) as e:
            s.compute_qx()
        assert e.value.code == smpq.SMPQ_ENOCONV


# ----------------------------------------------------------------------------- the bench's own launch configuration


def test_bench_configuration_sampled(S):
    """All 256 classes of r_min = 4 on 8^3 x 16 in one batch (3072 sources, the
    tile width and precision bench.py times) against the oracle on 16 classes
    spread over the lattice: q(x) per site and their sum (512 sites) at the Q bar."""
    cfg = make_config("flux8x16")
    U, dims = cfg["U"], cfg["dims"]
    a, b = _interval("flux8x16")
    zolo, delta = _zolo(a, b)
    colour, n = probing.color_sites(dims, 4, 0)
    sample = list(range(0, 256, 16))
    ref, _ = qx.smp_qx(U, dims, KAPPA, zolo, colour, n, colours=sample, batch_colours=len(sample))
    with _session(S, precision=S.SMPQ_MIXED) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(a, b)
        s.build_sources(4, 0)
        q, Q, st = s.compute_qx()
        # again, with the launch shape the first call tuned: the same bits
        q2, Q2, st2 = s.compute_qx()
    assert st["n_rhs"] == 3072 and st["n_batches"] == 1
    assert np.array_equal(q2, q) and Q2 == Q
    mask = np.isin(colour, sample)
    err = np.abs(q[mask] - ref[mask]).max()
    dQ = abs(q.real[mask].sum() - ref.real[mask].sum())
    print("bench configuration: max |dq| over %d sampled sites = %.3e, |dQ| over them = %.3e, Q = %.9f, "
          "%d launches for %d iterations" % (mask.sum(), err, dQ, Q, st["kernel_launches"], st["max_iterations"]))
    assert err <= 1e-8
    assert dQ <= 1e-9
    assert abs(Q - 2.0) < 0.05  # closed-form index k = 2, r_min = 4 probing bias
    # three launches per CG iteration (plus setup, phase switch, residual
    # replacement, contraction and the iterations of the last check interval
    # after convergence); the first call also ran the autotuner's timings
    print("    second call: %d launches, staged FP32 D_W %d" % (st2["kernel_launches"], st2["staged"]))
    assert st2["kernel_launches"] <= 3 * (st2["max_iterations"] + 20) + 60


# ----------------------------------------------------------------------------- SMP trace of D_W^{-1}


@pytest.mark.parametrize("r,mode", [(2, 0), (4, 0), (2, 1)])
def test_trace_dwinv_4x4_vs_dense(S, flux4, dense4, r, mode):
    U, dims = flux4["U"], flux4["dims"]
    colour, n = probing.color_sites(dims, r, mode)
    ref = qx.dense_smp_trace(np.linalg.inv(dense4["Dw"]), colour)
    with _session(S) as s:
        s.load_gauge(dims, U)
        s.build_sources(r, mode)
        t, T, st = s.trace_dwinv()
    assert np.abs(t - ref).max() <= 1e-8
    assert abs(T - ref.real.sum()) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_trace_dwinv_8x16_sampled(S, prec):
    cfg = make_config("flux8x16")
    U, dims = cfg["U"], cfg["dims"]
    colour, n = probing.color_sites(dims, 4, 0)
    sample = [0, 200]
    ref, _ = qx.smp_trace_dwinv(U, dims, KAPPA, colour, n, colours=sample, batch_colours=2)
    precision = S.SMPQ_FP64 if prec == "fp64" else S.SMPQ_MIXED
    with _session(S, precision=precision) as s:
        s.load_gauge(dims, U)
        s.build_sources(4, 0)
        t, T, st = s.trace_dwinv()
    mask = np.isin(colour, sample)
    err = np.abs(t[mask] - ref[mask]).max()
    print("trace D_W^-1 8^3x16 %s: max |dt| = %.3e, Tr = %.6f" % (prec, err, T))
    assert err <= 1e-8 * np.abs(ref[mask]).max()  # |t(x)| ~ 8: relative bar


# ----------------------------------------------------------------------------- uneven batch


def test_uneven_batch_matches_single_runs(S, flux4, zolo4, g5dov4):
    """Three lattices of different sizes and schemes in one batch call (their
    right-hand sides in the same launches) give the q(x) of three separate
    calls, to the accuracy of the mixed path (the batch switches precision
    when every lattice is below the switch residual, and reduces in its own
    tile shape), and each lattice agrees with the oracle: 4^4 with the dense
    matrix, 8^3 x 16 on two sampled classes."""
    from paper_1901_02211_gb300 import Session, smpq
    cases = [("flux4", 2, 0), ("flux4x8", 2, 1), ("flux8x16", 4, 0)]
    sessions, ref = [], []
    for name, r, mode in cases:
        cfg = make_config(name)
        a, b = (zolo4["a"], zolo4["b"]) if name == "flux4" else _interval(name)
        s = Session(precision=smpq.SMPQ_MIXED, true_residual=1)
        s.load_gauge(cfg["dims"], cfg["U"])
        s.set_spectrum(a, b)
        s.build_sources(r, mode)
        q, Q, st = s.compute_qx()
        sessions.append(s)
        ref.append((q, Q))
    bufs_re = [np.zeros(s.V) for s in sessions]
    bufs_im = [np.zeros(s.V) for s in sessions]
    Qs, stats = smpq.smpq_compute_qx_batch([s.ctx for s in sessions], bufs_re, bufs_im)
    for i, (q, Q) in enumerate(ref):
        qb = bufs_re[i] + 1j * bufs_im[i]
        d = np.abs(qb - q).max()
        print("uneven batch, lattice %d: max |q_batch - q_single| = %.3e, Q %.12f vs %.12f, %d iterations, "
              "%d batches, true residual %.2e" % (i, d, Qs[i], Q, stats[i]["max_iterations"], stats[i]["n_batches"],
                                                  stats[i]["true_resid"]))
        assert d <= 1e-9
        assert abs(Qs[i] - Q) <= 1e-9
        assert 0 <= stats[i]["true_resid"] <= mixed_resid_bar(1e-3)  # the mixed path's measured base residual
    # against the oracle
    q4 = bufs_re[0] + 1j * bufs_im[0]
    dense = qx.dense_smp_qx(g5dov4, probing.color_sites((4, 4, 4, 4), 2, 0)[0])
    assert np.abs(q4 - dense).max() <= 1e-8
    cfg = make_config("flux8x16")
    zolo, _ = _zolo(*_interval("flux8x16"))
    colour, n = probing.color_sites(cfg["dims"], 4, 0)
    sample = [5, 200]
    oref, _ = qx.smp_qx(cfg["U"], cfg["dims"], KAPPA, zolo, colour, n, colours=sample, batch_colours=2)
    mask = np.isin(colour, sample)
    q8 = bufs_re[2] + 1j * bufs_im[2]
    assert np.abs(q8[mask] - oref[mask]).max() <= 1e-8
    for s in sessions:
        s.close()


# ----------------------------------------------------------------------------- 16^3 x 32 (sampled)


def test_qx_16x32_sampled(S):
    """16^3 x 32 flux configuration (Q = -1, noise 0.15), r_min = 4, one class
    against the oracle.  The Zolotarev interval is fixed a priori (parity only
    needs both sides to use the same rational)."""
    cfg = make_config("flux16x32")
    U, dims = cfg["U"], cfg["dims"]
    a, b = 0.01, 7.5
    zolo, delta = _zolo(a, b)
    colour, n = probing.color_sites(dims, 4, 0)
    sample = [93]
    ref, _ = qx.smp_qx(U, dims, KAPPA, zolo, colour, n, colours=sample, batch_colours=1)
    with _session(S, precision=S.SMPQ_MIXED) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(a, b)
        s.build_sources(4, 0)
        q, Q, st = s.compute_qx(classes=sample)
    mask = np.isin(colour, sample)
    err = np.abs(q[mask] - ref[mask]).max()
    print("16^3x32 mixed: max |dq| over %d sites = %.3e, iterations %d" % (mask.sum(), err, st["max_iterations"]))
    assert err <= 1e-8


# ----------------------------------------------------------------------------- autotuner


def test_autotuner_shapes_and_cache_file(S, tmp_path):
    """The autotuner picks a D_W launch shape (RHS tile, tiles per block of each
    phase, FP32 columns per thread, staged FP32 neighbours), writes it to the
    cache file, and a second context reads it back without timing.  Shapes
    forced through the file (two FP32 columns per thread, one and eight tiles
    per block; the staged FP32 and float-float D_W on 24-column tiles, three
    tiles per block, so the last block holds one) give the same q(x) to
    rounding, and all agree with the oracle."""
    cfg = make_config("flux8x16")
    U, dims = cfg["U"], cfg["dims"]
    a, b = _interval("flux8x16")
    zolo, delta = _zolo(a, b)
    colour, n = probing.color_sites(dims, 4, 0)
    classes = [3, 100, 200, 250]  # 48 sources: tiles 12, 24 and 48 all divide the batch
    ref, _ = qx.smp_qx(U, dims, KAPPA, zolo, colour, n, colours=classes, batch_colours=len(classes))
    mask = np.isin(colour, classes)
    path = str(tmp_path / "tune.txt")
    out = []
    for k, forced in enumerate((None, None, (12, 1, 8, 2, 0), (24, 3, 3, 1, 3))):
        if forced is not None:
            path = str(tmp_path / ("forced%d.txt" % k))
            S.smpq_tune_cache_store(path, _device_key(S), dims, 48, S.SMPQ_MIXED, forced, 1.0)
        with _session(S, precision=S.SMPQ_MIXED, tune_cache=path) as s:
            s.load_gauge(dims, U)
            s.set_spectrum(a, b)
            s.build_sources(4, 0)
            q, Q, st = s.compute_qx(classes=classes)
        shape = (st["rhs_tile"], st["tiles_per_block_hi"], st["tiles_per_block_lo"], st["cols_per_thread"],
                 st["staged"])
        err = np.abs(q[mask] - ref[mask]).max()
        print("autotuner: shape %s from cache %d, max |dq| vs oracle %.3e" % (shape, st["shape_from_cache"], err))
        assert err <= 1e-8
        out.append((shape, st["shape_from_cache"], q))
    assert out[0][1] == 0 and out[1][1] == 1 and out[1][0] == out[0][0]
    assert out[2][1] == 1 and out[2][0] == (12, 1, 8, 2, 0)
    assert out[3][1] == 1 and out[3][0] == (24, 3, 3, 1, 3)  # staged FP32 and float-float D_W
    assert np.abs(out[2][2][mask] - out[0][2][mask]).max() <= 1e-10
    assert np.abs(out[3][2][mask] - out[0][2][mask]).max() <= 1e-10
    assert len(open(str(tmp_path / "tune.txt")).read().splitlines()) == 1


def test_staged_batch_matches_plain(S, flux4, zolo4):
    """Neighbour staging in both phases of the mixed solve (staging = 1), in the
    one-solve batch of two lattices (the multi-lattice kernels), against single
    runs with plain loads (staging = 0): the same arithmetic, so q(x) agrees to
    rounding of the reductions."""
    from paper_1901_02211_gb300 import Session, smpq
    cases = [("flux4", 2), ("flux8x16", 2)]
    singles, staged = [], []
    for name, r in cases:
        cfg = make_config(name)
        a, b = (zolo4["a"], zolo4["b"]) if name == "flux4" else _interval(name)
        for stg, out in ((0, singles), (1, staged)):
            s = Session(precision=smpq.SMPQ_MIXED, staging=stg, autotune=0)
            s.load_gauge(cfg["dims"], cfg["U"])
            s.set_spectrum(a, b)
            s.build_sources(r, 0)
            out.append(s)
    ref = [s.compute_qx()[0] for s in singles]
    bufs_re = [np.zeros(s.V) for s in staged]
    bufs_im = [np.zeros(s.V) for s in staged]
    Qs, stats = smpq.smpq_compute_qx_batch([s.ctx for s in staged], bufs_re, bufs_im)
    for i in range(len(cases)):
        d = np.abs(bufs_re[i] + 1j * bufs_im[i] - ref[i]).max()
        print("staged batch, lattice %d: max |q_staged - q_plain| = %.3e, staged bits %d" % (i, d, stats[i]["staged"]))
        assert stats[i]["staged"] == 3
        assert d <= 1e-10
    for s in singles + staged:
        s.close()


def _device_key(S):
    """The device string the library keys its tuning cache with."""
    import torch
    p = torch.cuda.get_device_properties(0)
    return "%s/%dsm" % (p.name, p.multi_processor_count)
