"""Analyses on top of the q(x) path (the paper's Sec. 3 studies, on synthetic
configurations).  All compute runs in libsmpq through the C ABI.

  rmin_sweep : Q_P for several colouring schemes P(m, mode) and the
               systematic error |Q_P - Q| against the exact index, with
               N^SMP and N^SMP / N^PT (the analogue of Tables 2-3 and of the
               error-versus-r_min and error-versus-efficiency figures);
  locality   : |D_ov(x, y)| against the minimum-image Euclidean and taxi
               distance |x - y|, from the 12 point-source columns of one site,
               with the decay rate gamma of the bound |D_ov(x,y)| <= C e^{-gamma|x-y|}
               (Eq. 12) fitted for |x - y| >= 3.

Usage:  python -m paper_1901_02211_gb300.experiments rmin [config]
        python -m paper_1901_02211_gb300.experiments locality [config]
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

from . import smpq
from .session import Session

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _min_image(dims, x, y):
    d = np.abs(np.asarray(x) - np.asarray(y))
    return np.minimum(d, np.asarray(dims) - d)


def _coords(dims, s):
    nx, ny, nz, nt = dims
    return np.stack([s % nx, (s // nx) % ny, (s // (nx * ny)) % nz, s // (nx * ny * nz)], axis=-1)


def schemes_for(dims):
    """Symmetric schemes (r, mode) that tile L(n_x, n_y, n_z, n_t) (Eq. 19)."""
    out = []
    for r in range(2, min(dims) + 1):
        if any(n % r for n in dims):
            continue
        out.append((r, 0))
        if all((n // r) % 2 == 0 for n in dims):
            out.append((r, 1))
        if r % 2 == 0:
            out.append((r, 2))
    return out


def r_min_of(r, mode):
    """Eq. 19: r_min = r (modes 0, 2) or sqrt(2) r (mode 1)."""
    return r * math.sqrt(2) if mode == 1 else float(r)


def rmin_sweep(dims, U, lmin2, lmax2, Q_exact, schemes=None, precision=smpq.SMPQ_MIXED, device=0, max_rhs=None,
               exact_qx=False):
    """Q_P and |Q_P - Q| for each scheme; returns a list of dicts.

    exact_qx: also evaluate the exact q(x) by point sources (the scheme with
    r = n_mu, needs a hypercubic lattice) and report the root-mean-square
    per-site probing error of every scheme against it."""
    rows = []
    with Session(device=device, precision=precision) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(lmin2, lmax2)
        V = int(np.prod(dims))
        q_exact = None
        if exact_qx:
            if len(set(dims)) != 1:
                raise ValueError("point sources through the scheme r = n need a hypercubic lattice")
            s.build_sources(dims[0], 0)
            q_exact, _, _ = s.compute_qx()
        for r, mode in (schemes or schemes_for(dims)):
            n = s.build_sources(r, mode)
            if max_rhs and 12 * n > max_rhs:
                continue
            t0 = time.perf_counter()
            q, Q, st = s.compute_qx()
            dt = time.perf_counter() - t0
            row = dict(r=r, mode=mode, m=dims[0] // r, r_min=r_min_of(r, mode), N_smp=12 * n,
                       ratio=12 * n / (12.0 * V), Q_P=Q, err=abs(Q - Q_exact), max_im_q=st["max_im_q"],
                       iterations=st["max_iterations"], seconds=dt)
            if q_exact is not None:
                row["site_rms"] = float(np.sqrt(np.mean(np.abs(q - q_exact) ** 2)))
                row["Q_pointsource"] = float(q_exact.real.sum())
            rows.append(row)
    return rows


def locality(dims, U, lmin2, lmax2, site=0, device=0):
    """Frobenius norm of the 12x12 block D_ov(y, site) for every y, with distances.

    Returns dict(euclid, taxi, norm, gamma_euclid, gamma_taxi).
    """
    V = int(np.prod(dims))
    src = np.zeros((V, 4, 3, 12), dtype=np.complex128)
    for k in range(12):
        src[site, k // 3, k % 3, k] = 1.0
    with Session(device=device, precision=smpq.SMPQ_FP64) as s:
        s.load_gauge(dims, U)
        s.set_spectrum(lmin2, lmax2)
        col = s.apply_dov(src)
    norm = np.sqrt(np.sum(np.abs(col) ** 2, axis=(1, 2, 3)))
    d = _min_image(dims, _coords(dims, np.arange(V)), _coords(dims, np.array(site)))
    euclid = np.sqrt((d * d).sum(-1))
    taxi = d.sum(-1)
    out = dict(euclid=euclid, taxi=taxi, norm=norm)
    for key, dist in (("euclid", euclid), ("taxi", taxi)):
        uniq = np.unique(dist[dist >= 3])
        mean = np.array([norm[dist == u].mean() for u in uniq])
        ok = mean > 0
        slope, _ = np.polyfit(uniq[ok], np.log(mean[ok]), 1)
        out["gamma_" + key] = float(-slope)
        out["profile_" + key] = (uniq.tolist(), mean.tolist())
    return out


def _load(name, device=0, lanczos_steps=300):
    """The synthetic configuration and its Zolotarev interval, measured on the
    GPU (smpq_measure_spectrum: Lanczos on H_W^2, widened to 0.98 / 1.02)."""
    sys.path.insert(0, ROOT)
    from synth import make_config
    cfg = make_config(name)
    with Session(device=device) as s:
        s.load_gauge(cfg["dims"], cfg["U"])
        lo, hi = s.measure_spectrum(lanczos_steps)
    return cfg, 0.98 * lo, 1.02 * hi


def main(argv):
    what = argv[1] if len(argv) > 1 else "rmin"
    name = argv[2] if len(argv) > 2 else "flux8x16"
    cfg, a, b = _load(name)
    if what == "rmin":
        rows = rmin_sweep(cfg["dims"], cfg["U"], a, b, cfg["Q_closed"], max_rhs=12 * 4096)
        print("| P(m, mode) | r_min | N^SMP | N^SMP/N^PT | Q_P | \\|Q_P - Q\\| | iterations | s |")
        print("|---|---|---|---|---|---|---|---|")
        for r in rows:
            print("| (%d, %d) | %.3f | %d | 1/%d | %.6f | %.2e | %d | %.2f |" % (
                r["m"], r["mode"], r["r_min"], r["N_smp"], round(1 / r["ratio"]), r["Q_P"], r["err"],
                r["iterations"], r["seconds"]))
    else:
        out = locality(cfg["dims"], cfg["U"], a, b)
        print("gamma (Euclid) = %.3f, gamma (taxi) = %.3f" % (out["gamma_euclid"], out["gamma_taxi"]))
        for key in ("euclid", "taxi"):
            xs, ys = out["profile_" + key]
            print(key, " ".join("%.2f:%.2e" % (x, y) for x, y in zip(xs, ys)))


if __name__ == "__main__":
    main(sys.argv)
