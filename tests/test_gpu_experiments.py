"""The paper's qualitative findings (Sec. 2.2 and Sec. 3) on a synthetic
configuration, through the GPU path:

  * the SMP systematic error |Q_P - Q| falls as r_min grows (Table 3);
  * the off-diagonal elements of D_ov decay exponentially with distance, faster
    in Euclidean than in taxi-driver distance (Eq. 12 and the locality figure).
"""
import json
import os

import numpy as np
import pytest

from synth import make_config

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "spectra.json")


def _setup(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = make_config(name)
    with open(GOLD) as f:
        sp = json.load(f)[name]
    return cfg, 0.98 * sp["lmin2"], 1.02 * sp["lmax2"]


def test_error_falls_with_rmin():
    """4^4 flux configuration (Q = 1): the per-site probing error against the
    exact point-source q(x), and |Q_P - Q|, fall as r_min grows; at equal
    r_min the Combine mode (more nearest neighbours) is worse than Normal (Sec. 2.2)."""
    from paper_1901_02211_gb300 import experiments
    cfg, a, b = _setup("flux4")
    rows = experiments.rmin_sweep(cfg["dims"], cfg["U"], a, b, cfg["Q_closed"],
                                  schemes=[(2, 0), (2, 1), (2, 2), (4, 2)], exact_qx=True)
    e = {(r["r"], r["mode"]): r for r in rows}
    for r in rows:
        print("P r=%d mode=%d r_min=%.3f N=%d Q_P=%.6f |Q_P-Q|=%.3e site rms %.3e" % (
            r["r"], r["mode"], r["r_min"], r["N_smp"], r["Q_P"], r["err"], r["site_rms"]))
    assert abs(rows[0]["Q_pointsource"] - 1.0) < 1e-8  # exact trace = index
    rms = {k: v["site_rms"] for k, v in e.items()}
    err = {k: v["err"] for k, v in e.items()}
    assert rms[(4, 2)] < rms[(2, 1)] < rms[(2, 0)] < rms[(2, 2)]
    assert err[(4, 2)] < err[(2, 1)] < err[(2, 0)]


def test_locality_of_dov():
    from paper_1901_02211_gb300 import experiments
    cfg, a, b = _setup("flux8x16")
    out = experiments.locality(cfg["dims"], cfg["U"], a, b, site=0)
    print("gamma Euclid %.3f, taxi %.3f" % (out["gamma_euclid"], out["gamma_taxi"]))
    assert out["gamma_euclid"] > 0.5
    assert out["gamma_taxi"] > 0.2
    assert out["gamma_euclid"] > out["gamma_taxi"]
    xs, ys = out["profile_euclid"]
    assert ys[-1] < 1e-2 * ys[0]  # exponential fall-off over the lattice
