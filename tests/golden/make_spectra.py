"""Write tests/golden/spectra.json: extreme eigenvalues of H_W^2 = D_W^dag D_W
(kappa = 0.21, Sec. 2.1) for the named synthetic configurations.

Calls only the oracle (ARPACK on the compiled oracle operator) and the input
generators.  Run from the repository root:  python tests/golden/make_spectra.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import spectrum  # noqa: E402
from synth import make_config  # noqa: E402

NAMES = ["flux4", "flux4x8", "flux8x16"]


def main():
    out = {}
    for name in NAMES:
        cfg = make_config(name)
        lmin2, lmax2 = spectrum.h2_extremes(cfg["U"], cfg["dims"], 0.21, tol=1e-9)
        out[name] = {"lmin2": lmin2, "lmax2": lmax2, "kappa": 0.21, "bc": [1, 1, 1, 1]}
        print(name, lmin2, lmax2, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spectra.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
