"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates inputs*: gauge fields (quantised-flux backgrounds,
Haar-random links, SU(3) noise, random gauge transforms, stout-style smoothing),
random spinors and random sample sets.  It holds none of the arithmetic of the
probing method itself (no Dirac operator, no rational sign function, no solver,
no trace), so both the CPU oracle and the CUDA path may consume what it makes.
"""
from .gauge import (  # noqa: F401
    site_coords,
    site_index,
    flux_field,
    haar_su3,
    su3_noise,
    apply_noise,
    random_gauge,
    gauge_transform,
    stout_smooth,
    random_spinor,
    make_config,
    CONFIGS,
)
