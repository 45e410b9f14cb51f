import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KAPPA = 0.21  # Sec. 2.1
NPOLES = 14   # Sec. 2.1 (14-term Zolotarev)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~30 s")


@pytest.fixture(scope="session")
def flux4():
    from synth import make_config
    return make_config("flux4")


@pytest.fixture(scope="session")
def dense4(flux4):
    """Dense eigen-decomposition of H_W = gamma_5 D_W on the 4^4 flux configuration."""
    from oracle import dirac
    U, dims = flux4["U"], flux4["dims"]
    V = int(np.prod(dims))
    Dw = dirac.dense_dw(U, dims, KAPPA)
    g5 = np.kron(np.eye(V), np.kron(dirac.GAMMA5, np.eye(3)))
    H = g5 @ Dw
    lam, W = np.linalg.eigh(H)
    return dict(H=H, lam=lam, W=W, g5=g5, Dw=Dw)


@pytest.fixture(scope="session")
def zolo4(dense4):
    from oracle import zolotarev
    l2 = dense4["lam"] ** 2
    a, b = 0.98 * l2.min(), 1.02 * l2.max()
    c0, c, q, delta = zolotarev.zolotarev(NPOLES, a, b)
    return dict(a=a, b=b, c0=c0, c=c, q=q, delta=delta)


@pytest.fixture(scope="session")
def g5dov4(dense4, zolo4):
    """Dense gamma_5 D_ov = gamma_5 + H R(H^2) with the same rational as the solver path."""
    lam, W = dense4["lam"], dense4["W"]
    f = lam * (zolo4["c0"] + np.sum(zolo4["c"][None, :] / (lam[:, None] ** 2 + zolo4["q"][None, :]), axis=1))
    return dense4["g5"] + (W * f[None, :]) @ W.conj().T
