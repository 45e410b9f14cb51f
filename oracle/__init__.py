"""CPU FP64 oracle for the symmetric multi-probing (SMP) estimate of q(x).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline / reference legs may import this package.  The product
path (the C-ABI library and its Python binding) never imports, links or runs
anything here, and this package never imports the product path.

Each module follows one part of the paper (arXiv:1901.02211) in plain numpy /
scipy FP64, written for readability, not speed:

  dirac.py     Wilson kernel D_W with hopping parameter kappa (Sec. 2.1, around
               Eq. 3), gamma_5, H_W = gamma_5 D_W, H_W^2 = D_W^dag D_W (Eq. 4);
  zolotarev.py rational sign function eps(H) = H (c0 + sum_i c_i/(H^2 + q_i))
               (Eq. 4) from Zolotarev's optimal approximation;
  msolve.py    shifted solves (D_W^dag D_W + q_i) x_i = b (Eqs. 6-8) by
               multi-shift CG, plus a single-shift CG used by the pins;
  probing.py   symmetric colouring P(m_x, m_y, m_z, m_t, mode) for the Normal,
               Split and Combine modes, site sets S(X, P) and SMP sources
               (Sec. 2.2, Eqs. 15, 18-19; Tables 1-2);
  qx.py        q(x) = 1/2 tr(gamma_5 D_ov)(x, x) by point sources (Eq. 5) and its
               SMP estimate (Eq. 16), and Q = sum_x q(x);
  spectrum.py  spectral bounds of H_W^2 (setup for Eq. 4; the paper is silent);
  lowmodes.py  the lowest eigenmodes of H_W treated exactly in eps(H_W) (Eq. 4),
               with the rational on the shortened interval (not in the paper;
               its Sec. 3 compares against low modes of D_ov).

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, dense linear algebra on 4^4 or the integers the paper prints.
"""
