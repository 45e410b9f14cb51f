"""Zolotarev rational sign function (Eq. 4; Sec. 2.1).

The paper writes eps(H_W) = H_W (c0 + sum_{i=1}^{n} c_i / (H_W^2 + q_i)) with a
14-term Zolotarev expansion, without printing coefficients.  This module builds
R(x) = c0 + sum_i c_i/(x + q_i), the type-(n, n) rational with the least maximal
relative error for 1/sqrt(x) on [a, b] = [lambda_min^2, lambda_max^2] of H_W^2,
from Zolotarev's theorem as written out for overlap fermions by
Chiu, Hsieh, Huang and Huang, Phys. Rev. D 66 (2002) 114502, and
van den Eshof et al., Comput. Phys. Commun. 146 (2002) 203:

  with y = x/a in [1, b/a], modulus k' = sqrt(1 - a/b), K' = K(k'),
  c_l = sn^2(l K'/(2n+1); k') / cn^2(l K'/(2n+1); k'),   l = 1..2n,
  R(y) ~ d0 * prod_{l=1}^{n} (y + c_{2l}) / (y + c_{2l-1}).

The scale d0 equalises the relative error at the two ends of the interval
(both ends are alternation points of the optimal error curve), and the product
is converted to partial fractions.  Jacobi elliptic functions come from scipy.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ellipj, ellipk


def zolotarev_product(n, a, b):
    """Return (d0, zeros_c_even[n], poles_c_odd[n], delta) in the variable y = x/a."""
    if not (0 < a < b):
        raise ValueError("need 0 < a < b")
    m = 1.0 - a / b  # parameter m = k'^2 of the elliptic functions
    K = ellipk(m)
    l = np.arange(1, 2 * n + 1, dtype=np.float64)
    sn, cn, _, _ = ellipj(l * K / (2 * n + 1), m)
    c = (sn / cn) ** 2
    zeros = c[1::2]  # c_2, c_4, ..., c_2n
    poles = c[0::2]  # c_1, c_3, ..., c_{2n-1}
    ymax = b / a

    def f(y):
        return np.sqrt(y) * np.prod((y + zeros) / (y + poles))

    f1, f2 = f(1.0), f(ymax)
    d0 = 2.0 / (f1 + f2)
    delta = abs(f1 - f2) / (f1 + f2)
    return d0, zeros, poles, delta


def zolotarev(n, a, b):
    """Coefficients of R(x) = c0 + sum_i c_i/(x + q_i) ~ 1/sqrt(x) on [a, b].

    Returns (c0, c[n], q[n], delta) with q ascending; delta is the maximal
    relative error |1 - sqrt(x) R(x)| on [a, b].
    """
    d0, zeros, poles, delta = zolotarev_product(n, a, b)
    # partial fractions in y: d0 * prod (y+z_j)/(y+p_j) = d0 + sum_l d0*res_l/(y+p_l)
    res = np.empty(n)
    for i in range(n):
        num = np.prod(zeros - poles[i])
        den = np.prod(np.delete(poles, i) - poles[i])
        res[i] = d0 * num / den
    s = np.sqrt(a)
    # 1/sqrt(x) = (1/s) * 1/sqrt(y),  y = x/a:  (1/s) res/(x/a + p) = (res * a / s)/(x + p a)
    c0 = d0 / s
    c = res * a / s
    q = poles * a
    return c0, c, q, delta


def rational(x, c0, c, q):
    """R(x) = c0 + sum_i c_i/(x + q_i) for scalar or array x."""
    x = np.asarray(x, dtype=np.float64)
    return c0 + np.sum(c[None, :] / (x.reshape(-1, 1) + q[None, :]), axis=1).reshape(x.shape)
