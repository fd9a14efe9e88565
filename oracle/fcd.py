"""Fractional centred-difference coefficients (paper Sec. 2.1, eq. 'coefficients').

    c_k = (-1)^k Gamma(alpha+1) / ( Gamma(alpha/2 - k + 1) Gamma(alpha/2 + k + 1) ),  k in Z,

with c_k = c_{-k}.  The Riesz derivative of order 1 < alpha <= 2 on a grid of step h is
approximated by -(1/h^alpha) sum_k c_{j-k} u_k (Sec. 2.1).
"""
from __future__ import annotations

import math

import numpy as np


def fcd_coefficients(alpha: float, count: int) -> np.ndarray:
    """Return c_0 .. c_{count-1} (float64).

    c_0 = Gamma(alpha+1) / Gamma(alpha/2+1)^2 is the k = 0 case of the formula.  The others use the
    ratio of consecutive terms, which follows from Gamma(z+1) = z Gamma(z) applied to both Gamma
    factors of the formula:

        c_{k+1} / c_k = -(alpha/2 - k) / (alpha/2 + k + 1) = (k - alpha/2) / (alpha/2 + k + 1).

    This avoids the overflow of Gamma(alpha/2 + k + 1) for large k; it is exact in exact arithmetic
    (the test suite checks it against the Gamma formula in 50-digit arithmetic).
    """
    if count <= 0:
        return np.zeros(0)
    c = np.empty(count, dtype=np.float64)
    c[0] = math.gamma(alpha + 1.0) / math.gamma(alpha / 2.0 + 1.0) ** 2
    half = alpha / 2.0
    for k in range(count - 1):
        c[k + 1] = c[k] * (k - half) / (half + k + 1.0)
    return c
