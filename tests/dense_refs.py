"""Dense matrices built directly from the paper's definitions, for pinning the oracle.

These builders do not call the oracle's operator code: they assemble the Kronecker sums with
np.kron and the real 2x2 block matrices literally, so that a transposed operand, a wrong axis,
a wrong sign or a dropped term in the oracle's structured code shows up as a mismatch.
"""
from __future__ import annotations

import mpmath
import numpy as np


def fcd_mp(alpha: float, count: int, dps: int = 50) -> np.ndarray:
    """c_k from the Gamma-function formula (Sec. 2.1, eq. 'coefficients') in `dps`-digit arithmetic.
    1/Gamma is taken with rgamma so the poles at alpha = 2 give exact zeros."""
    with mpmath.workdps(dps):
        a = mpmath.mpf(alpha)
        g = mpmath.gamma(a + 1)
        out = []
        for k in range(count):
            v = (-1) ** k * g * mpmath.rgamma(a / 2 - k + 1) * mpmath.rgamma(a / 2 + k + 1)
            out.append(float(v))
    return np.array(out)


def toeplitz_dense(c: np.ndarray, n: int) -> np.ndarray:
    T = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            T[i, j] = c[abs(i - j)]
    return T


def kron_sum(mats):
    """sum_a I (x) .. (x) M_a (x) .. (x) I with axis 0 (x) innermost: for d = 2 this is
    I (x) M_x + M_y (x) I (Sec. 2.2, eq. '2DToeplitz') acting on vec(U) with x fastest."""
    d = len(mats)
    ns = [m.shape[0] for m in mats]
    N = int(np.prod(ns))
    out = np.zeros((N, N))
    for a in range(d):
        term = np.ones((1, 1))
        for b in reversed(range(d)):           # slowest axis first in the Kronecker product
            term = np.kron(term, mats[a] if b == a else np.eye(ns[b]))
        out += term
    return out


def T_dense(problem, c: np.ndarray, scale: float = 1.0) -> np.ndarray:
    mats = []
    for a in range(problem.d):
        mu = scale * problem.dt / problem.h(a) ** problem.alpha
        mats.append(mu * toeplitz_dense(c, problem.n[a]))
    return kron_sum(mats)


def hankel_dense(c: np.ndarray, n: int) -> np.ndarray:
    """HC(T_0) entry by entry from the picture of eq. 'HCform' (1-based i, j)."""
    H = np.zeros((n, n))
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            s = i + j
            if 2 <= s <= n - 1:
                H[i - 1, j - 1] = c[s]
            elif n + 3 <= s <= 2 * n:
                H[i - 1, j - 1] = c[2 * n + 2 - s]
    return H


def tauT_dense(problem, c: np.ndarray, scale: float = 1.0) -> np.ndarray:
    mats = []
    for a in range(problem.d):
        mu = scale * problem.dt / problem.h(a) ** problem.alpha
        n = problem.n[a]
        mats.append(mu * (toeplitz_dense(c, n) - hankel_dense(c, n)))
    return kron_sum(mats)


def block_mats(T: np.ndarray, D: np.ndarray):
    """calT = [[0, T], [-T, 0]], calD = [[I, -D], [D, I]], R = calT + calD  (eq. 'TBANsplitting')."""
    N = T.shape[0]
    I = np.eye(N)
    Dm = np.diag(D.ravel())
    Z = np.zeros((N, N))
    calT = np.block([[Z, T], [-T, Z]])
    calD = np.block([[I, -Dm], [Dm, I]])
    return calT, calD, calT + calD


def F_tilde_dense(tauT: np.ndarray, D: np.ndarray, omega: float) -> np.ndarray:
    """F~ = (1/2w)[wI + tau(calT)](wI + calD)  (eq. 'taupre')."""
    tcalT, calD, _ = block_mats(tauT, D)
    I2 = np.eye(tcalT.shape[0])
    return (omega * I2 + tcalT) @ (omega * I2 + calD) / (2 * omega)


def F_G_dense(T: np.ndarray, D: np.ndarray, omega: float):
    """F = (1/2w)(wI + calT)(wI + calD), G = (1/2w)(wI - calT)(wI - calD)  (eq. 'defpreconditionger1')."""
    calT, calD, R = block_mats(T, D)
    I2 = np.eye(calT.shape[0])
    F = (omega * I2 + calT) @ (omega * I2 + calD) / (2 * omega)
    G = (omega * I2 - calT) @ (omega * I2 - calD) / (2 * omega)
    return F, G, R
