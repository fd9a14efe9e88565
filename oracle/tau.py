"""tau-matrix approximation of the Toeplitz matrices (paper Sec. 4).

    tau(T_1) = T_1 - HC(T_1)                           (eq. 'taudefine')
    HC(T_1)  = Hankel correction with anti-diagonals c_2 .. c_{M-1} from the top-left corner and
               c_{M-1} .. c_2 towards the bottom-right corner   (eq. 'HCform')
    tau(T_1) = S Lambda S                              (eq. 'taudiagonal')
    [S]_{ij} = sqrt(2/(M+1)) sin(pi i j/(M+1)),  1 <= i, j <= M

The printed normalisation of S reads sqrt(1/(M+1)); with it S*S = I/2, which contradicts
tau = S Lambda S with S symmetric and the eigenvalues "determined by the first column".  The
orthogonal (and involutory) DST-I normalisation sqrt(2/(M+1)) is used instead.

The d-level tau matrix is the Kronecker sum of the per-axis tau matrices (eq. '2Dtau'); with
unequal steps each axis carries its own mu_a (Sec. 4 states the h_x != h_y case is analogous).
"""
from __future__ import annotations

import numpy as np

from .operators import toeplitz_T0, apply_along_axis


def hankel_correction(c: np.ndarray, n: int) -> np.ndarray:
    """HC(T_0) for the n x n symmetric Toeplitz T_0 with first row c_0..c_{n-1} (eq. 'HCform').

    With 1-based indices (i, j): the entry is c_{i+j} on the anti-diagonals i+j = 2..n-1 (upper-left
    triangle, c_2 at the corner), c_{2n+2-i-j} on the anti-diagonals i+j = n+3..2n (lower-right
    triangle, c_2 at the corner), and 0 on the three middle anti-diagonals i+j = n, n+1, n+2."""
    i = np.arange(1, n + 1)
    s = i[:, None] + i[None, :]                      # i + j, 1-based
    upper = s <= n - 1
    lower = s >= n + 3
    H = np.zeros((n, n), dtype=np.float64)
    H[upper] = c[s[upper]]
    H[lower] = c[2 * n + 2 - s[lower]]
    return H


def tau_matrix(c: np.ndarray, n: int) -> np.ndarray:
    """tau(T_0) = T_0 - HC(T_0)  (eq. 'taudefine')."""
    return toeplitz_T0(c, n) - hankel_correction(c, n)


def dst_matrix(n: int) -> np.ndarray:
    """[S]_{ij} = sqrt(2/(n+1)) sin(pi i j/(n+1)), i, j = 1..n (orthonormal DST-I)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(k, k) / (n + 1))


def tau_eigenvalues(c: np.ndarray, n: int) -> np.ndarray:
    """Eigenvalues Lambda of tau(T_0) from its first column t (eq. 'taudiagonal').

    tau = S Lambda S and S e_1 has no zero entry, so S t = S tau e_1 = Lambda S e_1 gives
    lambda_k = (S t)_k / (S e_1)_k, k = 1..n."""
    t = tau_matrix(c, n)[:, 0]
    S = dst_matrix(n)
    return (S @ t) / S[:, 0]


def apply_S_d(u: np.ndarray, S_axes, d: int) -> np.ndarray:
    """The d-level transform S_d = S_z (x) S_y (x) S_x applied to a grid function."""
    out = u
    for a in range(d):
        out = apply_along_axis(S_axes[a], out, a, d)
    return out
