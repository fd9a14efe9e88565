"""The comparators of Sec. 5 -- TEST INFRASTRUCTURE: the circulant-based TBAN preconditioner F_C
("C-GMRES") and no preconditioner ("GMRES").

Sec. 5 defines

    F_C = (1/(2w)) (w I + C_d)(w I + D_d),   C_1 = [[0, C], [-C, 0]],   C_2 = [[0, C^], [-C^, 0]],
    C^ = I (x) C + C (x) I,

with C Strang's circulant approximation of T_1 = mu T_0.  Strang's circulant keeps the central
diagonals of a symmetric Toeplitz matrix and wraps them around: for T_0 with first column
c_0..c_{n-1} its first column is s_j = c_j for 0 <= j <= n/2 and s_j = c_{n-j} for n/2 < j < n (n odd
here, so the split is at (n-1)/2 and s_j = s_{n-j}).  With unequal steps each axis carries its own
mu_a (as for the tau matrix, Sec. 4), and d = 3 is the same Kronecker sum with a third term.

A circulant is diagonalised by the unitary DFT matrix [F]_{jk} = exp(-2 pi i jk/n)/sqrt(n):
C = F^H diag(lam) F with lam_k = sum_j s_j exp(-2 pi i jk/n), real because s is symmetric.  So the
block sub-solve (w I + C_d) s = r decouples, in the DFT basis, into the 2x2 systems
[[w, lam], [-lam, w]] per mode -- the same algebra as the tau sub-solve in the DST basis
(oracle.precond), with F in place of S.  The DFT is applied as a dense matrix product.
"""
from __future__ import annotations

import numpy as np

from .fcd import fcd_coefficients
from .operators import apply_along_axis
from .precond import TauTBANPreconditioner


def strang_first_column(c: np.ndarray, n: int) -> np.ndarray:
    """s_j = c_j (0 <= j <= n/2), c_{n-j} (n/2 < j < n)."""
    j = np.arange(n)
    return np.where(2 * j <= n, c[np.minimum(j, n - 1)], c[(n - j) % n]).astype(np.float64)


def strang_circulant(c: np.ndarray, n: int) -> np.ndarray:
    """Dense n x n circulant with [C]_{ij} = s_{(i-j) mod n}."""
    s = strang_first_column(c, n)
    i = np.arange(n)
    return s[(i[:, None] - i[None, :]) % n]


def dft_matrix(n: int) -> np.ndarray:
    """Unitary DFT matrix [F]_{jk} = exp(-2 pi i jk/n)/sqrt(n)."""
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n) / np.sqrt(n)


def circulant_eigenvalues(c: np.ndarray, n: int) -> np.ndarray:
    """lam_k = sum_j s_j exp(-2 pi i jk/n) = sqrt(n) (F s)_k (real: s is symmetric)."""
    lam = np.sqrt(n) * (dft_matrix(n) @ strang_first_column(c, n))
    return lam.real


def apply_F_d(u: np.ndarray, F_axes, d: int, inverse: bool = False) -> np.ndarray:
    """F_d = F_z (x) F_y (x) F_x (or its inverse F_d^H) applied to a grid function."""
    out = u.astype(np.complex128)
    for a in range(d):
        M = F_axes[a].conj().T if inverse else F_axes[a]
        out = apply_along_axis(M, out, a, d)
    return out


class CirculantTBANPreconditioner(TauTBANPreconditioner):
    """F_C^{-1} = 2w (w I + D_d)^{-1} (w I + C_d)^{-1}: the (w I + D_d) sub-solve is the tau
    preconditioner's; the other sub-solve uses the circulant in the DFT basis."""

    def __init__(self, problem, omega: float = 1.0, scale: float = 1.0):
        self.d = problem.d
        self.omega = float(omega)
        c = fcd_coefficients(problem.alpha, max(problem.n))
        self.F = [dft_matrix(problem.n[a]) for a in range(self.d)]
        mu = [scale * problem.dt / problem.h(a) ** problem.alpha for a in range(self.d)]
        lam = np.zeros(tuple(reversed(problem.n)))
        for a in range(self.d):
            la = mu[a] * circulant_eigenvalues(c, problem.n[a])
            shape = [1] * self.d
            shape[self.d - 1 - a] = problem.n[a]
            lam = lam + la.reshape(shape)
        self.Lambda = lam

    def solve_tau_block(self, r: np.ndarray) -> np.ndarray:
        """s = (w I + C_d)^{-1} r (the name follows the base class: the first block sub-solve)."""
        w = self.omega
        r1 = apply_F_d(r[0], self.F, self.d)
        r2 = apply_F_d(r[1], self.F, self.d)
        lam = self.Lambda
        den = w * w + lam * lam
        s1 = (w * r1 - lam * r2) / den
        s2 = (lam * r1 + w * r2) / den
        return np.stack([apply_F_d(s1, self.F, self.d, inverse=True).real,
                         apply_F_d(s2, self.F, self.d, inverse=True).real])


class IdentityPreconditioner:
    """No preconditioner: GMRES on R x = f itself (the paper's "GMRES" column)."""

    def apply_inverse(self, r: np.ndarray, D: np.ndarray) -> np.ndarray:
        return r


def make_preconditioner(problem, omega: float, scale: float):
    """The preconditioner a problem asks for (problem.precond: 0 tau, 1 Strang circulant, 2 none)."""
    kind = getattr(problem, "precond", 0)
    if kind == 1:
        return CirculantTBANPreconditioner(problem, omega, scale)
    if kind == 2:
        return IdentityPreconditioner()
    return TauTBANPreconditioner(problem, omega, scale)
