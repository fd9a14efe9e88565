"""The discrete operators of the scheme (paper Sec. 2 and Sec. 3).

Grid functions are float64/complex128 numpy arrays of shape (n_z, n_y, n_x) / (n_y, n_x) /
(n_x,): axis a (0 = x, 1 = y, 2 = z) is numpy axis d-1-a, so x is fastest, matching the
column-stacking vec of Sec. 2.2.

Real block vectors x = [z; y] (Sec. 3, u = y + i z) are float64 arrays of shape (2, *grid):
x[0] = z (imaginary part of u), x[1] = y (real part of u).
"""
from __future__ import annotations

import numpy as np

from .fcd import fcd_coefficients


def toeplitz_T0(c: np.ndarray, n: int) -> np.ndarray:
    """Dense symmetric Toeplitz matrix T_0 with [T_0]_{jk} = c_{j-k} = c_{|j-k|}
    (Sec. 2.1, eq. 'equ2')."""
    idx = np.arange(n)
    return c[np.abs(idx[:, None] - idx[None, :])].astype(np.float64)


def apply_along_axis(M: np.ndarray, u: np.ndarray, a: int, d: int) -> np.ndarray:
    """Apply the n_a x n_a matrix M along grid axis a of u (a dense matrix product)."""
    ax = d - 1 - a
    moved = np.moveaxis(u, ax, -1)
    out = moved @ M.T
    return np.moveaxis(out, -1, ax)


class ToeplitzOperator:
    """T_d = sum_a mu_a T_0^{(a)} acting along axis a, with mu_a = dt / h_a^alpha.

    d = 1: T_1 = mu T_0 (Sec. 2.1).  d = 2: T_2 = I (x) T_x + T_y (x) I on vec(U) (Sec. 2.2,
    eq. '2DToeplitz'), i.e. T_x acts on the first (x) index.  d = 3 is the same Kronecker sum with
    a third term (the paper states the method applies to d = 3, Sec. 2).  `scale` multiplies every
    mu_a (the first time step uses scale = 1/2)."""

    def __init__(self, problem, scale: float = 1.0):
        self.d = problem.d
        self.n = tuple(problem.n)
        nmax = max(self.n)
        self.c = fcd_coefficients(problem.alpha, nmax)
        self.mu = [scale * problem.dt / problem.h(a) ** problem.alpha for a in range(self.d)]
        self.T0 = [toeplitz_T0(self.c, self.n[a]) for a in range(self.d)]

    def __call__(self, u: np.ndarray) -> np.ndarray:
        out = np.zeros_like(u)
        for a in range(self.d):
            out = out + self.mu[a] * apply_along_axis(self.T0[a], u, a, self.d)
        return out


def diag_D(u_n: np.ndarray, rho: float, dt: float) -> np.ndarray:
    """Diagonal of D_d^{n+1} = rho dt diag(|u^n|^2) (Sec. 2.1 after eq. 'discretizedCNLSMaxForm';
    Sec. 2.2: rho dt diag(vec(conj(U^n) . U^n)))."""
    return (rho * dt * (u_n.real ** 2 + u_n.imag ** 2)).astype(np.float64)


def block_R_apply(x: np.ndarray, T: ToeplitzOperator, D: np.ndarray) -> np.ndarray:
    """R_d x for x = [z; y]  (Sec. 3, eq. 'positiveBlockForm'):

        R_d = [[ I,      T_d - D_d ],
               [ D_d - T_d,  I      ]]
    """
    z, y = x[0], x[1]
    top = z + T(y) - D * y
    bot = D * z - T(z) + y
    return np.stack([top, bot])


def complex_to_block(u: np.ndarray) -> np.ndarray:
    """u = y + i z  ->  x = [z; y]  (Sec. 3)."""
    return np.stack([u.imag.astype(np.float64), u.real.astype(np.float64)])


def block_to_complex(x: np.ndarray) -> np.ndarray:
    """x = [z; y]  ->  u = y + i z."""
    return (x[1] + 1j * x[0]).astype(np.complex128)


def rhs_block(b: np.ndarray) -> np.ndarray:
    """b = p + i q  ->  f = [-p; q]  (Sec. 3, eq. 'positiveBlockForm')."""
    return np.stack([-b.real.astype(np.float64), b.imag.astype(np.float64)])
