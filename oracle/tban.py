"""The TBAN iteration (Sec. 3, Method 3.1) -- TEST INFRASTRUCTURE.

With the TBAN splitting R_d = T_d + D_d (eq. 'TBANsplitting'; T_d = [[0, T], [-T, 0]] anti-symmetric,
D_d = [[I, -D], [D, I]] normal) Method 3.1 alternates two half-steps

    (w I + T_d) x^{k+1/2} = (w I - D_d) x^k + f,
    (w I + D_d) x^{k+1}   = (w I - T_d) x^{k+1/2} + f,

which is the fixed-point iteration F x^{k+1} = G x^k + f of the splitting R_d = F - G with
F = (1/2w)(w I + T_d)(w I + D_d), G = (1/2w)(w I - T_d)(w I - D_d) (eq. 'defpreconditionger1'),
i.e. x^{k+1} = x^k + F^{-1}(f - R_d x^k).  Theorem 3.1: it converges for every w > 0 with
rho(F^{-1} G) <= sigma(w) = sqrt(((w-1)^2 + d_max^2) / ((w+1)^2 + d_max^2)), d_max = max D.

`tban_exact` runs Method 3.1 as printed: the (w I + T_d) half-step in the complex storage u = y + i z
is (w + i T_d) u = g, solved here with a dense matrix (small grids only), and the (w I + D_d)
half-step pointwise.  `stationary` runs x^{k+1} = x^k + P^{-1}(f - R_d x^k) for any preconditioner P
of oracle.precond / oracle.circulant: with the sine-transform F~ (tau(T_d) in place of T_d inside F)
this is the stationary iteration the practical preconditioner induces, the GPU's TBAN solve.
"""
from __future__ import annotations

import numpy as np

from .operators import (ToeplitzOperator, block_R_apply, complex_to_block, block_to_complex)


def dense_T(problem, scale: float = 1.0) -> np.ndarray:
    """T_d as a dense matrix (columns T_d e_j), from the oracle's Toeplitz operator."""
    T = ToeplitzOperator(problem, scale)
    N = int(np.prod(problem.n[: problem.d]))
    cols = []
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        cols.append(T(e.reshape(problem.shape)).ravel())
    return np.array(cols).T


def tban_exact(problem, D: np.ndarray, f: np.ndarray, omega: float, iters: int, scale: float = 1.0,
               x0: np.ndarray | None = None):
    """Method 3.1 on R_d x = f (block vectors [z; y]); returns the iterates x^0 .. x^iters."""
    T = ToeplitzOperator(problem, scale)
    Td = dense_T(problem, scale)
    N = Td.shape[0]
    A_half = omega * np.eye(N) + 1j * Td                     # (w I + T_d) in the complex storage
    x = np.zeros_like(f) if x0 is None else x0.copy()
    out = [x.copy()]
    a = omega + 1.0
    for _ in range(iters):
        z, y = x[0], x[1]
        # (w I - D_d) x + f
        g = np.stack([(omega - 1.0) * z + D * y + f[0], (omega - 1.0) * y - D * z + f[1]])
        xh = complex_to_block(np.linalg.solve(A_half, block_to_complex(g).ravel()).reshape(problem.shape))
        # (w I - T_d) x^{k+1/2} + f, then the pointwise (w I + D_d) solve
        zh, yh = xh[0], xh[1]
        h = np.stack([omega * zh - T(yh) + f[0], omega * yh + T(zh) + f[1]])
        den = a * a + D * D
        x = np.stack([(a * h[0] + D * h[1]) / den, (-D * h[0] + a * h[1]) / den])
        out.append(x.copy())
    return out


def sigma_bound(omega: float, D: np.ndarray) -> float:
    """sigma(w) of Theorem 3.1."""
    dm = float(np.max(D))
    return float(np.sqrt(((omega - 1.0) ** 2 + dm * dm) / ((omega + 1.0) ** 2 + dm * dm)))


def stationary(problem, D: np.ndarray, f: np.ndarray, P, tol: float, max_it: int, scale: float = 1.0):
    """x^{k+1} = x^k + P^{-1}(f - R_d x^k) from x^0 = 0 until ||f - R_d x|| / ||f|| < tol.
    Returns (x, iterations, relative residual)."""
    T = ToeplitzOperator(problem, scale)
    fn = float(np.linalg.norm(f))
    x = np.zeros_like(f)
    if fn == 0.0:
        return x, 0, 0.0
    r = f.copy()
    k = 0
    rel = 1.0
    while k < max_it:
        x = x + P.apply_inverse(r, D)
        r = f - block_R_apply(x, T, D)
        k += 1
        rel = float(np.linalg.norm(r)) / fn
        if rel < tol:
            break
    return x, k, rel
