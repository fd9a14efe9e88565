"""Right-preconditioned restarted GMRES (paper Sec. 5: "PGMRES", zero initial guess, stop when the
l2-norm relative residual of the tested system drops below the tolerance or the iteration count
exceeds the maximum).

The algorithm is the standard one (Saad, Iterative Methods for Sparse Linear Systems, GMRES with
right preconditioning and Givens rotations), written out step by step:

    r = f - A x,  beta = ||r||,  v_1 = r / beta,  g = beta e_1
    for j = 1..m:
        w = A M^{-1} v_j
        for i = 1..j:  h_ij = <v_i, w>;  w = w - h_ij v_i          (modified Gram-Schmidt)
        h_{j+1,j} = ||w||
        apply the previous rotations to column j of H; form the rotation (c_j, s_j) that
        annihilates h_{j+1,j} (r = hypot(h_jj, h_{j+1,j}), c = h_jj/r, s = h_{j+1,j}/r);
        g_{j+1} = -s_j g_j,  g_j = c_j g_j
        stop if |g_{j+1}| / ||f|| < tol   (|g_{j+1}| is the residual norm of the current iterate)
        v_{j+1} = w / h_{j+1,j}
    y = R^{-1} g (upper triangular),  x = x + M^{-1} (V y)
    on restart, recompute the true residual r = f - A x and test it.

Vectors are the real block vectors of the paper (x = [z; y]); <a, b> is the Euclidean product.
The iteration count IT is the total number of Arnoldi steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    relres: float        # |g_{j+1}| / ||f|| at exit (or the true residual at a restart exit)
    converged: bool


def _dot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.dot(a.ravel(), b.ravel()))


def _norm(a: np.ndarray) -> float:
    return math.sqrt(_dot(a, a))


def gmres_right(apply_A, apply_Minv, f: np.ndarray, tol: float, restart: int = 20,
                max_it: int = 2000) -> GmresResult:
    """Solve A x = f by GMRES(m) with right preconditioner M, x_0 = 0."""
    fnorm = _norm(f)
    x = np.zeros_like(f)
    if fnorm == 0.0:
        return GmresResult(x, 0, 0.0, True)
    m = restart
    it = 0
    r = f.copy()
    beta = fnorm
    while True:
        if beta / fnorm < tol:
            return GmresResult(x, it, beta / fnorm, True)
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        done = False
        relres = beta / fnorm
        for j in range(m):
            w = apply_A(apply_Minv(V[j]))
            for i in range(j + 1):                      # modified Gram-Schmidt
                H[i, j] = _dot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = _norm(w)
            H[j + 1, j] = hnext
            for i in range(j):                          # previous rotations on column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rr = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / rr
            sn[j] = H[j + 1, j] / rr
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            relres = abs(g[j + 1]) / fnorm
            if relres < tol or hnext == 0.0:
                done = True
                break
            if it >= max_it:
                break
            V.append(w / hnext)
        # y = R^{-1} g by back substitution on the k x k upper triangle
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        u = np.zeros_like(f)
        for i in range(k):
            u = u + y[i] * V[i]
        x = x + apply_Minv(u)
        if done:
            return GmresResult(x, it, relres, True)
        if it >= max_it:
            return GmresResult(x, it, relres, False)
        r = f - apply_A(x)
        beta = _norm(r)
