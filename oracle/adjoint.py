"""Reverse-mode gradient of the discrete time stepper (oracle.scheme) -- TEST INFRASTRUCTURE.

The paper has no adjoint; what is computed here is the exact derivative of its discrete scheme
(Sec. 2.1 eq. 'discretizedCNLSMaxForm', Sec. 2.2 eq. 'discretizedRFSE2DMaxForm', and the first
step read as in oracle.scheme), derived below.  The linear solves are the oracle's own
tau-preconditioned GMRES (Sec. 4, Sec. 5), applied to the conjugate system.

Convention.  A real loss L of complex states has the gradient g = dL/dRe(u) + i dL/dIm(u), so that
dL = Re(g^H du) (the real inner product of the block vectors of Sec. 3).

Step n >= 1.  M_n u^{n+1} = N_n u^{n-1} with M_n = D_n - T + iI, N_n = T - D_n + iI and
D_n = rho dt |u^n|^2.  T is real symmetric and D_n real diagonal, so M_n^T = M_n and
M_n^H = conj(M_n).  Differentiating, M_n du^{n+1} = N_n du^{n-1} - dD_n (u^{n+1} + u^{n-1}), so
for the (complete) gradient g_{n+1} of u^{n+1}:

    lambda   = M_n^{-H} g_{n+1} = conj(M_n^{-1} conj(g_{n+1}))       (one solve, same matrix)
    g_{n-1} += N_n^H lambda = (T - D_n - iI) lambda
    s_j      = -Re(conj(lambda_j) (u^{n+1}_j + u^{n-1}_j))
    g_n     += 2 rho dt s * u^n                                     (d|u|^2 = 2 Re(conj(u) du))
    dL/drho += dt sum_j |u^n_j|^2 s_j

First step (T -> T/2, D = rho (dt/2) |u~|^2).  Corrector, u~ = (u^0 + u^1*)/2 with the predictor
u^1* (first_step = 1):

    lambda_c = M_c^{-H} g_1,  g_0 += (T/2 - D_c - iI) lambda_c,  s^c = -Re(conj(lambda_c)(u^1 + u^0))
    g_u~ = rho dt s^c * u~,   dL/drho += (dt/2) sum |u~|^2 s^c,  g_0 += g_u~ / 2,  g_1* = g_u~ / 2

Predictor, D_p = rho (dt/2) |u^0|^2 (for first_step = 0 it is the whole first step, g_1* = g_1):

    lambda_p = M_p^{-H} g_1*, g_0 += (T/2 - D_p - iI) lambda_p,  s^p = -Re(conj(lambda_p)(u^1* + u^0))
    g_0 += rho dt s^p * u^0,  dL/drho += (dt/2) sum |u^0|^2 s^p

Closed form that pins this (checked in the tests): every step is the Cayley transform of a real
symmetric matrix, so ||u^N|| = ||u^0|| for any rho; L = ||u^N||^2 then has dL/du^0 = 2 u^0 and
dL/drho = 0.
"""
from __future__ import annotations

import numpy as np

from .operators import diag_D, block_to_complex
from .scheme import SchemeOracle


class SchemeAdjoint:
    """Forward run that keeps every state, and its reverse pass."""

    def __init__(self, problem):
        self.p = problem
        self.sch = SchemeOracle(problem)
        self.solve_iters = []

    # -- forward, keeping what the reverse pass reads ------------------------------------------
    def forward(self, u0: np.ndarray, nsteps: int):
        """Returns (states u^0..u^nsteps, predictor u^1* or None)."""
        p, s = self.p, self.sch
        u0 = np.asarray(u0, dtype=np.complex128).reshape(p.shape)
        states = [u0]
        pred = None
        if nsteps <= 0:
            return states, pred
        D = diag_D(u0, p.rho, p.dt / 2)
        u1 = block_to_complex(s.solve(s.T_half, s.P_half, D, s.rhs(s.T_half, D, u0)).x)
        if p.first_step == 1:
            pred = u1
            D = diag_D(0.5 * (u0 + pred), p.rho, p.dt / 2)
            u1 = block_to_complex(s.solve(s.T_half, s.P_half, D, s.rhs(s.T_half, D, u0)).x)
        states.append(u1)
        for _ in range(1, nsteps):
            u_prev, u_cur = states[-2], states[-1]
            D = diag_D(u_cur, p.rho, p.dt)
            states.append(block_to_complex(s.solve(s.T, s.P, D, s.rhs(s.T, D, u_prev)).x))
        return states, pred

    # -- pieces of the reverse pass -------------------------------------------------------------
    def adjoint_solve(self, T, P, D: np.ndarray, g: np.ndarray) -> np.ndarray:
        """lambda = M^{-H} g = conj(M^{-1} conj(g)), M = D - T + iI."""
        res = self.sch.solve(T, P, D, np.conj(g))
        self.solve_iters.append(res.iters)
        return np.conj(block_to_complex(res.x))

    @staticmethod
    def transpose_rhs(T, D: np.ndarray, lam: np.ndarray) -> np.ndarray:
        """N^H lambda = (T - D - iI) lambda."""
        return T(lam) - D * lam - 1j * lam

    @staticmethod
    def s_field(lam: np.ndarray, u_new: np.ndarray, u_old: np.ndarray) -> np.ndarray:
        """s_j = -Re(conj(lambda_j)(u_new_j + u_old_j))."""
        return -np.real(np.conj(lam) * (u_new + u_old))

    # -- reverse pass ---------------------------------------------------------------------------
    def backward(self, states, pred, grads):
        """grads: dict {step k: dL/du^k} (any subset of 0..N).  Returns (dL/du^0, dL/drho)."""
        p, sch = self.p, self.sch
        N = len(states) - 1
        g = [np.zeros(p.shape, dtype=np.complex128) for _ in range(N + 1)]
        for k, v in grads.items():
            g[k] = g[k] + np.asarray(v, dtype=np.complex128).reshape(p.shape)
        grho = 0.0
        for n in range(N - 1, 0, -1):            # step n: (u^{n-1}, u^n) -> u^{n+1}
            u_old, u_cur, u_new = states[n - 1], states[n], states[n + 1]
            D = diag_D(u_cur, p.rho, p.dt)
            lam = self.adjoint_solve(sch.T, sch.P, D, g[n + 1])
            g[n - 1] = g[n - 1] + self.transpose_rhs(sch.T, D, lam)
            s = self.s_field(lam, u_new, u_old)
            g[n] = g[n] + 2.0 * p.rho * p.dt * s * u_cur
            grho += p.dt * float(np.sum(np.abs(u_cur) ** 2 * s))
        if N >= 1:
            u0, u1 = states[0], states[1]
            g1_pred = g[1]
            if p.first_step == 1:
                ubar = 0.5 * (u0 + pred)
                D = diag_D(ubar, p.rho, p.dt / 2)
                lam = self.adjoint_solve(sch.T_half, sch.P_half, D, g[1])
                g[0] = g[0] + self.transpose_rhs(sch.T_half, D, lam)
                s = self.s_field(lam, u1, u0)
                g_bar = p.rho * p.dt * s * ubar
                grho += 0.5 * p.dt * float(np.sum(np.abs(ubar) ** 2 * s))
                g[0] = g[0] + 0.5 * g_bar
                g1_pred = 0.5 * g_bar
                u1 = pred
            D = diag_D(u0, p.rho, p.dt / 2)
            lam = self.adjoint_solve(sch.T_half, sch.P_half, D, g1_pred)
            g[0] = g[0] + self.transpose_rhs(sch.T_half, D, lam)
            s = self.s_field(lam, u1, u0)
            g[0] = g[0] + p.rho * p.dt * s * u0
            grho += 0.5 * p.dt * float(np.sum(np.abs(u0) ** 2 * s))
        return g[0], grho

    def gradient(self, u0: np.ndarray, nsteps: int, target: np.ndarray):
        """L = sum_j |u^N_j - target_j|^2: returns (L, dL/du^0, dL/drho, u^N)."""
        states, pred = self.forward(u0, nsteps)
        r = states[-1] - np.asarray(target).reshape(self.p.shape)
        L = float(np.sum(np.abs(r) ** 2))
        g0, grho = self.backward(states, pred, {len(states) - 1: 2.0 * r})
        return L, g0, grho, states[-1]
