"""The linearly implicit three-level scheme and its linear systems (paper Sec. 2, Sec. 5).

1-D (eq. 'discretizedRFSE', LICD) and 2-D (eq. 'discretizedRFSE2D', TLID); d = 3 is the same
scheme with the third Kronecker term (Sec. 2 says the method applies to d = 3):

    i (u^{n+1} - u^{n-1}) / (2 dt) - sum_a (1/h_a^alpha) sum_k c_{j-k} uhat_k + rho |u^n_j|^2 uhat_j = 0,
    uhat = (u^{n+1} + u^{n-1}) / 2.

Multiplying by 2 dt with T_d = sum_a (dt/h_a^alpha) T_0^{(a)} and D = rho dt |u^n|^2 gives the
matrix form of eq. 'discretizedCNLSMaxForm' / 'discretizedRFSE2DMaxForm':

    (D - T + iI) u^{n+1} = b^{n+1},   b^{n+1} = (T - D + iI) u^{n-1}.

The paper does not print b; this is its value from the scheme above.  Each system is solved in the
real block form R x = f of Sec. 3 by tau-preconditioned GMRES (Sec. 5 protocol, zero initial guess).

First step.  The scheme needs u^1; Sec. 5 takes it from a second-order scheme in the cited
references, which the paper does not reproduce.  Reading used here: the Crank-Nicolson step

    i (u^1 - u^0)/dt - (1/h^alpha) T_0 (u^1 + u^0)/2 + rho |u~|^2 (u^1 + u^0)/2 = 0,

which is the same linear system with mu_a -> mu_a/2 and D -> rho (dt/2) |u~|^2.  first_step = 1
(default) is predictor-corrector: u~ = u^0 gives a predictor u^1*, then u~ = (u^0 + u^1*)/2.
first_step = 0 keeps the predictor.

Invariants (derived from the scheme; they pin the oracle in the tests):
  mass   Q^n = (h^d/2)(||u^{n+1}||^2 + ||u^n||^2) is constant (each step is the Cayley transform of
         the real symmetric T - D, so ||u^{n+1}|| = ||u^{n-1}||);
  energy E^n = (h^d/2)[<L u^{n+1}, u^{n+1}> + <L u^n, u^n>] - (rho h^d/2) sum_j |u_j^{n+1}|^2 |u_j^n|^2,
         L = T_d/dt, is constant for n >= 1.
"""
from __future__ import annotations

import numpy as np

from .operators import (ToeplitzOperator, diag_D, block_R_apply, rhs_block, block_to_complex)
from .circulant import make_preconditioner
from .gmres import gmres_right, GmresResult


class SchemeOracle:
    """Time stepper for one problem (workloads.Problem)."""

    def __init__(self, problem):
        self.p = problem
        self.T = ToeplitzOperator(problem, 1.0)
        self.T_half = ToeplitzOperator(problem, 0.5)
        # the sine-transform TBAN preconditioner (Sec. 4), or a comparator of Sec. 5 (problem.precond)
        self.P = make_preconditioner(problem, problem.omega, 1.0)
        self.P_half = make_preconditioner(problem, problem.omega, 0.5)

    # -- one linear system --------------------------------------------------------------------
    def rhs(self, T: ToeplitzOperator, D: np.ndarray, u_old: np.ndarray) -> np.ndarray:
        """b = (T - D + iI) u_old (complex)."""
        return T(u_old) - D * u_old + 1j * u_old

    def solve(self, T, P, D: np.ndarray, b: np.ndarray) -> GmresResult:
        """(D - T + iI) u = b via R x = f, x = [z; y], f = [-p; q] (Sec. 3)."""
        f = rhs_block(b)
        return gmres_right(lambda x: block_R_apply(x, T, D),
                           lambda r: P.apply_inverse(r, D),
                           f, self.p.tol, self.p.restart, self.p.max_it)

    # -- time steps ---------------------------------------------------------------------------
    def first_step(self, u0: np.ndarray):
        """u^0 -> u^1 (half-step reading above).  Returns (u^1, total iterations, last relres)."""
        p = self.p
        D = diag_D(u0, p.rho, p.dt / 2)
        res = self.solve(self.T_half, self.P_half, D, self.rhs(self.T_half, D, u0))
        u1 = block_to_complex(res.x)
        its = res.iters
        if p.first_step == 1:
            ubar = 0.5 * (u0 + u1)
            D = diag_D(ubar, p.rho, p.dt / 2)
            res = self.solve(self.T_half, self.P_half, D, self.rhs(self.T_half, D, u0))
            u1 = block_to_complex(res.x)
            its += res.iters
        return u1, its, res.relres

    def step(self, u_prev: np.ndarray, u_cur: np.ndarray):
        """(u^{n-1}, u^n) -> u^{n+1}.  Returns (u^{n+1}, iterations, relres)."""
        p = self.p
        D = diag_D(u_cur, p.rho, p.dt)
        res = self.solve(self.T, self.P, D, self.rhs(self.T, D, u_prev))
        return block_to_complex(res.x), res.iters, res.relres

    def run(self, u0: np.ndarray, nsteps: int):
        """Trajectory u^1..u^nsteps with per-step iteration counts and relative residuals."""
        traj, iters, relres = [], [], []
        if nsteps <= 0:
            return traj, iters, relres
        u1, it, rr = self.first_step(u0)
        traj.append(u1); iters.append(it); relres.append(rr)
        u_prev, u_cur = u0, u1
        for _ in range(1, nsteps):
            u_next, it, rr = self.step(u_prev, u_cur)
            traj.append(u_next); iters.append(it); relres.append(rr)
            u_prev, u_cur = u_cur, u_next
        return traj, iters, relres

    # -- invariants ---------------------------------------------------------------------------
    def cell(self) -> float:
        v = 1.0
        for a in range(self.p.d):
            v *= self.p.h(a)
        return v

    def mass(self, u_next: np.ndarray, u_cur: np.ndarray) -> float:
        """Q^n = (h^d/2)(||u^{n+1}||^2 + ||u^n||^2)."""
        return 0.5 * self.cell() * float(np.sum(np.abs(u_next) ** 2) + np.sum(np.abs(u_cur) ** 2))

    def energy(self, u_next: np.ndarray, u_cur: np.ndarray) -> float:
        """E^n as in the module docstring (L = T_d / dt)."""
        p = self.p
        hd = self.cell()

        def quad(u):
            return float(np.real(np.vdot(u, self.T(u)))) / p.dt

        nl = float(np.sum(np.abs(u_next) ** 2 * np.abs(u_cur) ** 2))
        return 0.5 * hd * (quad(u_next) + quad(u_cur)) - 0.5 * p.rho * hd * nl
