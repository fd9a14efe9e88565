"""The sine-transform TBAN preconditioner (paper Sec. 4, eq. 'taupre'):

    F~_{d,w} = (1/(2w)) [w I + tau(T_d)] (w I + D_d),
    tau(T_d) = [[0, tau(T_d)], [-tau(T_d), 0]],   D_d = [[I, -D_d], [D_d, I]]   (eq. 'TBANsplitting').

Applying F~^{-1} to a residual r (the generalized residual equations, eq. 'generalizedResEqns')
means two block sub-solves (Sec. 4, "two linear subsystems with coefficient matrices
w I + T_d and w I + D_d"):

    (w I + tau(T_d)) s = r :  [[w I, tau(T_d)], [-tau(T_d), w I]] [s1; s2] = [r1; r2]
    (w I + D_d)      t = s :  [[(w+1) I, -D_d], [D_d, (w+1) I]]   [t1; t2] = [s1; s2]
    z = 2 w t.

tau(T_d) = S_d Lambda_d S_d (eq. 'taudiagonal', '2Dtau'), so the first sub-solve decouples into
2x2 systems [[w, lam], [-lam, w]] per sine mode; the second into 2x2 systems per grid point.
"""
from __future__ import annotations

import numpy as np

from .fcd import fcd_coefficients
from .tau import dst_matrix, tau_eigenvalues, apply_S_d


class TauTBANPreconditioner:
    """F~_{d,w}^{-1} for a problem (grid, alpha, dt) and a diagonal D.  `scale` multiplies every
    mu_a, exactly as in operators.ToeplitzOperator."""

    def __init__(self, problem, omega: float = 1.0, scale: float = 1.0):
        self.d = problem.d
        self.omega = float(omega)
        c = fcd_coefficients(problem.alpha, max(problem.n))
        self.S = [dst_matrix(problem.n[a]) for a in range(self.d)]
        mu = [scale * problem.dt / problem.h(a) ** problem.alpha for a in range(self.d)]
        # Lambda_d(k) = sum_a mu_a lambda^{(a)}_{k_a}  (Kronecker sum, eq. '2Dtau')
        lam = np.zeros(tuple(reversed(problem.n)))
        for a in range(self.d):
            la = mu[a] * tau_eigenvalues(c, problem.n[a])
            shape = [1] * self.d
            shape[self.d - 1 - a] = problem.n[a]
            lam = lam + la.reshape(shape)
        self.Lambda = lam

    def solve_tau_block(self, r: np.ndarray) -> np.ndarray:
        """s = (w I + tau(T_d))^{-1} r."""
        w = self.omega
        r1 = apply_S_d(r[0], self.S, self.d)
        r2 = apply_S_d(r[1], self.S, self.d)
        lam = self.Lambda
        den = w * w + lam * lam
        s1 = (w * r1 - lam * r2) / den
        s2 = (lam * r1 + w * r2) / den
        return np.stack([apply_S_d(s1, self.S, self.d), apply_S_d(s2, self.S, self.d)])

    def solve_D_block(self, s: np.ndarray, D: np.ndarray) -> np.ndarray:
        """t = (w I + D_d)^{-1} s."""
        a = self.omega + 1.0
        den = a * a + D * D
        t1 = (a * s[0] + D * s[1]) / den
        t2 = (-D * s[0] + a * s[1]) / den
        return np.stack([t1, t2])

    def apply_inverse(self, r: np.ndarray, D: np.ndarray) -> np.ndarray:
        """z = F~^{-1} r = 2w (wI + D_d)^{-1} (wI + tau(T_d))^{-1} r."""
        return 2.0 * self.omega * self.solve_D_block(self.solve_tau_block(r), D)
