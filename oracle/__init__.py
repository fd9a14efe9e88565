"""Plain, slow, FP64 CPU oracle for the tau-preconditioned GMRES time stepper of
"Sine-transform-based fast solvers for Riesz fractional nonlinear Schroedinger equations with
attractive nonlinearities" (Chen, Yang, Zhang; arXiv 2410.03643).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, tables or helpers); the only module both sides
read is ``workloads`` (seeded grids and initial data, no method arithmetic).

Everything here follows the paper's own formulation, in its notation:

* ``fcd``       -- the fractional centred-difference coefficients c_k (Sec. 2.1).
* ``operators`` -- the symmetric d-level Toeplitz matrix T_d, the diagonal D_d, and the real
                   2x2 block system matrix R_d = [[I, T-D], [D-T, I]] acting on x = [z; y]
                   (Sec. 2, Sec. 3 eq. 'positiveBlockForm').
* ``tau``       -- the Hankel correction, the tau matrix, the DST-I matrix S and the tau
                   eigenvalues taken from the first column (Sec. 4 eqs. 'taudefine', 'HCform',
                   'taudiagonal').
* ``precond``   -- the sine-transform TBAN preconditioner F~ = (1/2w)[wI + tau(T)](wI + D) applied
                   by its two block sub-solves (Sec. 4 eq. 'taupre', 'generalizedResEqns').
* ``gmres``     -- right-preconditioned restarted GMRES with modified Gram-Schmidt and Givens
                   rotations (Sec. 5 protocol: zero initial guess, relative-residual stop).
* ``scheme``    -- the three-level linearly implicit scheme (Sec. 2.1 eq. 'discretizedRFSE',
                   Sec. 2.2 eq. 'discretizedRFSE2D'), its first step, and the discrete mass/energy.
* ``circulant`` -- the comparators of Sec. 5: Strang's circulant TBAN preconditioner F_C (C-GMRES)
                   and no preconditioner (GMRES).
* ``tban``      -- the TBAN iteration, Method 3.1 (Sec. 3), as printed (dense half-step solves) and in
                   the stationary form x += P^{-1}(f - R x) with the practical preconditioners.
* ``adjoint``   -- the reverse-mode gradient of that discrete scheme with respect to u^0 and rho
                   (derived from the scheme; the paper has no adjoint), one conjugate solve per step.

The oracle works on the REAL block vectors x = [z; y] of the paper (u = y + i z), not on complex
vectors, so that the complex-arithmetic CUDA path and this oracle reach the same numbers by
different routes.  Transforms and Toeplitz products are dense matrix products (the plain
definitions); no FFT is used anywhere in the oracle.
"""
from . import fcd, operators, tau, precond, circulant, gmres, scheme, tban, adjoint  # noqa: F401
