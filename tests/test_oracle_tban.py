"""Pins of the TBAN iteration (Sec. 3, Method 3.1; oracle.tban) against dense matrices assembled from
the block definitions, Theorem 3.1's bound, and a dense solve."""
import numpy as np
import pytest

import workloads as W
from oracle.operators import diag_D, complex_to_block
from oracle.precond import TauTBANPreconditioner
from oracle.tban import tban_exact, sigma_bound, stationary

mpmath = pytest.importorskip("mpmath")
from tests import dense_refs as R  # noqa: E402

CASES = [
    W.Problem(d=1, n=(31,), lo=(-8.0,), hi=(8.0,), alpha=1.5, rho=2.0, dt=0.05),
    W.Problem(d=2, n=(7, 9), lo=(-4.0, -3.0), hi=(4.0, 3.0), alpha=1.8, rho=1.0, dt=0.1),
]


def _setup(p):
    c = R.fcd_mp(p.alpha, max(p.n[: p.d]))
    T = R.T_dense(p, c)
    u = W.u0_sech_product(p, [1.0] * p.d) * 1.5 if p.d > 1 else W.u0_sech_1d(p) * 1.5
    D = diag_D(u, p.rho, p.dt)
    f = complex_to_block(W.random_field(p.shape, 8))
    return T, D, f


@pytest.mark.parametrize("omega", (0.5, 1.0, 2.5))
@pytest.mark.parametrize("p", CASES, ids=["1d", "2d"])
def test_one_tban_step_is_the_fixed_point_map(p, omega):
    """x^{k+1} = F^{-1}(G x^k + f) with F, G of eq. 'defpreconditionger1' built densely."""
    T, D, f = _setup(p)
    F, G, _ = R.F_G_dense(T, D.ravel(), omega)
    x0 = complex_to_block(W.random_field(p.shape, 9))
    x1 = tban_exact(p, D, f, omega, 1, x0=x0)[1]
    want = np.linalg.solve(F, G @ x0.reshape(-1) + f.reshape(-1))
    np.testing.assert_allclose(x1.reshape(-1), want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("omega", (0.5, 1.0, 2.5))
@pytest.mark.parametrize("p", CASES, ids=["1d", "2d"])
def test_tban_converges_within_theorem_3_1(p, omega):
    T, D, f = _setup(p)
    _, _, Rm = R.F_G_dense(T, D.ravel(), omega)
    xs = np.linalg.solve(Rm, f.reshape(-1))
    its = tban_exact(p, D, f, omega, 60)
    err = [np.linalg.norm(x.reshape(-1) - xs) for x in its]
    sig = sigma_bound(omega, D)
    assert sig < 1.0
    assert err[-1] <= 1e-9 * err[0] or err[-1] < 1e-12
    # the error contracts at most like sigma(w)^k (up to the constant of the similarity in the proof)
    k = 30
    assert err[k] <= 10.0 * sig ** k * err[0] + 1e-13


@pytest.mark.parametrize("p", CASES, ids=["1d", "2d"])
def test_sine_transform_stationary_iteration(p):
    """x^{k+1} = x^k + F~^{-1}(f - R x^k): converges to the dense solution, with the asymptotic rate of
    the spectral radius of I - F~^{-1} R."""
    T, D, f = _setup(p)
    c = R.fcd_mp(p.alpha, max(p.n[: p.d]))
    Ft = R.F_tilde_dense(R.tauT_dense(p, c), D.ravel(), 1.0)
    _, _, Rm = R.F_G_dense(T, D.ravel(), 1.0)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(Rm.shape[0]) - np.linalg.solve(Ft, Rm))))
    assert rho < 1.0
    x, it, rel = stationary(p, D, f, TauTBANPreconditioner(p, 1.0, 1.0), 1e-12, 500)
    xs = np.linalg.solve(Rm, f.reshape(-1))
    np.testing.assert_allclose(x.reshape(-1), xs, rtol=0, atol=1e-10 * np.abs(xs).max())
    assert rel < 1e-12
    # iterations needed by a contraction with factor rho, up to a modest constant
    assert it <= np.log(1e-12 / 50.0) / np.log(rho) + 3


def _it_omega(alpha, omega):
    from oracle.scheme import SchemeOracle
    p = W.Problem(d=1, n=(1023,), lo=(-20.0,), hi=(20.0,), alpha=alpha, rho=2.0, dt=0.05, tol=1e-8, omega=omega,
                  restart=256)
    o = SchemeOracle(p)
    u0 = W.u0_sech_1d(p, 2.0)
    u1, _, _ = o.first_step(u0)
    D = diag_D(u1, p.rho, p.dt)
    return o.solve(o.T, o.P, D, o.rhs(o.T, D, u0)).iters


@pytest.mark.parametrize("alpha", (1.1, 1.9))
def test_omega_sweep_shape_of_fig_1(alpha):
    """Fig. 1 (1-D, rho = 2, the 2nd time level): IT grows rapidly as w -> 0, reaches its minimum just
    to the right of w = 1 and grows slowly beyond."""
    omegas = (0.1, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0, 4.0)
    its = [_it_omega(alpha, w) for w in omegas]
    best = omegas[int(np.argmin(its))]
    assert 1.0 <= best <= 1.5, (best, its)
    assert its[0] > 5 * min(its)
    assert its[-1] < its[0]
    assert its[1] > its[2] > its[3] >= min(its)
