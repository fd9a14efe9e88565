"""Pins of the oracle's reverse pass (oracle.adjoint) against routes that share none of its code:

* central finite differences of a brute-force forward run that assembles the dense matrices of the
  scheme (coefficients from the Gamma formula in 50-digit arithmetic, np.kron) and solves each step
  with numpy.linalg.solve;
* the closed form of the norm loss: every step is a Cayley transform of a real symmetric matrix, so
  ||u^N|| = ||u^0|| for all rho, and L = ||u^N||^2 has dL/du^0 = 2 u^0 and dL/drho = 0.
"""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import SchemeAdjoint

mpmath = pytest.importorskip("mpmath")
from tests import dense_refs as R  # noqa: E402


def dense_forward(p, u0, nsteps):
    """The scheme of Sec. 2 with dense matrices and direct solves (first step as the oracle reads it)."""
    c = R.fcd_mp(p.alpha, max(p.n))
    T = R.T_dense(p, c, 1.0)
    Th = R.T_dense(p, c, 0.5)
    I = np.eye(T.shape[0])

    def step(Tm, D, u_old):
        M = np.diag(D) - Tm + 1j * I
        Nm = Tm - np.diag(D) + 1j * I
        return np.linalg.solve(M, Nm @ u_old)

    u0 = np.asarray(u0, dtype=np.complex128).ravel()
    if nsteps == 0:
        return u0
    u1 = step(Th, p.rho * (p.dt / 2) * np.abs(u0) ** 2, u0)
    if p.first_step == 1:
        u1 = step(Th, p.rho * (p.dt / 2) * np.abs(0.5 * (u0 + u1)) ** 2, u0)
    prev, cur = u0, u1
    for _ in range(1, nsteps):
        prev, cur = cur, step(T, p.rho * p.dt * np.abs(cur) ** 2, prev)
    return cur


CASES = [
    ("1d", W.Problem(d=1, n=(15,), lo=(-8.0,), hi=(8.0,), alpha=1.5, rho=2.0, dt=0.02, tol=1e-13), 5),
    ("2d", W.Problem(d=2, n=(7, 5), lo=(-5.0, -4.0), hi=(5.0, 4.0), alpha=1.3, rho=1.5, dt=0.03, tol=1e-13), 4),
    # large dt and rho: the predictor differs visibly from u^1, which a mistake in its terms shows
    ("1d-strong", W.Problem(d=1, n=(15,), lo=(-6.0,), hi=(6.0,), alpha=1.5, rho=4.0, dt=0.25, tol=1e-13), 2),
    ("3d", W.Problem(d=3, n=(5, 3, 3), lo=(-3.0,) * 3, hi=(3.0,) * 3, alpha=1.8, rho=1.0, dt=0.05, tol=1e-13), 3),
]


def _u0(p):
    if p.d == 1:
        return W.u0_sech_1d(p, 2.0) * (1.5 if p.dt > 0.1 else 1.0)
    if p.d == 2:
        return W.u0_sech_product(p, [1.0, -0.5])
    return W.u0_gaussian(p, 1.0)


@pytest.mark.parametrize("first_step", (0, 1))
@pytest.mark.parametrize("name,p,nsteps", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_dense_finite_differences(name, p, nsteps, first_step):
    p = p.replace(first_step=first_step)
    u0 = _u0(p)
    target = W.random_field(p.shape, 11) * 0.1 + u0
    L, g0, grho, uN = SchemeAdjoint(p).gradient(u0, nsteps, target)
    # the oracle's forward agrees with the dense forward
    np.testing.assert_allclose(uN.ravel(), dense_forward(p, u0, nsteps), rtol=0, atol=1e-11)

    def loss(u, rho):
        q = p.replace(rho=rho)
        return float(np.sum(np.abs(dense_forward(q, u, nsteps) - target.ravel()) ** 2))

    h = 1e-6
    dirs, rdirs = W.fd_directions(p.shape, 4, seed=643)
    for d in dirs:
        fd = (loss(u0 + h * d, p.rho) - loss(u0 - h * d, p.rho)) / (2 * h)
        ad = float(np.real(np.vdot(g0, d)))
        assert abs(fd - ad) <= 1e-7 * max(1.0, abs(fd)), (fd, ad)
    fd = (loss(u0, p.rho + h) - loss(u0, p.rho - h)) / (2 * h)
    assert abs(fd - grho) <= 1e-7 * max(1.0, abs(fd)), (fd, grho)


@pytest.mark.parametrize("first_step", (0, 1))
def test_adjoint_norm_loss_closed_form(first_step):
    """L = ||u^N||^2 = ||u^0||^2 for every rho: dL/du^0 = 2 u^0, dL/drho = 0."""
    p = W.Problem(d=2, n=(15, 15), lo=(-6.0, -6.0), hi=(6.0, 6.0), alpha=1.6, rho=3.0, dt=0.02, tol=1e-13,
                  first_step=first_step)
    u0 = W.u0_sech_product(p, [1.0, 2.0]) * 1.5
    adj = SchemeAdjoint(p)
    for nsteps in (1, 2, 7):
        states, pred = adj.forward(u0, nsteps)
        assert abs(np.linalg.norm(states[-1]) - np.linalg.norm(u0)) < 1e-11
        g0, grho = adj.backward(states, pred, {nsteps: 2.0 * states[-1]})
        np.testing.assert_allclose(g0, 2.0 * u0, rtol=0, atol=1e-10)
        assert abs(grho) < 1e-9


def test_adjoint_zero_steps_and_intermediate_losses():
    """N = 0: the loss sees u^0 directly.  A loss on two states is the sum of the two gradients."""
    p = CASES[1][1]
    u0 = _u0(p)
    t = W.random_field(p.shape, 5)
    L, g0, grho, _ = SchemeAdjoint(p).gradient(u0, 0, t)
    np.testing.assert_allclose(g0, 2.0 * (u0 - t), rtol=0, atol=1e-15)
    assert grho == 0.0
    adj = SchemeAdjoint(p)
    states, pred = adj.forward(u0, 4)
    ga, ra = adj.backward(states, pred, {4: states[4]})
    gb, rb = adj.backward(states, pred, {2: states[2]})
    gc, rc = adj.backward(states, pred, {4: states[4], 2: states[2]})
    np.testing.assert_allclose(gc, ga + gb, rtol=0, atol=1e-12)
    assert abs(rc - (ra + rb)) < 1e-12


def test_adjoint_linear_case_is_the_propagator_transpose():
    """rho = 0: u^N = Phi u^0 with a complex linear Phi built column by column from the dense forward;
    the gradient of L = Re(c^H u^N) is Phi^H c."""
    p = CASES[1][1].replace(rho=0.0)
    N = int(np.prod(p.n))
    Phi = np.stack([dense_forward(p, np.eye(N)[:, k].astype(np.complex128), 3) for k in range(N)], axis=1)
    c = W.random_field(N, 9)
    adj = SchemeAdjoint(p)
    states, pred = adj.forward(np.zeros(p.shape, dtype=np.complex128), 3)
    g0, grho = adj.backward(states, pred, {3: c.reshape(p.shape)})
    np.testing.assert_allclose(g0.ravel(), Phi.conj().T @ c, rtol=0, atol=1e-11)
