"""Pins of the oracle's comparators (oracle.circulant, Sec. 5): Strang's circulant and the circulant
TBAN preconditioner F_C against dense constructions and library routines, plain GMRES against a dense
solve, and the iteration relations the paper prints in Tables 1-8."""
import os

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle.circulant import (strang_first_column, strang_circulant, circulant_eigenvalues, dft_matrix,
                              CirculantTBANPreconditioner, make_preconditioner)
from oracle.fcd import fcd_coefficients
from oracle.operators import diag_D, complex_to_block, block_to_complex
from oracle.scheme import SchemeOracle

mpmath = pytest.importorskip("mpmath")
from tests import dense_refs as R  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", (7, 15, 63))
def test_strang_circulant_keeps_the_central_band_of_T0(n):
    c = R.fcd_mp(1.6, n)
    C = strang_circulant(c, n)
    T0 = R.toeplitz_dense(c, n)
    i = np.arange(n)
    band = np.abs(i[:, None] - i[None, :]) <= (n - 1) // 2
    np.testing.assert_allclose(C[band], T0[band], rtol=0, atol=1e-15)
    np.testing.assert_allclose(C, scipy.linalg.circulant(C[:, 0]), rtol=0, atol=0)   # circulant
    np.testing.assert_allclose(C, C.T, rtol=0, atol=0)                               # symmetric
    s = strang_first_column(c, n)
    np.testing.assert_allclose(s[1:], s[1:][::-1], rtol=0, atol=0)


@pytest.mark.parametrize("n", (7, 31, 255))
def test_circulant_eigenvalues_match_fft_and_eigensolver(n):
    c = fcd_coefficients(1.3, n)
    lam = circulant_eigenvalues(c, n)
    np.testing.assert_allclose(lam, np.fft.fft(strang_first_column(c, n)).real, rtol=0, atol=2e-12)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(strang_circulant(c, n)), rtol=0, atol=1e-12)
    F = dft_matrix(n)
    np.testing.assert_allclose(F.conj().T @ np.diag(lam) @ F, strang_circulant(c, n), rtol=0, atol=1e-12)


@pytest.mark.parametrize("omega,scale", ((0.5, 1.0), (1.0, 1.0), (2.0, 1.0), (1.0, 0.5)))
@pytest.mark.parametrize("dims", ((15,), (7, 5), (5, 3, 7)))
def test_circulant_preconditioner_matches_dense_solve(dims, omega, scale):
    """F_C = (1/2w)(wI + C_d)(wI + D_d) assembled from its block definition (Sec. 5) with Strang's
    circulants built by scipy from their first columns (scale 1/2: the first step's mu_a / 2)."""
    d = len(dims)
    p = W.Problem(d=d, n=dims, lo=(-4.0,) * d, hi=(4.0,) * d, alpha=1.7, rho=1.5, dt=0.05)
    c = R.fcd_mp(p.alpha, max(dims))
    mats = []
    for a in range(d):
        n = dims[a]
        s = np.array([c[j] if 2 * j <= n else c[n - j] for j in range(n)])
        mats.append(scale * p.dt / p.h(a) ** p.alpha * scipy.linalg.circulant(s))
    Chat = R.kron_sum(mats)
    u = W.random_field(p.shape, 3)
    D = diag_D(u, p.rho, p.dt)
    F = R.F_tilde_dense(Chat, D.ravel(), omega)
    r = complex_to_block(W.random_field(p.shape, 4))
    ref = np.linalg.solve(F, r.reshape(-1)).reshape(r.shape)
    got = CirculantTBANPreconditioner(p, omega, scale).apply_inverse(r, D)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_plain_gmres_solves_the_system():
    p = W.Problem(d=2, n=(15, 7), lo=(-5.0, -5.0), hi=(5.0, 5.0), alpha=1.5, rho=1.0, dt=0.05, tol=1e-12,
                  restart=256, precond=2)
    assert type(make_preconditioner(p, 1.0, 1.0)).__name__ == "IdentityPreconditioner"
    o = SchemeOracle(p)
    u = W.u0_gaussian_2d_paper(p)
    D = diag_D(u, p.rho, p.dt)
    b = o.rhs(o.T, D, u)
    res = o.solve(o.T, o.P, D, b)
    c = R.fcd_mp(p.alpha, 15)
    M = np.diag(D.ravel()) - R.T_dense(p, c) + 1j * np.eye(D.size)
    np.testing.assert_allclose(block_to_complex(res.x).ravel(), np.linalg.solve(M, b.ravel()), rtol=0, atol=1e-10)


def _second_level_iters(alpha, n, precond):
    """IT at the 2nd time level with the 2-D protocol of Sec. 5.2 ([-5,5]^2, rho = 1, the Gaussian
    initial datum, tol 1e-8, zero initial guess, no restart); dt = 1/20 as in Fig. 8."""
    p = W.Problem(d=2, n=(n, n), lo=(-5.0, -5.0), hi=(5.0, 5.0), alpha=alpha, rho=1.0, dt=0.05, tol=1e-8,
                  restart=256, precond=precond)
    o = SchemeOracle(p)
    u0 = W.u0_gaussian_2d_paper(p)
    u1, _, _ = o.first_step(u0)
    D = diag_D(u1, p.rho, p.dt)
    res = o.solve(o.T, o.P, D, o.rhs(o.T, D, u0))
    assert res.relres < 1e-8
    return res.iters


def test_paper_fixture_states_the_relations():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "comparator_iterations.txt")) if not l.startswith("#")]
    rows = [(int(a), int(b), float(c), int(d), int(e), int(f)) for a, b, c, d, e, f in rows]
    assert len(rows) == 40
    for dim, size, alpha, it_tau, it_c, it_g in rows:
        if it_c > 0:
            assert it_tau < it_c
        if it_g > 0:
            assert it_c < it_g
    # GMRES roughly doubles when the size doubles (1-D, alpha = 1.2) or quadruples (2-D)
    g1 = [r[5] for r in rows if r[0] == 1 and r[2] == 1.2 and r[5] > 0]
    assert all(1.8 < b / a < 2.4 for a, b in zip(g1, g1[1:]))


@pytest.mark.parametrize("alpha", (1.2, 1.4))
def test_oracle_reproduces_the_relations_of_tables_5_to_8(alpha):
    it = {pc: [_second_level_iters(alpha, n, pc) for n in (31, 63, 127)] for pc in (0, 1, 2)}
    tau, circ, plain = it[0], it[1], it[2]
    assert max(tau) - min(tau) <= 1                               # flat in the mesh size
    assert all(t <= c < g for t, c, g in zip(tau, circ, plain))    # tau <= C-GMRES < GMRES
    assert circ[-1] > circ[0]                                     # C-GMRES grows with n
    assert all(b > 1.5 * a for a, b in zip(plain, plain[1:]))     # GMRES grows with n


def test_circulant_iterations_grow_with_alpha():
    circ = [_second_level_iters(a, 63, 1) for a in (1.2, 1.5, 1.8)]
    tau = [_second_level_iters(a, 63, 0) for a in (1.2, 1.5, 1.8)]
    assert circ[0] <= circ[1] <= circ[2] and circ[2] > circ[0]
    assert max(tau) - min(tau) <= 1
