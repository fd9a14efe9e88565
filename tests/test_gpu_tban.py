"""The stationary TBAN iteration (rfnse_tban_solve, Sec. 3 Method 3.1 with the practical
preconditioners as F) and the omega dependence of tau-GMRES (Fig. 1) on the GPU, against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle.circulant import make_preconditioner
from oracle.operators import diag_D, block_to_complex, rhs_block
from oracle.scheme import SchemeOracle
from oracle.tban import stationary

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_03643_gb300 import build
    build.build_library()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel().copy()).to("cuda")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CASES = [
    W.Problem(d=1, n=(255,), lo=(-20.0,), hi=(20.0,), alpha=1.5, rho=2.0, dt=0.01, tol=1e-10),
    W.Problem(d=2, n=(63, 31), lo=(-6.0, -4.0), hi=(6.0, 5.0), alpha=1.7, rho=2.0, dt=0.01, tol=1e-10),
    W.Problem(d=3, n=(15, 7, 31), lo=(-4.0, -3.0, -5.0), hi=(4.0, 3.0, 5.0), alpha=1.3, rho=1.0, dt=0.01,
              tol=1e-10),
]


@pytest.mark.parametrize("precond", (0, 1))
@pytest.mark.parametrize("half", (False, True))
@pytest.mark.parametrize("p", CASES, ids=["1d", "2d", "3d"])
def test_tban_solve_matches_oracle(p, half, precond):
    from paper_2410_03643_gb300 import Solver
    p = p.replace(precond=precond)
    scale = 0.5 if half else 1.0
    u = W.u0_sech_product(p, [1.0] * p.d) if p.d > 1 else W.u0_sech_1d(p)
    D = diag_D(u, p.rho, p.dt * scale)
    b = W.random_field(p.shape, 41)
    x, it_ref, rel_ref = stationary(p, D, rhs_block(b), make_preconditioner(p, p.omega, scale), p.tol, p.max_it,
                                    scale)
    s = Solver(p, precision=1)          # the TBAN solve is FP64 whatever the context's precision
    got, it, rr = s.tban_solve(dev(D), dev(b), half)
    assert rr < p.tol and abs(it - it_ref) <= 1, (it, it_ref)
    assert rel(got.cpu().numpy(), block_to_complex(x).ravel()) < 1e-10
    s.close()


def test_tban_solve_reports_noconvergence():
    from paper_2410_03643_gb300 import Solver, NoConvergence
    p = CASES[1].replace(max_it=2, tol=1e-14)
    s = Solver(p)
    D = diag_D(W.random_field(p.shape, 3), p.rho, p.dt)
    with pytest.raises(NoConvergence):
        s.tban_solve(dev(D), dev(W.random_field(p.shape, 4)))
    s.close()


def _second_level_it(n, alpha, omega):
    """tau-GMRES IT at the 2nd time level of the 1-D test of Sec. 5.1 ([-20,20], rho = 2,
    sech(x)e^{2ix}, tol 1e-8, no restart) with dt = 0.05."""
    from paper_2410_03643_gb300 import Solver
    p = W.Problem(d=1, n=(n,), lo=(-20.0,), hi=(20.0,), alpha=alpha, rho=2.0, dt=0.05, tol=1e-8, omega=omega,
                  restart=256)
    s = Solver(p)
    u0 = dev(W.u0_sech_1d(p, 2.0))
    s.set_state(u0)
    s.run(1)
    _, u1, _ = s.get_state()
    D = (p.rho * p.dt) * torch.abs(u1) ** 2
    b = -s.apply_A(u0, D) + 2j * u0
    _, it, rr = s.solve(D, b)
    s.close()
    assert rr < 1e-8
    return it


@pytest.mark.parametrize("omega", (0.25, 0.75, 1.0, 1.5, 3.0))
def test_omega_dependence_matches_oracle(omega):
    p = W.Problem(d=1, n=(1023,), lo=(-20.0,), hi=(20.0,), alpha=1.5, rho=2.0, dt=0.05, tol=1e-8, omega=omega,
                  restart=256)
    o = SchemeOracle(p)
    u0 = W.u0_sech_1d(p, 2.0)
    u1, _, _ = o.first_step(u0)
    D = diag_D(u1, p.rho, p.dt)
    want = o.solve(o.T, o.P, D, o.rhs(o.T, D, u0)).iters
    assert abs(_second_level_it(1023, 1.5, omega) - want) <= 1


@pytest.mark.parametrize("alpha", (1.1, 1.5, 1.9))
def test_fig_1_shape_on_a_large_grid(alpha):
    """n = 2047 (the largest 1-D grid): IT grows rapidly as w -> 0, is smallest just right of w = 1,
    grows slowly beyond."""
    omegas = (0.1, 0.5, 1.0, 1.25, 1.5, 2.0, 4.0)
    its = [_second_level_it(2047, alpha, w) for w in omegas]
    best = omegas[int(np.argmin(its))]
    assert 1.0 <= best <= 1.5, (best, its)
    assert its[0] > 5 * min(its) and its[-1] < its[0], its
