"""The comparators of Sec. 5 on the GPU (rfnse_params.precond = 1: the circulant TBAN preconditioner
F_C of "C-GMRES"; 2: plain GMRES) against the oracle's comparators (oracle.circulant), and the
iteration relations of Tables 5-8 on grids the CPU oracle cannot reach."""
import numpy as np
import pytest

import workloads as W
from oracle.circulant import CirculantTBANPreconditioner
from oracle.operators import diag_D, complex_to_block, block_to_complex
from oracle.scheme import SchemeOracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_03643_gb300 import build
    build.build_library()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def Solver(*a, **k):
    from paper_2410_03643_gb300 import Solver as S
    return S(*a, **k)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel().copy()).to("cuda")


def host(t, shape):
    return t.detach().cpu().numpy().reshape(shape)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300))


SMALL = [
    W.Problem(d=1, n=(255,), lo=(-20.0,), hi=(20.0,), alpha=1.5, rho=2.0, dt=0.05),
    W.Problem(d=1, n=(7,), lo=(-2.0,), hi=(2.0,), alpha=1.9, rho=1.0, dt=0.05),
    W.Problem(d=2, n=(63, 31), lo=(-6.0, -4.0), hi=(6.0, 5.0), alpha=1.7, rho=2.0, dt=0.02),
    W.Problem(d=2, n=(15, 127), lo=(-3.0, -8.0), hi=(3.0, 8.0), alpha=1.2, rho=1.0, dt=0.02),
    W.Problem(d=3, n=(15, 7, 31), lo=(-4.0, -3.0, -5.0), hi=(4.0, 3.0, 5.0), alpha=1.3, rho=1.0, dt=0.02),
]
IDS = ["1d255", "1d7", "2d63x31", "2d15x127", "3d15x7x31"]


@pytest.mark.parametrize("p", SMALL, ids=IDS)
@pytest.mark.parametrize("precision", (0, 1))
@pytest.mark.parametrize("half", (False, True))
def test_circulant_preconditioner_matches_oracle(p, precision, half):
    s = Solver(p.replace(precond=1))
    v = W.random_field(p.shape, 25)
    D = diag_D(W.random_field(p.shape, 26), p.rho, p.dt)
    got = host(s.apply_prec(dev(v), dev(D), half, precision), p.shape)
    P = CirculantTBANPreconditioner(p, p.omega, 0.5 if half else 1.0)
    want = block_to_complex(P.apply_inverse(complex_to_block(v), D))
    assert rel(got, want) < (1e-12 if precision == 0 else 5e-6)
    s.close()


@pytest.mark.parametrize("p", SMALL[:3], ids=IDS[:3])
def test_identity_preconditioner_is_the_identity(p):
    s = Solver(p.replace(precond=2))
    v = W.random_field(p.shape, 25)
    D = diag_D(W.random_field(p.shape, 26), p.rho, p.dt)
    for precision in (0, 1):
        got = host(s.apply_prec(dev(v), dev(D), False, precision), p.shape)
        assert rel(got, v) < (1e-15 if precision == 0 else 1e-7)
    s.close()


@pytest.mark.parametrize("precond", (1, 2))
@pytest.mark.parametrize("p", SMALL, ids=IDS)
@pytest.mark.parametrize("precision", (0, 1))
def test_single_solve_matches_oracle(p, precision, precond):
    p = p.replace(tol=1e-10, precond=precond, restart=256)
    s = Solver(p, precision=precision)
    u_n = W.u0_sech_product(p, [1.0] * p.d)
    D = diag_D(u_n, p.rho, p.dt)
    b = W.random_field(p.shape, 27)
    u, it, rr = s.solve(dev(D), dev(b))
    o = SchemeOracle(p)
    res = o.solve(o.T, o.P, D, b)
    got = host(u, p.shape)
    if precision == 0:
        assert rel(got, block_to_complex(res.x)) < 1e-10
        assert abs(it - res.iters) <= 1, (it, res.iters)
    else:
        assert rel(got, block_to_complex(res.x)) < 1e-8
    assert rr < p.tol
    s.close()


@pytest.mark.parametrize("precond", (1, 2))
@pytest.mark.parametrize("loop", (0, 1))
@pytest.mark.parametrize("precision", (0, 1))
def test_trajectory_matches_oracle(precision, loop, precond):
    p = SMALL[2].replace(tol=1e-10, precond=precond, restart=256)
    u0 = W.u0_sech_product(p, [1.0, 1.0])
    s = Solver(p, precision=precision, device_loop=loop)
    s.set_state(dev(u0))
    traj = torch.empty(4 * p.size, dtype=torch.complex128, device="cuda")
    iters, _ = s.run(4, traj)
    got = traj.cpu().numpy().reshape((4,) + p.shape)
    ref, its_ref, _ = SchemeOracle(p).run(u0, 4)
    for k in range(4):
        assert rel(got[k], ref[k]) < (1e-10 if precision == 0 else 1e-8), k
        if precision == 0:
            assert abs(int(iters[k]) - its_ref[k]) <= 1, (k, iters, its_ref)
    s.close()


def _second_level(n, alpha, precond, precision=0):
    """IT and solve time at the 2nd time level with the 2-D protocol of Sec. 5.2 ([-5,5]^2, rho = 1,
    Gaussian initial datum, tol 1e-8, zero initial guess; restart 256, i.e. none for these counts)."""
    p = W.Problem(d=2, n=(n, n), lo=(-5.0, -5.0), hi=(5.0, 5.0), alpha=alpha, rho=1.0, dt=0.05, tol=1e-8,
                  restart=256, precond=precond)
    s = Solver(p, precision=precision)
    s.set_state(dev(W.u0_gaussian_2d_paper(p)))
    s.run(1)
    _, u1, _ = s.get_state()
    D = (p.rho * p.dt) * torch.abs(u1) ** 2
    u0 = dev(W.u0_gaussian_2d_paper(p))
    b = -s.apply_A(u0, D) + 2j * u0           # (T - D + iI) u^0 = -(D - T + iI) u^0 + 2i u^0
    _, it, rr = s.solve(D, b)
    s.close()
    return it, rr


def test_second_level_matches_the_oracle_at_small_size():
    for precond in (0, 1, 2):
        p = W.Problem(d=2, n=(63, 63), lo=(-5.0, -5.0), hi=(5.0, 5.0), alpha=1.4, rho=1.0, dt=0.05, tol=1e-8,
                      restart=256, precond=precond)
        o = SchemeOracle(p)
        u0 = W.u0_gaussian_2d_paper(p)
        u1, _, _ = o.first_step(u0)
        D = diag_D(u1, p.rho, p.dt)
        want = o.solve(o.T, o.P, D, o.rhs(o.T, D, u0)).iters
        got, rr = _second_level(63, 1.4, precond)
        assert abs(got - want) <= 1 and rr < 1e-8, (precond, got, want)


def test_iteration_relations_of_tables_5_to_8_on_large_grids():
    """tau-GMRES flat in n, C-GMRES above it and growing, GMRES far above and growing fast, on
    127^2 .. 511^2 (n = 16129 .. 261121 unknowns)."""
    its = {pc: [_second_level(n, 1.4, pc)[0] for n in (127, 255, 511)] for pc in (0, 1)}
    plain = [_second_level(n, 1.4, 2)[0] for n in (127, 255)]
    tau, circ = its[0], its[1]
    assert max(tau) - min(tau) <= 1, tau
    assert all(t < c for t, c in zip(tau, circ)), (tau, circ)
    assert circ[-1] > circ[0], circ
    assert plain[0] > 3 * circ[0] and plain[1] > 1.5 * plain[0], plain
