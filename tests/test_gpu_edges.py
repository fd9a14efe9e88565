"""Edge cases of the grid on the GPU against the oracle: the largest supported axis (n = 2047, FFT
length 4096, which no fixed-length FFT covers), the smallest (n = 3, FFT length 8), the largest and the
smallest axis in one ragged grid, in both precisions, for single solves and short trajectories."""
import numpy as np
import pytest

import workloads as W
from oracle.operators import diag_D, block_to_complex
from oracle.scheme import SchemeOracle

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


EDGE = [
    W.Problem(d=1, n=(2047,), lo=(-20.0,), hi=(20.0,), alpha=1.5, rho=2.0, dt=0.01, tol=1e-10),
    W.Problem(d=1, n=(3,), lo=(-1.0,), hi=(1.0,), alpha=1.7, rho=1.0, dt=0.05, tol=1e-10),
    W.Problem(d=2, n=(2047, 7), lo=(-20.0, -3.0), hi=(20.0, 3.0), alpha=1.3, rho=2.0, dt=0.01, tol=1e-10),
    W.Problem(d=2, n=(3, 2047), lo=(-2.0, -20.0), hi=(2.0, 20.0), alpha=1.9, rho=1.0, dt=0.01, tol=1e-10),
    W.Problem(d=3, n=(3, 3, 3), lo=(-2.0,) * 3, hi=(2.0,) * 3, alpha=1.6, rho=1.0, dt=0.05, tol=1e-10),
    W.Problem(d=3, n=(7, 3, 255), lo=(-3.0, -2.0, -8.0), hi=(3.0, 2.0, 8.0), alpha=1.2, rho=2.0, dt=0.01,
              tol=1e-10),
]
IDS = ["1d2047", "1d3", "2d2047x7", "2d3x2047", "3d3", "3d7x3x255"]


def _u0(p):
    return W.u0_sech_product(p, [1.0] * p.d) if p.d > 1 else W.u0_sech_1d(p)


@pytest.mark.parametrize("precision", (0, 1))
@pytest.mark.parametrize("p", EDGE, ids=IDS)
def test_edge_grid_solve_and_trajectory(p, precision):
    from paper_2410_03643_gb300 import Solver
    s = Solver(p, precision=precision)
    D = diag_D(_u0(p), p.rho, p.dt)
    b = W.random_field(p.shape, 71)
    u, it, rr = s.solve(dev(D), dev(b))
    o = SchemeOracle(p)
    res = o.solve(o.T, o.P, D, b)
    tol = 1e-10 if precision == 0 else 1e-8
    assert rel(u.cpu().numpy().reshape(p.shape), block_to_complex(res.x)) < tol
    if precision == 0:
        assert abs(it - res.iters) <= 1
    s.set_state(dev(_u0(p)))
    traj = torch.empty(3 * p.size, dtype=torch.complex128, device="cuda")
    s.run(3, traj)
    ref, _, _ = o.run(_u0(p), 3)
    got = traj.cpu().numpy().reshape((3,) + p.shape)
    for k in range(3):
        assert rel(got[k], ref[k]) < tol, k
    s.close()
