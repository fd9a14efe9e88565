"""Reverse pass on the GPU (rfnse_tape_forward / rfnse_tape_backward / rfnse_adjoint_solve) against the
oracle's reverse pass (oracle.adjoint), and the autograd wrapper against finite differences."""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import SchemeAdjoint
from oracle.operators import diag_D

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


SMALL = [
    ("1d", W.Problem(d=1, n=(63,), lo=(-10.0,), hi=(10.0,), alpha=1.5, rho=2.0, dt=0.01, tol=1e-12)),
    ("2d", W.Problem(d=2, n=(31, 15), lo=(-8.0, -6.0), hi=(8.0, 6.0), alpha=1.3, rho=1.5, dt=0.01, tol=1e-12)),
    ("3d", W.Problem(d=3, n=(15, 7, 7), lo=(-4.0,) * 3, hi=(4.0,) * 3, alpha=1.8, rho=1.0, dt=0.02, tol=1e-12)),
]


def _u0(p):
    if p.d == 1:
        return W.u0_sech_1d(p, 2.0)
    if p.d == 2:
        return W.u0_sech_product(p, [1.0, -0.5])
    return W.u0_gaussian(p, 1.0)


@pytest.mark.parametrize("first_step", (0, 1))
@pytest.mark.parametrize("nsteps,every", ((7, 3), (7, 1), (7, 10), (1, 5), (2, 1)))
@pytest.mark.parametrize("name,p", SMALL, ids=[c[0] for c in SMALL])
def test_tape_gradient_matches_oracle(name, p, nsteps, every, first_step):
    from paper_2410_03643_gb300 import Solver
    p = p.replace(first_step=first_step)
    u0 = _u0(p)
    target = u0 * (1.0 + 0.05 * W.random_field(p.shape, 21))
    L, g0_ref, grho_ref, uN_ref = SchemeAdjoint(p).gradient(u0, nsteps, target)
    s = Solver(p, precision=0)
    uN, _ = s.tape_forward(dev(u0), nsteps, every)
    assert rel(uN.cpu().numpy(), uN_ref.ravel()) < 1e-10
    gN = 2.0 * (uN - dev(target))
    g0, grho, its = s.tape_backward(gN)
    assert its >= 1
    assert rel(g0.cpu().numpy(), g0_ref.ravel()) < 1e-8
    assert abs(grho - grho_ref) <= 1e-8 * max(1.0, abs(grho_ref))
    # the context is left at the taped run's final state
    _, uc, step = s.get_state()
    assert step == nsteps and rel(uc.cpu().numpy(), uN_ref.ravel()) < 1e-10
    s.close()


def test_tape_gradient_mixed_precision():
    from paper_2410_03643_gb300 import Solver
    p = SMALL[1][1].replace(tol=1e-10)
    u0 = _u0(p)
    target = u0 * (1.0 + 0.05 * W.random_field(p.shape, 21))
    _, g0_ref, grho_ref, _ = SchemeAdjoint(p).gradient(u0, 6, target)
    s = Solver(p, precision=1)
    uN, _ = s.tape_forward(dev(u0), 6, 4)
    g0, grho, _ = s.tape_backward(2.0 * (uN - dev(target)))
    assert rel(g0.cpu().numpy(), g0_ref.ravel()) < 1e-7
    assert abs(grho - grho_ref) <= 1e-7 * max(1.0, abs(grho_ref))
    s.close()


@pytest.mark.parametrize("half", (0, 1))
def test_adjoint_solve_matches_oracle(half):
    from paper_2410_03643_gb300 import Solver
    p = SMALL[1][1]
    u = _u0(p)
    D = diag_D(u, p.rho, p.dt / (2 if half else 1))
    g = W.random_field(p.shape, 4)
    adj = SchemeAdjoint(p)
    T, P = (adj.sch.T_half, adj.sch.P_half) if half else (adj.sch.T, adj.sch.P)
    ref = adj.adjoint_solve(T, P, D, g)
    s = Solver(p, precision=0)
    lam, its, rr = s.adjoint_solve(dev(D), dev(g), bool(half))
    assert rr < p.tol and its >= 1
    assert rel(lam.cpu().numpy(), ref.ravel()) < 1e-10
    s.close()


def test_zero_steps_and_errors():
    from paper_2410_03643_gb300 import Solver, RfnseError
    p = SMALL[0][1]
    u0 = _u0(p)
    s = Solver(p, precision=0)
    with pytest.raises(RfnseError):
        s.tape_backward(dev(u0))             # nothing taped yet
    uN, _ = s.tape_forward(dev(u0), 0, 5)
    assert rel(uN.cpu().numpy(), u0) == 0.0
    g = dev(W.random_field(p.shape, 3))
    g0, grho, its = s.tape_backward(g)
    assert torch.equal(g0, g) and grho == 0.0 and its == 0
    s.close()


@pytest.mark.parametrize("first_step", (0, 1))
def test_gradient_workload_full_size(first_step):
    """The 255^2, 20-step gradient workload: the whole gradient against the oracle's, and the norm
    loss against its closed form (dL/du0 = 2 u0, dL/drho = 0)."""
    from paper_2410_03643_gb300 import Solver
    p, u0, nsteps, u0t, rho_t = W.config_adjoint()
    p = p.replace(first_step=first_step)
    s_t = Solver(p.replace(rho=rho_t), precision=0)
    target, _ = s_t.tape_forward(dev(u0t), nsteps, 5)
    s_t.close()
    s = Solver(p, precision=0)
    uN, _ = s.tape_forward(dev(u0), nsteps, 5)
    g0, grho, _ = s.tape_backward(2.0 * (uN - target))
    L_ref, g0_ref, grho_ref, _ = SchemeAdjoint(p).gradient(u0, nsteps, target.cpu().numpy())
    assert rel(g0.cpu().numpy(), g0_ref.ravel()) < 1e-8
    assert abs(grho - grho_ref) <= 1e-8 * abs(grho_ref)
    gn, grn, _ = s.tape_backward(2.0 * uN)
    assert rel(gn.cpu().numpy(), 2.0 * u0.ravel()) < 1e-9
    assert abs(grn) < 1e-8 * float(np.sum(np.abs(u0) ** 2))
    s.close()


@pytest.mark.parametrize("n", (127, 255))
def test_autograd_rollout_finite_differences(n):
    """torch.autograd through rollout() on the gradient workload (255^2, alpha = 1.5, rho = 2, dt = 0.005,
    20 steps, FP64; and the same at 127^2): 8 seeded directions in u0 and the rho direction, central
    differences with h = 1e-6 of the GPU forward, agreement to 1e-6 relative.  The solves run at tol
    1e-13 so that the forward map's own error (a jump of about tol in u^N wherever an iteration count
    changes) stays far below what h = 1e-6 resolves."""
    from paper_2410_03643_gb300 import rollout
    p, u0, nsteps, u0t, rho_t = W.config_adjoint(n=n)
    p = p.replace(tol=1e-13)
    target = rollout(p, dev(u0t), torch.tensor(rho_t, dtype=torch.float64), nsteps).detach()
    x = dev(u0).requires_grad_(True)
    rho = torch.tensor(p.rho, dtype=torch.float64, requires_grad=True)
    loss = torch.sum(torch.abs(rollout(p, x, rho, nsteps) - target) ** 2)
    loss.backward()
    g0 = x.grad.cpu().numpy()

    def L(u, r):
        with torch.no_grad():
            out = rollout(p, dev(u), torch.tensor(r, dtype=torch.float64), nsteps)
            return float(torch.sum(torch.abs(out - target) ** 2))

    h = 1e-6
    dirs, _ = W.fd_directions(p.shape, 8)
    scale = np.linalg.norm(u0)
    errs = []
    for d in dirs:
        d = d * scale
        fd = (L(u0 + h * d, p.rho) - L(u0 - h * d, p.rho)) / (2 * h)
        ad = float(np.real(np.vdot(g0, d.ravel())))
        errs.append(abs(fd - ad) / abs(fd))
    fd = (L(u0, p.rho + h) - L(u0, p.rho - h)) / (2 * h)
    errs.append(abs(fd - float(rho.grad)) / abs(fd))
    print(f"adjoint vs central differences, n = {n}: relative errors {[f'{e:.2e}' for e in errs]}")
    assert max(errs) < 1e-6, errs
