"""Batched time stepping (rfnse_batch_*): many independent instances with different grids, alpha,
rho; after the first steps one graph launch advances all of them.  Every instance must match its own
single-instance run (same kernels) and the CPU oracle."""
import numpy as np
import pytest

import workloads as W
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
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300))


def _small_batch():
    rng = np.random.default_rng(7)
    out = []
    for nx, ny in ((31, 63), (15, 15), (63, 31), (127, 31), (31, 127), (7, 15)):
        alpha = float(rng.uniform(1.1, 1.95))
        rho = float(rng.uniform(0.5, 3.0))
        kx, ky = (float(v) for v in rng.uniform(-3, 3, size=2))
        p = W.Problem(d=2, n=(nx, ny), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=alpha, rho=rho, dt=0.005,
                      tol=1e-10)
        out.append((p, W.u0_sech_product(p, [kx, ky])))
    return out


@pytest.mark.parametrize("precision", (0, 1))
def test_batch_matches_single_instances_and_oracle(precision):
    from paper_2410_03643_gb300 import Batch, Solver
    inst = _small_batch()
    nsteps = 5
    b = Batch([p for p, _ in inst], precision=precision)
    for i, (p, u0) in enumerate(inst):
        b.set_state(i, dev(u0))
    iters, _ = b.run(nsteps)
    assert iters.shape == (nsteps, len(inst))
    for i, (p, u0) in enumerate(inst):
        _, uc, step = b.get_state(i)
        assert step == nsteps
        s = Solver(p, precision=precision)
        s.set_state(dev(u0))
        its_single, _ = s.run(nsteps)
        _, uc_single, _ = s.get_state()
        s.close()
        assert rel(uc.cpu().numpy(), uc_single.cpu().numpy()) < 1e-12
        assert list(iters[:, i]) == list(its_single)
        ref, its_ref, _ = SchemeOracle(p).run(u0, nsteps)
        assert rel(uc.cpu().numpy().reshape(p.shape), ref[-1]) < (1e-10 if precision == 0 else 1e-8)
        if precision == 0:
            assert all(abs(int(a) - int(r)) <= 1 for a, r in zip(iters[:, i], its_ref))
    b.close()


def test_batch_state_reload_and_continue():
    """Reloading one instance mid-run falls back to individual steps, then the batch graph again."""
    from paper_2410_03643_gb300 import Batch
    inst = _small_batch()[:3]
    b = Batch([p for p, _ in inst], precision=1)
    for i, (p, u0) in enumerate(inst):
        b.set_state(i, dev(u0))
    b.run(4)
    up, uc, step = b.get_state(1)
    b.set_state(1, uc, up, step)
    b.run(2)
    for i, (p, u0) in enumerate(inst):
        _, uc, step = b.get_state(i)
        assert step == 6
        ref, _, _ = SchemeOracle(p).run(u0, 6)
        assert rel(uc.cpu().numpy().reshape(p.shape), ref[-1]) < 1e-8
    b.close()


@pytest.mark.parametrize("precision", (1, 0))
def test_batched_workload_64_uneven_instances_every_instance(precision):
    """The 64-instance workload (n_x, n_y from {127, 255, 511}, seed 2410), 4 steps through the batch
    (from the second step on one graph launch per step for all instances): every instance's u^4 against
    the oracle, 1e-10 (FP64 form) / 1e-8 (mixed form) relative L2, iteration counts within +-1 (FP64)."""
    from paper_2410_03643_gb300 import Batch
    inst, _ = W.config_batched()
    nsteps = 4
    b = Batch([p for p, _ in inst], precision=precision)
    for i, (p, u0) in enumerate(inst):
        b.set_state(i, dev(u0))
    iters, _ = b.run(nsteps)
    assert np.all(iters >= 1)
    tol = 1e-10 if precision == 0 else 1e-8
    worst = 0.0
    for i, (p, u0) in enumerate(inst):
        _, uc, step = b.get_state(i)
        assert step == nsteps
        ref, its_ref, _ = _oracle_batched(i, nsteps)
        err = rel(uc.cpu().numpy().reshape(p.shape), ref[-1])
        worst = max(worst, err)
        assert err < tol, (i, err)
        if precision == 0:
            assert all(abs(int(a) - int(r)) <= 1 for a, r in zip(iters[:, i], its_ref)), (i, iters[:, i], its_ref)
    b.close()


_ORACLE_BATCHED = {}


def _oracle_batched(i, nsteps):
    if (i, nsteps) not in _ORACLE_BATCHED:
        inst, _ = W.config_batched()
        p, u0 = inst[i]
        _ORACLE_BATCHED[(i, nsteps)] = SchemeOracle(p).run(u0, nsteps)
    return _ORACLE_BATCHED[(i, nsteps)]
