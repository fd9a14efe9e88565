"""Lock-step batches (rfnse_batch_set_lockstep): every launch of a time step covers all instances (line
passes over a work list of (instance, tile) items, one cooperative Gram-Schmidt launch, one launch per
cycle kernel).  Each instance must get the trajectory its own per-instance graph gives (up to the order
of partial sums) and the oracle's, with uneven grids, alpha, rho and convergence."""
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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def _instances(seed=11, count=5, sizes=(127, 255)):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny = (int(v) for v in rng.choice(sizes, size=2))
        alpha = float(rng.uniform(1.1, 1.95))
        rho = float(rng.uniform(0.5, 3.0))
        kx, ky = (float(v) for v in rng.uniform(-3, 3, size=2))
        p = W.Problem(d=2, n=(nx, ny), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=alpha, rho=rho, dt=0.005,
                      tol=1e-10)
        out.append((p, W.u0_sech_product(p, [kx, ky])))
    return out


def _run(inst, nsteps, lockstep, precision=1):
    from paper_2410_03643_gb300 import Batch
    b = Batch([p for p, _ in inst], precision=precision)
    assert b.lib.rfnse_batch_set_lockstep(b.h, int(lockstep)) == 0
    assert b.lib.rfnse_batch_lockstep(b.h) == int(lockstep)
    for i, (p, u0) in enumerate(inst):
        b.set_state(i, dev(u0))
    iters, _ = b.run(nsteps)
    states = [b.get_state(i)[1].cpu().numpy() for i in range(len(inst))]
    b.close()
    return states, iters


def test_lockstep_matches_per_instance_graphs_and_oracle():
    inst = _instances()
    nsteps = 6
    got, its = _run(inst, nsteps, True)
    want, its_w = _run(inst, nsteps, False)
    for i, (p, u0) in enumerate(inst):
        assert rel(got[i], want[i]) < 1e-12, i
        ref, _, _ = SchemeOracle(p).run(u0, nsteps)
        assert rel(got[i].reshape(p.shape), ref[-1]) < 1e-8, i
    assert np.all(np.abs(its.astype(int) - its_w.astype(int)) <= 1)


def test_lockstep_with_one_instance_and_with_uneven_sizes():
    """A batch of one, and a batch mixing 127, 255 and 511 per axis (three FFT lengths per pass)."""
    for inst in (_instances(seed=3, count=1), _instances(seed=5, count=4, sizes=(127, 255, 511))):
        got, _ = _run(inst, 4, True)
        for i, (p, u0) in enumerate(inst):
            ref, _, _ = SchemeOracle(p).run(u0, 4)
            assert rel(got[i].reshape(p.shape), ref[-1]) < 1e-8, i


def test_lockstep_reload_mid_run_and_switch_modes():
    """Reloading an instance with its own state keeps its cached products (the batch stays in
    lock-step); reloading it with new contents sends the batch back to per-instance first steps and
    then into the lock-step graph again; switching the mode between steps keeps every trajectory."""
    from paper_2410_03643_gb300 import Batch
    inst = _instances(seed=21, count=3)
    b = Batch([p for p, _ in inst], precision=1)
    assert b.lib.rfnse_batch_set_lockstep(b.h, 1) == 0
    for i, (p, u0) in enumerate(inst):
        b.set_state(i, dev(u0))
    b.run(3)
    up, uc, step = b.get_state(1)
    b.set_state(1, uc, up, step)
    b.run(1)
    p1, u01 = inst[1]
    ref1, _, _ = SchemeOracle(p1).run(u01, 4)
    b.set_state(1, dev(ref1[3]), dev(ref1[2]), 4)
    b.run(1)
    assert b.lib.rfnse_batch_set_lockstep(b.h, 0) == 0
    b.run(1)
    assert b.lib.rfnse_batch_set_lockstep(b.h, 1) == 0
    b.run(2)
    for i, (p, u0) in enumerate(inst):
        _, uc, step = b.get_state(i)
        assert step == 8
        ref, _, _ = SchemeOracle(p).run(u0, 8)
        assert rel(uc.cpu().numpy().reshape(p.shape), ref[-1]) < 1e-8, i
    b.close()


def test_lockstep_eligibility():
    """FP64 batches and grids without double-float residual products keep the per-instance graphs."""
    from paper_2410_03643_gb300 import Batch, rfnse
    inst = _instances(seed=2, count=2)
    b = Batch([p for p, _ in inst], precision=0)
    assert b.lib.rfnse_batch_lockstep(b.h) == 0
    assert b.lib.rfnse_batch_set_lockstep(b.h, 1) == rfnse.RFNSE_EINVAL
    b.close()
    small = W.Problem(d=2, n=(63, 127), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=1.5, rho=1.0, dt=0.005)
    b = Batch([small, inst[0][0]], precision=1)
    assert b.lib.rfnse_batch_lockstep(b.h) == 0
    b.close()
    b = Batch([inst[0][0], inst[1][0]], precision=1)
    assert b.lib.rfnse_batch_lockstep(b.h) == 0        # eligible, but few instances start per-instance
    assert b.lib.rfnse_batch_set_lockstep(b.h, 1) == 0
    assert b.lib.rfnse_batch_lockstep(b.h) == 1
    b.close()
    b = Batch([inst[0][0]] * 8, precision=1)
    assert b.lib.rfnse_batch_lockstep(b.h) == 1        # eight or more start in lock-step
    b.close()
