"""Failure detection on the host, without faulting the GPU: non-finite data and allocation failures.

A non-finite value in the initial data or a right-hand side must come back as RFNSE_ENUMERIC from
rfnse_run, rfnse_solve and rfnse_batch_run (the norm checks of the solver), and an allocation failure,
provoked by the library's test hook rather than by exhausting the shared GPU's memory, as
RFNSE_ENOMEM.  After either, the context (or batch) must still work: loading valid data and stepping
again gives the same trajectory as a fresh context.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

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
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _problem(nx=31, ny=15, **kw):
    return W.Problem(d=2, n=(nx, ny), lo=(-6.0, -4.0), hi=(6.0, 4.0), alpha=1.5, rho=2.0, dt=0.01, tol=1e-10, **kw)


def _poisoned(u0, value=np.nan):
    bad = np.array(u0, copy=True)
    bad.flat[bad.size // 3] = complex(value, 0.0)
    return bad


def _reference_run(p, u0, precision, nsteps):
    from paper_2410_03643_gb300 import Solver
    s = Solver(p, precision=precision)
    s.set_state(dev(u0))
    traj = torch.empty(nsteps * p.size, dtype=torch.complex128, device="cuda")
    s.run(nsteps, traj)
    s.close()
    return traj


@pytest.mark.parametrize("precision", (0, 1))
@pytest.mark.parametrize("device_loop", (0, 1))
@pytest.mark.parametrize("value", (np.nan, np.inf))
def test_non_finite_initial_data_is_enumeric_and_the_context_stays_usable(precision, device_loop, value):
    from paper_2410_03643_gb300 import Solver, rfnse
    p = _problem()
    u0 = W.u0_sech_product(p, [1.0, 1.0])
    s = Solver(p, precision=precision, device_loop=device_loop)
    s.set_state(dev(_poisoned(u0, value)))
    with pytest.raises(rfnse.RfnseError) as ei:
        s.run(1)
    assert ei.value.status == rfnse.RFNSE_ENUMERIC
    # a regular step (n >= 1) with non-finite history is caught as well
    s.set_state(dev(_poisoned(u0, value)), dev(u0), step=3)
    with pytest.raises(rfnse.RfnseError) as ei:
        s.run(1)
    assert ei.value.status == rfnse.RFNSE_ENUMERIC
    # valid data again: the same trajectory as a fresh context
    nsteps = 3
    s.set_state(dev(u0))
    traj = torch.empty(nsteps * p.size, dtype=torch.complex128, device="cuda")
    s.run(nsteps, traj)
    s.close()
    want = _reference_run(p, u0, precision, nsteps)
    assert rel(traj, want) < 1e-13


@pytest.mark.parametrize("precision", (0, 1))
def test_non_finite_right_hand_side_of_a_solve_is_enumeric(precision):
    from paper_2410_03643_gb300 import Solver, rfnse
    p = _problem(15, 31)
    s = Solver(p, precision=precision)
    D = dev(np.abs(W.random_field(p.shape, 3)) ** 2 * p.rho * p.dt)
    b = W.random_field(p.shape, 4)
    with pytest.raises(rfnse.RfnseError) as ei:
        s.solve(D, dev(_poisoned(b)))
    assert ei.value.status == rfnse.RFNSE_ENUMERIC
    x, its, _ = s.solve(D, dev(b))          # the context still solves
    A = s.apply_A(x, D)
    assert rel(A, dev(b)) < 2e-10
    s.close()


@pytest.mark.parametrize("precision", (0, 1))
def test_non_finite_instance_of_a_batch_is_enumeric_and_the_batch_stays_usable(precision):
    """Instance 1 gets a non-finite history at a regular step.  FP64 instances at step >= 1 go straight
    to the batch graph (one launch for all), mixed ones take their first batch step one by one: both
    paths must report ENUMERIC.  Reloading valid states then gives every instance its own trajectory."""
    from paper_2410_03643_gb300 import Batch, rfnse
    probs = [_problem(31, 15), _problem(15, 31), _problem(63, 15)]
    u0s = [W.u0_sech_product(p, [1.0, -0.5]) for p in probs]
    b = Batch(probs, precision=precision)
    for i, (p, u0) in enumerate(zip(probs, u0s)):
        up = _poisoned(u0) if i == 1 else u0
        b.set_state(i, dev(u0), dev(up), step=2)
    with pytest.raises(rfnse.RfnseError) as ei:
        b.run(1)
    assert ei.value.status == rfnse.RFNSE_ENUMERIC
    assert b"instance 1" in b.lib.rfnse_batch_last_error(b.h)
    nsteps = 4
    for i, u0 in enumerate(u0s):
        b.set_state(i, dev(u0))
    b.run(nsteps)
    for i, (p, u0) in enumerate(zip(probs, u0s)):
        _, uc, step = b.get_state(i)
        assert step == nsteps
        want = _reference_run(p, u0, precision, nsteps)[(nsteps - 1) * p.size:]
        assert rel(uc, want) < 1e-12, i
    b.close()


def test_allocation_failures_are_enomem_and_leave_working_state():
    """rfnse_create, rfnse_batch_create and the reverse-pass tape each see an allocation fail part way
    through (the hook fails the k-th allocation): ENOMEM, no handle, nothing half-built; with the limit
    removed everything works again."""
    from paper_2410_03643_gb300 import Batch, Solver, rfnse
    lib = rfnse.load_library()
    p = _problem()
    u0 = W.u0_sech_product(p, [1.0, 1.0])
    try:
        for after in (0, 1, 7, 25):
            rfnse.fail_allocations_after(after)
            with pytest.raises(rfnse.RfnseError) as ei:
                Solver(p, precision=1)
            assert ei.value.status == rfnse.RFNSE_ENOMEM
            assert b"allocation" in lib.rfnse_last_error(None)
        rfnse.fail_allocations_after(-1)
        s = Solver(p, precision=1)               # enough for one context: measure what it takes
        s.close()
        # a batch whose second instance runs out
        n_one = None
        for after in range(40, 400, 40):
            rfnse.fail_allocations_after(after)
            try:
                Solver(p, precision=1).close()
                n_one = after
                break
            except rfnse.RfnseError:
                continue
        assert n_one is not None
        rfnse.fail_allocations_after(n_one + 3)
        with pytest.raises(rfnse.RfnseError) as ei:
            Batch([p, p, p], precision=1)
        assert ei.value.status == rfnse.RFNSE_ENOMEM
        rfnse.fail_allocations_after(-1)
        # the tape of the reverse pass
        s = Solver(p, precision=0)
        rfnse.fail_allocations_after(0)
        with pytest.raises(rfnse.RfnseError) as ei:
            s.tape_forward(dev(u0), 4, 2)
        assert ei.value.status == rfnse.RFNSE_ENOMEM
        rfnse.fail_allocations_after(-1)
        uN, _ = s.tape_forward(dev(u0), 4, 2)    # the context still tapes and steps
        want = _reference_run(p, u0, 0, 4)[3 * p.size:]
        assert rel(uN, want) < 1e-13
        s.close()
        b = Batch([p, p], precision=1)
        b.close()
    finally:
        rfnse.fail_allocations_after(-1)
