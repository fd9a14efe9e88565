"""Debug mode (RFNSE_DEBUG=1 when the context is created): every line pass is checked after its launch.
A valid run gives the same trajectory as an ordinary context; non-finite initial data is reported as
RFNSE_ENUMERIC naming the first pass whose output held a non-finite value (without debug mode the
solver only sees it later, in the norm of the right-hand side)."""
import os

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


def _solver(p, precision, debug):
    from paper_2410_03643_gb300 import Solver
    old = os.environ.get("RFNSE_DEBUG")
    os.environ["RFNSE_DEBUG"] = "1" if debug else "0"
    try:
        return Solver(p, precision=precision)
    finally:
        if old is None:
            del os.environ["RFNSE_DEBUG"]
        else:
            os.environ["RFNSE_DEBUG"] = old


@pytest.mark.parametrize("precision", (0, 1))
@pytest.mark.parametrize("p", [
    W.Problem(d=2, n=(127, 63), lo=(-8.0, -6.0), hi=(8.0, 6.0), alpha=1.5, rho=2.0, dt=0.005),
    W.Problem(d=3, n=(31, 15, 127), lo=(-4.0, -3.0, -6.0), hi=(4.0, 3.0, 6.0), alpha=1.7, rho=1.0, dt=0.01),
], ids=["2d", "3d"])
def test_debug_mode_runs_and_names_the_first_non_finite_pass(p, precision):
    from paper_2410_03643_gb300 import rfnse
    u0 = W.u0_sech_product(p, [1.0] * p.d)
    nsteps = 3
    out = []
    for debug in (False, True):
        s = _solver(p, precision, debug)
        s.set_state(dev(u0))
        traj = torch.empty(nsteps * p.size, dtype=torch.complex128, device="cuda")
        s.run(nsteps, traj)
        out.append(traj)
        s.close()
    assert float(torch.linalg.vector_norm(out[1] - out[0]) / torch.linalg.vector_norm(out[0])) < 1e-12
    bad = np.array(u0, copy=True)
    bad.flat[5] = complex(np.nan, 0.0)
    s = _solver(p, precision, True)
    s.set_state(dev(bad))
    with pytest.raises(rfnse.RfnseError) as ei:
        s.run(1)
    assert ei.value.status == rfnse.RFNSE_ENUMERIC
    msg = str(ei.value)
    assert "non-finite output after" in msg and ("line pass" in msg or "double-float Toeplitz pass" in msg)
    s.set_state(dev(u0))                               # the context still steps
    s.run(1)
    s.close()
