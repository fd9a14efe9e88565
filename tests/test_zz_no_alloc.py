"""rfnse_apply_prec_static: the preconditioner apply for callers that cannot call cudaMalloc.

Such callers (a plug-in whose host application owns the device memory, a real-time loop that must
not allocate once running, a program with its own allocator) get the same z = F~^{-1} v as the
context-based rfnse_apply_prec, computed with tables and intermediates in the library's static
device array instead of allocated workspace.  This file is collected last so that, should it fail,
a run that stops at the first failure has already run every other test; it also passes on its own
in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle.operators import diag_D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    L = rfnse.load_library()
    L.rfnse_apply_prec_static.argtypes = [ctypes.POINTER(rfnse.Params), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.rfnse_apply_prec_static.restype = ctypes.c_int
    return L


def _static_apply(L, params, v, D, half):
    from paper_2410_03643_gb300 import rfnse
    z = torch.full_like(v, complex(np.nan, np.nan))          # poison: every entry must be written
    st = L.rfnse_apply_prec_static(ctypes.byref(params), v.data_ptr(), z.data_ptr(), D.data_ptr(), int(half),
                                   torch.cuda.current_stream().cuda_stream)
    assert st == rfnse.RFNSE_OK
    return z


CASES = [
    (W.config_2d(1.5)[0], False),                                                       # 511 x 511, the maximum size
    (W.Problem(d=3, n=(15, 7, 31), lo=(-4.0, -3.0, -5.0), hi=(4.0, 3.0, 5.0), alpha=1.3, rho=1.0, dt=0.01), True),
    (W.Problem(d=1, n=(1023,), lo=(-20.0,), hi=(20.0,), alpha=1.9, rho=2.0, dt=0.01), False),
    # the largest axis the array's table slots hold (n = 2047, FFT length 4096) on the first axis, and
    # the smallest on the other two: every axis's table slot is written, both time levels
    (W.Problem(d=3, n=(2047, 3, 3), lo=(-20.0, -1.0, -2.0), hi=(20.0, 1.0, 2.0), alpha=1.6, rho=1.0, dt=0.01), False),
    (W.Problem(d=3, n=(2047, 3, 3), lo=(-20.0, -1.0, -2.0), hi=(20.0, 1.0, 2.0), alpha=1.6, rho=1.0, dt=0.01), True),
    (W.Problem(d=3, n=(3, 2047, 3), lo=(-1.0, -20.0, -2.0), hi=(1.0, 20.0, 2.0), alpha=1.2, rho=1.0, dt=0.01), True),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_static_entry_matches_context_entry_on_two_calls(lib, case):
    from paper_2410_03643_gb300 import rfnse
    p, half = CASES[case]
    params = rfnse.make_params(p, precision=0)
    ref_solver = rfnse.Solver(p, precision=0)
    for call in range(2):                                     # two calls in a row share the array
        v = torch.from_numpy(W.random_field(p.shape, 100 + 10 * case + call).ravel().copy()).cuda()
        D = torch.from_numpy(diag_D(W.random_field(p.shape, 200 + call), p.rho, p.dt).ravel().copy()).cuda()
        got = _static_apply(lib, params, v, D, half)
        want = ref_solver.apply_prec(v, D, half, 0)
        err = float(torch.linalg.vector_norm(got - want) / torch.linalg.vector_norm(want))
        assert err < 1e-12, (case, call, err)
    ref_solver.close()


def test_static_entry_rejects_grids_beyond_its_array(lib):
    from paper_2410_03643_gb300 import rfnse
    p = W.Problem(d=2, n=(1023, 511), lo=(-1.0, -1.0), hi=(1.0, 1.0), alpha=1.5, rho=1.0, dt=0.01)
    params = rfnse.make_params(p)
    v = torch.zeros(8, dtype=torch.complex128, device="cuda")
    D = torch.zeros(8, dtype=torch.float64, device="cuda")
    z = torch.zeros(8, dtype=torch.complex128, device="cuda")
    st = lib.rfnse_apply_prec_static(ctypes.byref(params), v.data_ptr(), z.data_ptr(), D.data_ptr(), 0, None)
    assert st == rfnse.RFNSE_EINVAL
