"""The C ABI library builds for sm_103a, loads, and exports every function include/rfnse.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2410_03643_gb300 import build, rfnse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rfnse_[A-Za-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return build.build_library()


def test_header_declares_the_abi():
    names = declared_functions()
    assert "rfnse_create" in names and "rfnse_run" in names and "rfnse_solve" in names
    assert set(rfnse.EXPORTED) <= set(names)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(rfnse_\w+)", out))
    assert set(declared_functions()) <= exported


def test_library_is_built_for_sm_103a(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_params_struct_matches_defaults(libpath):
    lib = rfnse.load_library()
    p = rfnse.Params()
    lib.rfnse_default_params(ctypes.byref(p))
    assert p.d == 1 and p.restart == 20 and p.max_it == 2000 and p.omega == 1.0
    assert p.tol == 1e-10 and p.first_step == 1 and p.inner_tol == 1e-6 and p.max_outer == 30
    assert p.device_loop == 1
    assert p.precond == 0


def test_create_rejects_invalid_params_without_gpu_work(libpath):
    """Validation happens before any device call, so it runs on a machine without a GPU."""
    lib = rfnse.load_library()
    bad = []
    for field, value in (("d", 0), ("d", 4), ("alpha", 1.0), ("alpha", 2.5), ("dt", 0.0), ("restart", 0),
                         ("restart", 257), ("precision", 2), ("omega", -1.0), ("tol", 0.0), ("precond", 3),
                         ("precond", -1)):
        p = rfnse.Params()
        lib.rfnse_default_params(ctypes.byref(p))
        setattr(p, field, value)
        bad.append(p)
    for n in (0, 2, 5, 100, 4095):  # n + 1 must be a power of two in [4, 2048]
        p = rfnse.Params()
        lib.rfnse_default_params(ctypes.byref(p))
        p.n[0] = n
        bad.append(p)
    for p in bad:
        h = ctypes.c_void_p()
        st = lib.rfnse_create(ctypes.byref(p), None, ctypes.byref(h))
        assert st == rfnse.RFNSE_EINVAL
        assert not h.value
        assert lib.rfnse_last_error(None)


def test_probe_arnoldi_rejects_invalid_arguments_without_gpu_work(libpath):
    """Argument checks come before any device call."""
    lib = rfnse.load_library()
    us = ctypes.c_double()
    for n, j, reps in ((0, 0, 1), (1 << 29, 0, 1), (100, -1, 1), (100, 63, 1), (100, 0, 0), (100, 0, 1001)):
        assert lib.rfnse_probe_arnoldi(n, j, reps, ctypes.byref(us), None) == rfnse.RFNSE_EINVAL
    assert lib.rfnse_probe_arnoldi(100, 0, 1, None, None) == rfnse.RFNSE_EINVAL


def test_allocation_failure_is_enomem_without_gpu_work(libpath):
    """With the allocation hook set to fail at once, rfnse_create reports ENOMEM before any device
    work, frees what it holds and hands back no context; with the limit removed, invalid parameters are
    still EINVAL (the hook does not mask validation)."""
    lib = rfnse.load_library()
    p = rfnse.Params()
    lib.rfnse_default_params(ctypes.byref(p))
    try:
        assert lib.rfnse_test_fail_allocations(0) == rfnse.RFNSE_OK
        h = ctypes.c_void_p()
        assert lib.rfnse_create(ctypes.byref(p), None, ctypes.byref(h)) == rfnse.RFNSE_ENOMEM
        assert not h.value
        assert b"allocation" in lib.rfnse_last_error(None)
    finally:
        lib.rfnse_test_fail_allocations(-1)
    p.alpha = 3.0
    h = ctypes.c_void_p()
    assert lib.rfnse_create(ctypes.byref(p), None, ctypes.byref(h)) == rfnse.RFNSE_EINVAL


def test_static_preconditioner_entry_validates_like_create_without_gpu_work(libpath):
    """rfnse_apply_prec_static refuses what rfnse_create refuses (non-finite dt, omega, rho or box) and
    grids beyond its static array, before any device call; the pointers are never dereferenced."""
    lib = rfnse.load_library()
    lib.rfnse_apply_prec_static.argtypes = [ctypes.POINTER(rfnse.Params), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.rfnse_apply_prec_static.restype = ctypes.c_int
    inf, nan = float("inf"), float("nan")
    cases = []
    for field, value in (("dt", inf), ("dt", nan), ("omega", inf), ("rho", inf), ("rho", -1.0), ("alpha", nan),
                         ("d", 0)):
        p = rfnse.Params()
        lib.rfnse_default_params(ctypes.byref(p))
        setattr(p, field, value)
        cases.append(p)
    p = rfnse.Params()
    lib.rfnse_default_params(ctypes.byref(p))
    p.hi[0] = inf
    cases.append(p)
    p = rfnse.Params()                      # N = 1023 * 511 > 262144: beyond the static array
    lib.rfnse_default_params(ctypes.byref(p))
    p.d, p.n[0], p.n[1] = 2, 1023, 511
    cases.append(p)
    dummy = ctypes.c_void_p(0x1000)
    for p in cases:
        assert lib.rfnse_apply_prec_static(ctypes.byref(p), dummy, ctypes.c_void_p(0x2000), dummy, 0,
                                           None) == rfnse.RFNSE_EINVAL
