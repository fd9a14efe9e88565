"""ctypes binding of the C ABI in include/rfnse.h.

Argument marshalling only: every step of the solver runs in librfnse.so.  Device buffers are torch
tensors (complex128 / float64 on a CUDA device), passed by data_ptr(); host buffers are numpy arrays.
The library must have been built (paper_2410_03643_gb300.build.build_library, or
__graft_entry__.build()); importing this module never falls back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import build as _build

RFNSE_OK, RFNSE_EINVAL, RFNSE_ENOMEM, RFNSE_ECUDA, RFNSE_ENOCONV, RFNSE_ENUMERIC, RFNSE_ETIMEOUT = range(7)
_STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENUMERIC", 6: "ETIMEOUT"}


class RfnseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rfnse {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class NoConvergence(RfnseError):
    pass


class Params(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("alpha", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("restart", ctypes.c_int),
        ("max_it", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("first_step", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int),
        ("device_loop", ctypes.c_int),
        ("precond", ctypes.c_int),
    ]


EXPORTED = ("rfnse_default_params", "rfnse_create", "rfnse_destroy", "rfnse_last_error", "rfnse_size",
            "rfnse_set_state", "rfnse_get_state", "rfnse_run", "rfnse_apply_A", "rfnse_apply_prec",
            "rfnse_dst", "rfnse_toeplitz", "rfnse_solve", "rfnse_get_coefficients", "rfnse_launch_count",
            "rfnse_profile", "rfnse_profile_read", "rfnse_probe_fma", "rfnse_probe_arnoldi", "rfnse_batch_create",
            "rfnse_batch_destroy", "rfnse_batch_last_error", "rfnse_batch_context", "rfnse_batch_run",
            "rfnse_tape_forward", "rfnse_tape_backward", "rfnse_adjoint_solve", "rfnse_tban_solve",
            "rfnse_selftest_bounded_wait", "rfnse_test_fail_allocations", "rfnse_apply_prec_static",
            "rfnse_autotune", "rfnse_tuned_launches", "rfnse_batch_autotune", "rfnse_batch_set_lockstep",
            "rfnse_batch_lockstep", "rfnse_set_arnoldi_grid", "rfnse_arnoldi_grid")

K_INSCALE, K_DST, K_LAM, K_DSCALE, K_TOEP_X, K_TOEP_ACC, K_FP32, K_DF, K_ARNOLDI = 1, 2, 4, 8, 16, 32, 256, 1024, 2048

_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load librfnse.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2410_03643_gb300.build.build_library()")
    lib = ctypes.CDLL(path)
    vp, cp, ip, dp = ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.rfnse_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.rfnse_default_params.restype = None
    lib.rfnse_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    lib.rfnse_create.restype = ip
    lib.rfnse_destroy.argtypes = [vp]
    lib.rfnse_destroy.restype = None
    lib.rfnse_last_error.argtypes = [vp]
    lib.rfnse_last_error.restype = cp
    lib.rfnse_size.argtypes = [vp]
    lib.rfnse_size.restype = ctypes.c_longlong
    lib.rfnse_set_state.argtypes = [vp, vp, vp, ip, ip]
    lib.rfnse_set_state.restype = ip
    lib.rfnse_get_state.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int), ip]
    lib.rfnse_get_state.restype = ip
    lib.rfnse_run.argtypes = [vp, ip, vp, ctypes.POINTER(ctypes.c_int), dp, ip]
    lib.rfnse_run.restype = ip
    lib.rfnse_apply_A.argtypes = [vp, vp, vp, vp, ip]
    lib.rfnse_apply_A.restype = ip
    lib.rfnse_apply_prec.argtypes = [vp, vp, vp, vp, ip, ip]
    lib.rfnse_apply_prec.restype = ip
    lib.rfnse_dst.argtypes = [vp, ip, vp, vp, ip]
    lib.rfnse_dst.restype = ip
    lib.rfnse_toeplitz.argtypes = [vp, ip, vp, vp, ip]
    lib.rfnse_toeplitz.restype = ip
    lib.rfnse_solve.argtypes = [vp, vp, vp, vp, ip, ctypes.POINTER(ctypes.c_int), dp]
    lib.rfnse_solve.restype = ip
    lib.rfnse_get_coefficients.argtypes = [vp, dp, dp]
    lib.rfnse_get_coefficients.restype = ip
    lib.rfnse_launch_count.argtypes = []
    lib.rfnse_launch_count.restype = ctypes.c_longlong
    lib.rfnse_profile.argtypes = [vp, ip]
    lib.rfnse_profile.restype = ip
    lib.rfnse_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp, dp, dp]
    lib.rfnse_profile_read.restype = ip
    lib.rfnse_probe_fma.argtypes = [ip, dp]
    lib.rfnse_probe_fma.restype = ip
    lib.rfnse_probe_arnoldi.argtypes = [ctypes.c_longlong, ip, ip, dp, ctypes.POINTER(ctypes.c_int)]
    lib.rfnse_probe_arnoldi.restype = ip
    lib.rfnse_batch_create.argtypes = [ctypes.POINTER(Params), ip, vp, ctypes.POINTER(vp)]
    lib.rfnse_batch_create.restype = ip
    lib.rfnse_batch_destroy.argtypes = [vp]
    lib.rfnse_batch_destroy.restype = None
    lib.rfnse_batch_last_error.argtypes = [vp]
    lib.rfnse_batch_last_error.restype = cp
    lib.rfnse_batch_context.argtypes = [vp, ip]
    lib.rfnse_batch_context.restype = vp
    lib.rfnse_batch_run.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), dp]
    lib.rfnse_batch_run.restype = ip
    lib.rfnse_tape_forward.argtypes = [vp, vp, ip, ip, vp, ctypes.POINTER(ctypes.c_int), ip]
    lib.rfnse_tape_forward.restype = ip
    lib.rfnse_tape_backward.argtypes = [vp, vp, vp, dp, ctypes.POINTER(ctypes.c_int), ip]
    lib.rfnse_tape_backward.restype = ip
    lib.rfnse_adjoint_solve.argtypes = [vp, vp, vp, vp, ip, ctypes.POINTER(ctypes.c_int), dp]
    lib.rfnse_adjoint_solve.restype = ip
    lib.rfnse_tban_solve.argtypes = [vp, vp, vp, vp, ip, ctypes.POINTER(ctypes.c_int), dp]
    lib.rfnse_tban_solve.restype = ip
    lib.rfnse_selftest_bounded_wait.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp]
    lib.rfnse_selftest_bounded_wait.restype = ip
    lib.rfnse_autotune.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
    lib.rfnse_autotune.restype = ip
    lib.rfnse_tuned_launches.argtypes = [vp]
    lib.rfnse_tuned_launches.restype = ctypes.c_longlong
    lib.rfnse_batch_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.rfnse_batch_autotune.restype = ip
    lib.rfnse_set_arnoldi_grid.argtypes = [vp, ip]
    lib.rfnse_set_arnoldi_grid.restype = ip
    lib.rfnse_arnoldi_grid.argtypes = [vp]
    lib.rfnse_arnoldi_grid.restype = ip
    lib.rfnse_batch_set_lockstep.argtypes = [vp, ip]
    lib.rfnse_batch_set_lockstep.restype = ip
    lib.rfnse_batch_lockstep.argtypes = [vp]
    lib.rfnse_batch_lockstep.restype = ip
    lib.rfnse_test_fail_allocations.argtypes = [ctypes.c_longlong]
    lib.rfnse_test_fail_allocations.restype = ip
    if path == _build.library_path():
        _lib = lib
    return lib


def make_params(problem, precision: int = 0, inner_tol: float = 1e-6, max_outer: int = 30,
                device_loop: int = 1) -> Params:
    """Params from a workloads.Problem."""
    p = Params()
    p.d = problem.d
    for a in range(3):
        p.n[a] = problem.n[a] if a < problem.d else 1
        p.lo[a] = problem.lo[a] if a < problem.d else 0.0
        p.hi[a] = problem.hi[a] if a < problem.d else 1.0
    p.alpha = problem.alpha
    p.rho = problem.rho
    p.dt = problem.dt
    p.omega = problem.omega
    p.restart = problem.restart
    p.max_it = problem.max_it
    p.tol = problem.tol
    p.precision = precision
    p.first_step = problem.first_step
    p.inner_tol = inner_tol
    p.max_outer = max_outer
    p.device_loop = device_loop
    p.precond = getattr(problem, "precond", 0)
    return p


def selftest_bounded_wait(stream=None):
    """Run the bounded-wait self-test: returns (error flag, kernel ms); the flag must be 1."""
    lib = load_library()
    err = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    st = lib.rfnse_selftest_bounded_wait(ctypes.c_void_p(stream.cuda_stream) if stream is not None else None,
                                         ctypes.byref(err), ctypes.byref(ms))
    if st != RFNSE_OK:
        raise RfnseError(st, "bounded-wait self-test failed to run")
    return err.value, ms.value


def fail_allocations_after(after: int) -> None:
    """After `after` more successful allocations by contexts, batches and tapes, make every later one
    fail as if the GPU were out of memory (after < 0: no limit, the default)."""
    load_library().rfnse_test_fail_allocations(int(after))


def launch_count() -> int:
    """Kernels launched by librfnse.so in this process."""
    return int(load_library().rfnse_launch_count())


def probe_fma(fp64: bool) -> float:
    """Measured FMA throughput of the current device in flop/s (FP64 or FP32)."""
    v = ctypes.c_double()
    st = load_library().rfnse_probe_fma(int(fp64), ctypes.byref(v))
    if st != RFNSE_OK:
        raise RfnseError(st, "rfnse_probe_fma failed")
    return v.value


def probe_arnoldi(n: int, j: int, reps: int = 20) -> Tuple[float, int]:
    """Mean duration in microseconds of one cooperative Arnoldi step (MGS against j + 1 basis vectors
    of n values, Givens, convergence test) and the grid size it ran with."""
    us = ctypes.c_double()
    blocks = ctypes.c_int()
    st = load_library().rfnse_probe_arnoldi(int(n), int(j), int(reps), ctypes.byref(us), ctypes.byref(blocks))
    if st != RFNSE_OK:
        raise RfnseError(st, "rfnse_probe_arnoldi failed")
    return us.value, blocks.value


def _ptr(t) -> int:
    return int(t.data_ptr())


class Solver:
    """One solver context (rfnse_create).  `stream` is a torch.cuda.Stream or None (current)."""

    def __init__(self, problem, precision: int = 0, stream=None, inner_tol: float = 1e-6, max_outer: int = 30,
                 device_loop: int = 1):
        import torch
        self.lib = load_library()
        self.problem = problem
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = make_params(problem, precision, inner_tol, max_outer, device_loop)
        h = ctypes.c_void_p()
        st = self.lib.rfnse_create(ctypes.byref(self.params), ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(h))
        if st != RFNSE_OK:
            raise RfnseError(st, self.lib.rfnse_last_error(None).decode())
        self.h = h
        self.N = int(self.lib.rfnse_size(self.h))
        self.shape = tuple(reversed(problem.n))

    def close(self):
        if getattr(self, "h", None):
            self.lib.rfnse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st == RFNSE_OK:
            return
        msg = self.lib.rfnse_last_error(self.h).decode()
        if st == RFNSE_ENOCONV:
            raise NoConvergence(st, msg)
        raise RfnseError(st, msg)

    # -- state and stepping ------------------------------------------------------------------
    def set_state(self, u_cur, u_prev=None, step: int = 0):
        """u_cur / u_prev: torch complex128 CUDA tensors of N values."""
        self._check(self.lib.rfnse_set_state(self.h, _ptr(u_prev) if u_prev is not None else None,
                                             _ptr(u_cur), step, 1))

    def set_state_host(self, u_cur: np.ndarray, u_prev: Optional[np.ndarray] = None, step: int = 0):
        uc = np.ascontiguousarray(u_cur, dtype=np.complex128)
        up = np.ascontiguousarray(u_prev, dtype=np.complex128) if u_prev is not None else None
        self._check(self.lib.rfnse_set_state(self.h, up.ctypes.data if up is not None else None,
                                             uc.ctypes.data, step, 0))

    def get_state(self):
        import torch
        up = torch.empty(self.N, dtype=torch.complex128, device="cuda")
        uc = torch.empty(self.N, dtype=torch.complex128, device="cuda")
        step = ctypes.c_int()
        self._check(self.lib.rfnse_get_state(self.h, _ptr(up), _ptr(uc), ctypes.byref(step), 1))
        return up, uc, step.value

    def run(self, nsteps: int, traj=None, allow_noconv: bool = False) -> Tuple[np.ndarray, np.ndarray]:
        """Advance nsteps; traj: optional torch complex128 CUDA tensor of nsteps*N values."""
        iters = np.zeros(max(nsteps, 1), dtype=np.int32)
        relres = np.zeros(max(nsteps, 1), dtype=np.float64)
        st = self.lib.rfnse_run(self.h, nsteps, _ptr(traj) if traj is not None else None,
                                iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                relres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1)
        if not (allow_noconv and st == RFNSE_ENOCONV):
            self._check(st)
        return iters[:nsteps], relres[:nsteps]

    def run_host(self, nsteps: int, traj: Optional[np.ndarray] = None):
        """Same as run with a host (numpy complex128) trajectory buffer."""
        iters = np.zeros(max(nsteps, 1), dtype=np.int32)
        relres = np.zeros(max(nsteps, 1), dtype=np.float64)
        st = self.lib.rfnse_run(self.h, nsteps, traj.ctypes.data if traj is not None else None,
                                iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                relres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        self._check(st)
        return iters[:nsteps], relres[:nsteps]

    # -- building blocks ---------------------------------------------------------------------
    def apply_A(self, u, D, half: bool = False):
        import torch
        out = torch.empty_like(u)
        self._check(self.lib.rfnse_apply_A(self.h, _ptr(u), _ptr(out), _ptr(D), int(half)))
        return out

    def apply_prec(self, v, D, half: bool = False, precision: int = 0):
        import torch
        out = torch.empty_like(v)
        self._check(self.lib.rfnse_apply_prec(self.h, _ptr(v), _ptr(out), _ptr(D), int(half), precision))
        return out

    def dst(self, axis: int, x, precision: int = 0):
        import torch
        out = torch.empty_like(x)
        self._check(self.lib.rfnse_dst(self.h, axis, _ptr(x), _ptr(out), precision))
        return out

    def toeplitz(self, axis: int, x, half: bool = False):
        import torch
        out = torch.empty_like(x)
        self._check(self.lib.rfnse_toeplitz(self.h, axis, _ptr(x), _ptr(out), int(half)))
        return out

    def solve(self, D, b, half: bool = False):
        """u with (D - T + iI) u = b; returns (u, iters, relres)."""
        import torch
        u = torch.empty_like(b)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        self._check(self.lib.rfnse_solve(self.h, _ptr(D), _ptr(b), _ptr(u), int(half), ctypes.byref(it),
                                         ctypes.byref(rr)))
        return u, it.value, rr.value

    def tban_solve(self, D, b, half: bool = False, allow_noconv: bool = False):
        """u with (D - T + iI) u = b by the stationary TBAN iteration; returns (u, iters, relres)."""
        import torch
        u = torch.empty_like(b)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        st = self.lib.rfnse_tban_solve(self.h, _ptr(D), _ptr(b), _ptr(u), int(half), ctypes.byref(it),
                                       ctypes.byref(rr))
        if not (allow_noconv and st == RFNSE_ENOCONV):
            self._check(st)
        return u, it.value, rr.value

    def adjoint_solve(self, D, g, half: bool = False):
        """lam = (D - T + iI)^{-H} g; returns (lam, iters, relres)."""
        import torch
        lam = torch.empty_like(g)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        self._check(self.lib.rfnse_adjoint_solve(self.h, _ptr(D), _ptr(g), _ptr(lam), int(half), ctypes.byref(it),
                                                 ctypes.byref(rr)))
        return lam, it.value, rr.value

    # -- reverse pass ------------------------------------------------------------------------
    def tape_forward(self, u0, nsteps: int, every: int = 5):
        """Taped run of nsteps from u0 (torch complex128 CUDA, N values): returns (u^N, iters)."""
        import torch
        uN = torch.empty_like(u0)
        iters = np.zeros(max(nsteps, 1), dtype=np.int32)
        self._check(self.lib.rfnse_tape_forward(self.h, _ptr(u0), nsteps, every, _ptr(uN),
                                                iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), 1))
        return uN, iters[:nsteps]

    def tape_backward(self, gN):
        """(dL/du^0, dL/drho, conjugate-solve Arnoldi steps) of the last taped run from gN = dL/du^N."""
        import torch
        g0 = torch.empty_like(gN)
        grho = ctypes.c_double()
        it = ctypes.c_int()
        self._check(self.lib.rfnse_tape_backward(self.h, _ptr(gN), _ptr(g0), ctypes.byref(grho), ctypes.byref(it), 1))
        return g0, grho.value, it.value

    def autotune(self, reps: int = 5, force: bool = False):
        """Tune the launch geometry of the solver's line passes (rfnse_autotune); returns (configurations
        tuned, configurations whose geometry changed, estimated speed-up of one launch of each)."""
        nc, ch, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.rfnse_autotune(self.h, int(reps), int(force), ctypes.byref(nc), ctypes.byref(ch),
                                            ctypes.byref(sp)))
        return nc.value, ch.value, sp.value

    def tuned_launches(self) -> int:
        return int(self.lib.rfnse_tuned_launches(self.h))

    def profile(self, kind: int):
        """Time every launch of kernel class `kind` (K_* flags; 0 = off)."""
        self._check(self.lib.rfnse_profile(self.h, kind))

    def profile_read(self):
        """(launches, device ms, algorithmic flops, algorithmic bytes) since profile()."""
        n = ctypes.c_int()
        ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.rfnse_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                                ctypes.byref(by)))
        return n.value, ms.value, fl.value, by.value

    def coefficients(self):
        nmax = max(self.problem.n[: self.problem.d])
        c = np.zeros(nmax)
        lam = np.zeros(sum(self.problem.n[: self.problem.d]))
        self._check(self.lib.rfnse_get_coefficients(self.h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                    lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return c, lam


class Batch:
    """A batch of independent instances (rfnse_batch_create): one graph launch per time step of all."""

    def __init__(self, problems, precision: int = 0, stream=None, inner_tol: float = 1e-6, max_outer: int = 30,
                 device_loop: int = 1):
        import torch
        self.lib = load_library()
        self.problems = list(problems)
        self.count = len(self.problems)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (Params * self.count)(*[make_params(p, precision, inner_tol, max_outer, device_loop)
                                      for p in self.problems])
        h = ctypes.c_void_p()
        st = self.lib.rfnse_batch_create(arr, self.count, ctypes.c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(h))
        if st != RFNSE_OK:
            raise RfnseError(st, self.lib.rfnse_batch_last_error(None).decode())
        self.h = h
        self.ctx = [ctypes.c_void_p(self.lib.rfnse_batch_context(self.h, i)) for i in range(self.count)]
        self.sizes = [int(self.lib.rfnse_size(c)) for c in self.ctx]

    def close(self):
        if getattr(self, "h", None):
            self.lib.rfnse_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, ctx=None):
        if st == RFNSE_OK:
            return
        msg = (self.lib.rfnse_last_error(ctx) if ctx is not None else self.lib.rfnse_batch_last_error(self.h)).decode()
        if st == RFNSE_ENOCONV:
            raise NoConvergence(st, msg)
        raise RfnseError(st, msg)

    def set_state(self, i: int, u_cur, u_prev=None, step: int = 0):
        self._check(self.lib.rfnse_set_state(self.ctx[i], _ptr(u_prev) if u_prev is not None else None,
                                             _ptr(u_cur), step, 1), self.ctx[i])

    def get_state(self, i: int):
        import torch
        up = torch.empty(self.sizes[i], dtype=torch.complex128, device="cuda")
        uc = torch.empty(self.sizes[i], dtype=torch.complex128, device="cuda")
        step = ctypes.c_int()
        self._check(self.lib.rfnse_get_state(self.ctx[i], _ptr(up), _ptr(uc), ctypes.byref(step), 1), self.ctx[i])
        return up, uc, step.value

    def autotune(self, reps: int = 5):
        """Tune every instance's line passes (each distinct grid once); returns (configurations tuned,
        configurations whose geometry changed), summed over the instances."""
        nc, ch = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.rfnse_batch_autotune(self.h, int(reps), ctypes.byref(nc), ctypes.byref(ch)))
        return nc.value, ch.value

    def tuned_launches(self) -> int:
        return sum(int(self.lib.rfnse_tuned_launches(c)) for c in self.ctx)

    def set_lockstep(self, on: bool):
        """Lock-step mode (one launch per pass and kernel for all instances) on or off."""
        self._check(self.lib.rfnse_batch_set_lockstep(self.h, int(on)))

    @property
    def lockstep(self) -> bool:
        return bool(self.lib.rfnse_batch_lockstep(self.h))

    def run(self, nsteps: int, allow_noconv: bool = False):
        """Advance every instance nsteps; returns (iters, relres) of shape (nsteps, count)."""
        iters = np.zeros((max(nsteps, 1), self.count), dtype=np.int32)
        relres = np.zeros((max(nsteps, 1), self.count), dtype=np.float64)
        st = self.lib.rfnse_batch_run(self.h, nsteps, iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      relres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if not (allow_noconv and st == RFNSE_ENOCONV):
            self._check(st)
        return iters[:nsteps], relres[:nsteps]


def _rollout_function():
    import torch

    class Rollout(torch.autograd.Function):
        """u^N = scheme(u^0, rho) over nsteps time steps, differentiable in u^0 and rho.  The backward
        is the library's reverse pass (one conjugate solve and one recomputed forward step per step)."""

        @staticmethod
        def forward(ctx, u0, rho, problem, nsteps, every, precision, device_loop):
            solver = Solver(problem.replace(rho=float(rho)), precision=precision, device_loop=device_loop)
            flat = u0.detach().reshape(-1).contiguous()
            uN, _ = solver.tape_forward(flat, nsteps, every)
            ctx.solver = solver
            ctx.rho_meta = (rho.dtype, rho.device)
            return uN.reshape(u0.shape)

        @staticmethod
        def backward(ctx, gN):
            g0, grho, _ = ctx.solver.tape_backward(gN.reshape(-1).contiguous())
            ctx.solver.close()
            dtype, device = ctx.rho_meta
            return (g0.reshape(gN.shape), torch.tensor(grho, dtype=dtype, device=device), None, None, None, None,
                    None)

    return Rollout


_ROLLOUT = None


def rollout(problem, u0, rho, nsteps: int, every: int = 5, precision: int = 0, device_loop: int = 1):
    """Differentiable time stepping: u^N from u0 (complex128 CUDA tensor of the grid's N values, any
    shape) and rho (a 0-d float64 tensor, may require grad); problem gives everything else.
    Gradients follow torch's convention for complex tensors (dL/dRe + i dL/dIm for a real loss)."""
    global _ROLLOUT
    if _ROLLOUT is None:
        _ROLLOUT = _rollout_function()
    return _ROLLOUT.apply(u0, rho, problem, nsteps, every, precision, device_loop)
