"""Seeded synthetic workloads: grids, closed-form initial data and sampled instance parameters.

This module is shared by the tests, the benchmark and the oracle's callers.  It holds none of the
method's arithmetic (no difference coefficients, transforms, operators or solves): only the problem
statements — box, interior grid, time step, initial data — that both the CUDA path and the CPU
oracle take as inputs.

Grid convention (paper Sec. 2.1 and 2.2): an interval [lo, hi] split into n+1 equal parts,
h = (hi - lo)/(n + 1), interior points x_j = lo + j*h for j = 1..n, u = 0 on the boundary.

Array layout: a d-dimensional grid function is a complex128 numpy array of shape
(n_z, n_y, n_x) / (n_y, n_x) / (n_x,) — x is the fastest (last) axis, which is the column-stacking
``vec`` order of Sec. 2.2 (first index fastest).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Problem:
    """One RFNSE instance: grid, model parameters and solver settings.

    n, lo, hi are per axis in the order (x, y, z)."""

    d: int
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    alpha: float
    rho: float
    dt: float
    omega: float = 1.0
    restart: int = 20
    max_it: int = 2000
    tol: float = 1e-10
    first_step: int = 1  # 1 = predictor-corrector half step, 0 = predictor only
    precond: int = 0     # 0 = sine-transform (tau) TBAN, 1 = Strang-circulant TBAN, 2 = none

    def h(self, a: int) -> float:
        return (self.hi[a] - self.lo[a]) / (self.n[a] + 1)

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape, slowest axis first (z, y, x)."""
        return tuple(reversed(self.n))

    @property
    def size(self) -> int:
        return int(np.prod(self.n))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def grid_axis(lo: float, hi: float, n: int) -> np.ndarray:
    """Interior nodes lo + j*h, j = 1..n, h = (hi-lo)/(n+1)."""
    h = (hi - lo) / (n + 1)
    return lo + h * np.arange(1, n + 1, dtype=np.float64)


def mesh(p: Problem):
    """Coordinate arrays broadcast to p.shape; returned in axis order (x, y, z)."""
    axes = [grid_axis(p.lo[a], p.hi[a], p.n[a]) for a in range(p.d)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")  # (z, y, x) order
    return list(reversed(grids))


def sech(x):
    return 1.0 / np.cosh(x)


def u0_sech_1d(p: Problem, k: float = 2.0) -> np.ndarray:
    """sech(x) exp(i k x) — the 1-D test of Sec. 5.1 (k = 2)."""
    (x,) = mesh(p)
    return (sech(x) * np.exp(1j * k * x)).astype(np.complex128)


def u0_sech_product(p: Problem, slopes: Sequence[float] | None = None) -> np.ndarray:
    """prod_a sech(x_a) * exp(i sum_a k_a x_a); slopes default to 1 on every axis."""
    xs = mesh(p)
    if slopes is None:
        slopes = [1.0] * p.d
    amp = np.ones(p.shape)
    phase = np.zeros(p.shape)
    for a, x in enumerate(xs):
        amp = amp * sech(x)
        phase = phase + slopes[a] * x
    return (amp * np.exp(1j * phase)).astype(np.complex128)


def u0_gaussian(p: Problem, k1: float = 1.0) -> np.ndarray:
    """exp(-|x|^2/2) exp(i k1 x_1)."""
    xs = mesh(p)
    r2 = sum(x * x for x in xs)
    return (np.exp(-0.5 * r2) * np.exp(1j * k1 * xs[0])).astype(np.complex128)


def u0_gaussian_2d_paper(p: Problem) -> np.ndarray:
    """(2/sqrt(pi)) exp(-(x^2+y^2)) — the 2-D test of Sec. 5.2."""
    xs = mesh(p)
    r2 = sum(x * x for x in xs)
    return ((2.0 / math.sqrt(math.pi)) * np.exp(-r2)).astype(np.complex128)


def random_field(shape, seed: int) -> np.ndarray:
    """Seeded complex normal field (for parity inputs that are not physical states)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


# --- the five workloads ------------------------------------------------------------------------

def config_1d() -> Tuple[Problem, np.ndarray, int]:
    """d=1, n=1023 on [-20,20], alpha=1.5, rho=2, sech(x)e^{2ix}, dt=0.01, 50 steps, tol 1e-10."""
    p = Problem(d=1, n=(1023,), lo=(-20.0,), hi=(20.0,), alpha=1.5, rho=2.0, dt=0.01, tol=1e-10)
    return p, u0_sech_1d(p, 2.0), 50


def config_2d(alpha: float = 1.5, n: int = 511) -> Tuple[Problem, np.ndarray, int]:
    """d=2, n=511^2 on [-10,10]^2, alpha in {1.2,1.5,1.9}, rho=2, sech(x)sech(y)e^{i(x+y)},
    dt=0.005, 100 steps, tol 1e-10."""
    p = Problem(d=2, n=(n, n), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=alpha, rho=2.0, dt=0.005,
                tol=1e-10)
    return p, u0_sech_product(p, [1.0, 1.0]), 100


CONFIG_2D_ALPHAS = (1.2, 1.5, 1.9)


def config_3d(n: int = 255) -> Tuple[Problem, np.ndarray, int]:
    """d=3, n=255^3 on [-8,8]^3, alpha=1.7, rho=1, exp(-|x|^2/2)e^{ix_1}, dt=0.01, 20 steps,
    tol 1e-8."""
    p = Problem(d=3, n=(n, n, n), lo=(-8.0,) * 3, hi=(8.0,) * 3, alpha=1.7, rho=1.0, dt=0.01, tol=1e-8)
    return p, u0_gaussian(p, 1.0), 20


def config_batched(count: int = 64, seed: int = 2410, sizes=(127, 255, 511)):
    """Independent 2-D instances: n_x, n_y drawn i.i.d. from `sizes`, alpha ~ U[1.1,1.95],
    rho ~ U[0.5,3], u0 = sech(x)sech(y) e^{i(kx x + ky y)} with k ~ U[-3,3]; box [-10,10]^2,
    dt = 0.005, 20 steps each."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny = (int(v) for v in rng.choice(sizes, size=2))
        alpha = float(rng.uniform(1.1, 1.95))
        rho = float(rng.uniform(0.5, 3.0))
        kx, ky = (float(v) for v in rng.uniform(-3.0, 3.0, size=2))
        p = Problem(d=2, n=(nx, ny), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=alpha, rho=rho,
                    dt=0.005, tol=1e-10)
        out.append((p, u0_sech_product(p, [kx, ky])))
    return out, 20


def config_adjoint(n: int = 255):
    """Gradient workload: d=2, n=255^2 on [-10,10]^2, alpha=1.5, rho=2, dt=0.005, 20 steps, FP64,
    u0 = sech(x)sech(y)e^{i(x+y)}.  The target of L = sum |u(T) - u_target|^2 is the run from
    u0 (1 + 0.01 xi) with rho * 1.05, xi complex normal (seed 3643).  Returns
    (problem, u0, nsteps, u0_target, rho_target)."""
    p = Problem(d=2, n=(n, n), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=1.5, rho=2.0, dt=0.005,
                tol=1e-10)
    u0 = u0_sech_product(p, [1.0, 1.0])
    xi = random_field(p.shape, 3643) / math.sqrt(2.0)
    return p, u0, 20, u0 * (1.0 + 0.01 * xi), p.rho * 1.05


def fd_directions(shape, count: int = 8, seed: int = 643):
    """Seeded unit directions for finite-difference checks: `count` complex normal fields of the
    given shape (normalised to unit 2-norm) and `count` scalar directions for rho."""
    rng = np.random.default_rng(seed)
    dirs = []
    for _ in range(count):
        v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        dirs.append((v / np.linalg.norm(v)).astype(np.complex128))
    return dirs, rng.standard_normal(count)
