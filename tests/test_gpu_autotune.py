"""The autotuner of the line passes (rfnse_autotune): it tunes every pass configuration a solve
launches, the solves then launch those configurations with the chosen geometry, and the results are
those of an untuned context (the arithmetic of a line does not depend on the tile) and of the oracle."""
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


CASES = [
    # (problem, precision, configurations tuned: the line passes one context's solves launch, plus the
    # Arnoldi kernel's grid when N > 4096)
    (W.Problem(d=2, n=(255, 127), lo=(-8.0, -6.0), hi=(8.0, 6.0), alpha=1.4, rho=2.0, dt=0.005), 1, 5),
    (W.Problem(d=2, n=(127, 255), lo=(-6.0, -8.0), hi=(6.0, 8.0), alpha=1.8, rho=1.0, dt=0.005), 0, 9),
    (W.Problem(d=3, n=(31, 15, 63), lo=(-4.0, -3.0, -5.0), hi=(4.0, 3.0, 5.0), alpha=1.3, rho=1.0, dt=0.01), 1, 10),
    (W.Problem(d=1, n=(2047,), lo=(-20.0,), hi=(20.0,), alpha=1.6, rho=2.0, dt=0.01), 1, 2),
]


@pytest.mark.parametrize("device_loop", (0, 1))
@pytest.mark.parametrize("case", range(len(CASES)))
def test_autotuned_solver_matches_untuned_and_oracle(case, device_loop):
    from paper_2410_03643_gb300 import Solver
    p, precision, nconf = CASES[case]
    u0 = W.u0_sech_product(p, [1.0] * p.d)
    nsteps = 4

    def run(tune):
        s = Solver(p, precision=precision, device_loop=device_loop)
        info = s.autotune(reps=3, force=True) if tune else None
        s.set_state(dev(u0))
        traj = torch.empty(nsteps * p.size, dtype=torch.complex128, device="cuda")
        its, _ = s.run(nsteps, traj)
        used = s.tuned_launches()
        s.close()
        return traj.cpu().numpy().reshape((nsteps,) + p.shape), its, info, used

    a, its_a, _, used_a = run(False)
    b, its_b, info, used_b = run(True)
    n_configs, n_changed, speedup = info
    assert n_configs == nconf
    assert 0 <= n_changed <= n_configs and speedup >= 1.0
    assert used_a == 0 and used_b > 0            # the tuned geometries are the ones launched
    ref, _, _ = SchemeOracle(p).run(u0, nsteps)
    for k in range(nsteps):
        assert rel(b[k], a[k]) < 1e-12, k
        assert rel(b[k], ref[k]) < (1e-10 if precision == 0 else 1e-8), k
    assert all(abs(int(x) - int(y)) <= 1 for x, y in zip(its_a, its_b))


def test_batch_autotune_tunes_each_grid_once_and_keeps_results():
    from paper_2410_03643_gb300 import Batch
    probs = [W.Problem(d=2, n=(nx, ny), lo=(-10.0, -10.0), hi=(10.0, 10.0), alpha=a, rho=r, dt=0.005)
             for nx, ny, a, r in ((127, 255, 1.3, 1.0), (255, 127, 1.7, 2.0), (127, 255, 1.9, 0.5))]
    u0s = [W.u0_sech_product(p, [1.0, -1.0]) for p in probs]
    nsteps = 4
    out = []
    for tune in (False, True):
        b = Batch(probs, precision=1)
        if tune:
            n_configs, n_changed = b.autotune(reps=3)
            assert n_configs == 5 * len(probs)
        for i, u0 in enumerate(u0s):
            b.set_state(i, dev(u0))
        b.run(nsteps)
        out.append([b.get_state(i)[1].cpu().numpy() for i in range(len(probs))])
        if tune:
            assert b.tuned_launches() > 0
        b.close()
    for i, p in enumerate(probs):
        assert rel(out[1][i], out[0][i]) < 1e-12
        ref, _, _ = SchemeOracle(p).run(u0s[i], nsteps)
        assert rel(out[1][i].reshape(p.shape), ref[-1]) < 1e-8


@pytest.mark.parametrize("precision", (0, 1))
def test_arnoldi_kernel_launches_agree(precision):
    """The Arnoldi kernel on the grid-wide cooperative launch (1 and 2 blocks per SM) and on one
    thread-block cluster (8 and 16 CTAs, where they fit): the same solve to rounding and the oracle's."""
    from paper_2410_03643_gb300 import Solver, rfnse
    p = W.Problem(d=2, n=(511, 255), lo=(-10.0, -8.0), hi=(10.0, 8.0), alpha=1.5, rho=2.0, dt=0.005)
    u0 = W.u0_sech_product(p, [1.0, 1.0])
    nsteps = 3
    ref, its_ref, _ = SchemeOracle(p).run(u0, nsteps)
    got = {}
    for grid in (152, 304, -8, -16):
        for device_loop in (0, 1):
            s = Solver(p, precision=precision, device_loop=device_loop)
            st = s.lib.rfnse_set_arnoldi_grid(s.h, grid)
            if st != rfnse.RFNSE_OK:            # a cluster that does not fit this device
                s.close()
                assert grid < 0
                continue
            assert s.lib.rfnse_arnoldi_grid(s.h) == grid
            s.set_state(dev(u0))
            traj = torch.empty(nsteps * p.size, dtype=torch.complex128, device="cuda")
            its, _ = s.run(nsteps, traj)
            s.close()
            got[(grid, device_loop)] = traj.cpu().numpy().reshape((nsteps,) + p.shape)
            for k in range(nsteps):
                assert rel(got[(grid, device_loop)][k], ref[k]) < (1e-10 if precision == 0 else 1e-8), (grid, k)
            if precision == 0:
                assert all(abs(int(a) - int(b)) <= 1 for a, b in zip(its, its_ref))
    assert (-8, 0) in got  # an 8-CTA cluster fits every GB300
    base = got[(152, 1)]
    for key, val in got.items():
        assert rel(val[-1], base[-1]) < 1e-12, key
