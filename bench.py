#!/usr/bin/env python3
"""Benchmark: DOF x timesteps / s of the tau-preconditioned GMRES time stepper.

Workload (default): d = 2, n = 511 x 511 on [-10,10]^2, rho = 2, dt = 0.005, u0 = sech(x)sech(y)e^{i(x+y)},
alpha in {1.2, 1.5, 1.9} (three independent instances), tol 1e-10.  One bench step advances all three
instances by one time step (a GMRES solve each, all three through one rfnse_batch_run call) in the mixed
form (FP32 transforms inside FGMRES, FP64 Arnoldi/Givens, the refinement residual accurate to about
1e-14); the plain FP64 form is timed the same way and reported
beside it, with the difference between the two trajectories.  DOF = complex grid unknowns.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 2d|3d|1d|batched|adjoint|comparators|omega] [--instances K]
  python bench.py --alu-probe | --arnoldi-probe

The JSON line's roofline objects are the three largest kernel classes of the step, each timed launch
by launch (CUDA events) in a further serial run with host-driven loops: the cooperative Arnoldi
kernel, the FP32 fused x-pass and the double-float residual x-pass.  --instances K runs K 511^2
instances instead of three (the throughput saturates from about 6 on); --arnoldi-probe times the
Arnoldi kernel alone per column j; --alu-probe measures the FP64 and FP32 FMA rates.

Other workloads: 3d (255^3, mixed), 1d (n = 1023), batched (64 independent 2-D instances with grids
drawn from {127, 255, 511}^2: one step = one graph launch advancing all of them), adjoint (255^2,
20 steps, FP64: one step = a taped forward run plus its reverse pass, dL/du0 and dL/drho),
comparators (255^2: the same run with the sine-transform preconditioner, Strang's circulant and none),
omega (Fig. 1: tau-GMRES iterations versus the TBAN parameter w for five alpha, 1-D n = 2047).

Multi-GPU (torchrun): every rank advances its own copy of the three instances (independent problems,
no collective on the data path; weak scaling); value = all ranks' DOF x steps / max rank time.
--impl reference times the CPU oracle (test infrastructure) on the host cores, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "DOF*timesteps/s"
UNIT = "DOF*timesteps/s"
FP64_ALU_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the FP64 Toeplitz x-pass (ncu)
TRAFFIC_FP64_TOEP_X = {"2d": 10530816 + 0}
FP32_ALU_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9  # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# DRAM read+write per launch of the FP32 fused DST-x + (wI+D) + Toeplitz-x pass (ncu, 2-D 511^2,
# k_line_pass_fixed<float2, float2, double2, float2, 26, 10>)
TRAFFIC_FP32_FUSED_X = {"2d": 5288960 + 0}
# DRAM read+write per launch of the cooperative Arnoldi kernel (ncu, 2-D 511^2: mean of 10 consecutive
# launches, columns j = 1,0,1,2,0,1,0,1,2,0, the mix of the bench's solves; (j + 2) x 4.2 MB each)
TRAFFIC_ARNOLDI = {"2d": 11744538 + 0}
# DRAM read+write per launch of the double-float residual x-pass (ncu, 2-D 511^2, steady launch: the
# launches alternate 6.36 / 10.54 MB, the larger after the first step's extra product)
TRAFFIC_DF_TOEP_X = {"2d": 6360320 + 0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d", choices=["2d", "3d", "1d", "batched", "adjoint", "comparators", "omega"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--serial", action="store_true", help="advance the instances one after another on one stream")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the GMRES loops from the host (no CUDA graphs; same kernels, for kernel profilers)")
    ap.add_argument("--alu-probe", action="store_true",
                    help="only measure the FP64 and FP32 FMA rates of the GPU and print them")
    ap.add_argument("--arnoldi-probe", action="store_true",
                    help="only time the cooperative Arnoldi kernel (MGS + Givens) per column j on the 2-D and "
                         "3-D grid sizes and print the times")
    ap.add_argument("--instances", type=int, default=3,
                    help="2d workload: number of 511^2 instances advanced together (alphas cycle through "
                         "1.2, 1.5, 1.9); the default 3 is the headline configuration")
    return ap.parse_args()


def workload(name, instances=3):
    """[(problem, u0)] and a description."""
    if name == "2d":
        alphas = [W.CONFIG_2D_ALPHAS[i % len(W.CONFIG_2D_ALPHAS)] for i in range(instances)]
        inst = [W.config_2d(a)[:2] for a in alphas]
        tag = "" if instances == 3 else f"_x{instances}"
        desc = {"workload": "2d_n511x511_alpha{1.2,1.5,1.9}_rho2_dt0.005_tol1e-10" + tag, "d": 2, "n": [511, 511],
                "box": [-10, 10], "alphas": alphas, "instances": instances}
    elif name == "3d":
        p, u0, _ = W.config_3d()
        inst = [(p, u0)]
        desc = {"workload": "3d_n255^3_alpha1.7_rho1_dt0.01_tol1e-8", "d": 3, "n": [255, 255, 255],
                "box": [-8, 8], "alphas": [1.7], "instances": 1}
    elif name == "batched":
        inst, _ = W.config_batched()
        desc = {"workload": "batched_64x2d_n{127,255,511}^2_seed2410_dt0.005_tol1e-10", "d": 2,
                "instances": len(inst), "dof_per_step": int(sum(p.size for p, _ in inst)),
                "sampling": "n_x, n_y iid from {127,255,511}; alpha~U[1.1,1.95]; rho~U[0.5,3]; k~U[-3,3]"}
    else:
        p, u0, _ = W.config_1d()
        inst = [(p, u0)]
        desc = {"workload": "1d_n1023_alpha1.5_rho2_dt0.01_tol1e-10", "d": 1, "n": [1023], "box": [-20, 20],
                "alphas": [1.5], "instances": 1}
    return inst, desc


# --- clocks -------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t_on = self.t_off = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_on(self):
        self.t_on = time.time()

    def mark_off(self):
        self.t_off = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l for t, l in self.lines if self.t_on is not None and self.t_on - 0.05 <= t <= self.t_off + 0.05]
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smmax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smmax) if smmax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --- distributed helpers ------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, units_per_rank: float, steps: int, ms_max: float) -> float:
    """Whole-job throughput under weak scaling: every rank processes the same units per step, the job
    takes the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max * 1e-3)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --- the CPU oracle as the baseline / reference arm ---------------------------------------------
def oracle_sample(inst, nsteps: int):
    """Time `nsteps` regular time steps (n >= 1) of the first instance with the CPU oracle.
    Returns (DOF x steps / s, seconds, steps)."""
    from oracle.scheme import SchemeOracle
    p, u0 = inst[0]
    o = SchemeOracle(p)
    u1, _, _ = o.first_step(u0)
    up, uc = u0, u1
    t0 = time.perf_counter()
    for _ in range(nsteps):
        un, _, _ = o.step(up, uc)
        up, uc = uc, un
    dt = time.perf_counter() - t0
    return p.size * nsteps / dt, dt, nsteps


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    inst, desc = workload(args.workload, args.instances)
    from oracle.scheme import SchemeOracle
    # one bench step = one time step of one instance (instances visited in turn), CPU oracle
    states = []
    for p, u0 in inst:
        o = SchemeOracle(p)
        u1, _, _ = o.first_step(u0)
        states.append([o, u0, u1])
    k = 0

    def one():
        nonlocal k
        st = states[k % len(states)]
        o, up, uc = st
        un, _, _ = o.step(up, uc)
        st[1], st[2] = uc, un
        k += 1
        return o.p.size

    for _ in range(args.warmup):
        one()
    dof = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dof += one()
    dt = time.perf_counter() - t0
    value = dof / dt
    cores = host_cores()
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (closed-form initial data of the paper's shape)",
           "config": dict(desc, sample="one time step of one alpha instance per bench step"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} time steps, instances in turn, numpy/BLAS on {cores} host cores"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# --- our CUDA path --------------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    inst, desc = workload(args.workload, args.instances)
    main = torch.cuda.current_stream()
    concurrent = not args.serial and len(inst) > 1
    pool = ThreadPoolExecutor(max_workers=len(inst)) if concurrent else None
    # several instances advance together through the batch API (one graph launch per step for all);
    # host-driven loops (--host-loop, for kernel profilers) keep one host thread per instance
    use_batch = concurrent and not args.host_loop

    def make(precision, device_loop=None, batch=None):
        if device_loop is None:
            device_loop = 0 if args.host_loop else 1
        if use_batch if batch is None else batch:
            b = rfnse.Batch([p for p, _ in inst], precision=precision, stream=main, device_loop=device_loop)
            for i, (p, u0) in enumerate(inst):
                b.set_state(i, torch.from_numpy(u0.ravel().copy()).to(dev))
            torch.cuda.synchronize()
            return b
        solvers = []
        for p, u0 in inst:
            st = torch.cuda.Stream(device=dev) if concurrent else main
            s = rfnse.Solver(p, precision=precision, stream=st, device_loop=device_loop)
            s.set_state(torch.from_numpy(u0.ravel().copy()).to(dev))
            solvers.append(s)
        torch.cuda.synchronize()
        return solvers

    def advance(solvers, start_ev=None, serial=False):
        """One bench step: every instance advances one time step (instances in parallel streams)."""
        if isinstance(solvers, rfnse.Batch):
            return [int(v) for v in solvers.run(1)[0][0]]
        if serial or not concurrent:
            return [int(s.run(1)[0][0]) for s in solvers]
        if start_ev is not None:
            for s in solvers:
                s.stream.wait_event(start_ev)
        its = [int(f.result()[0][0]) for f in [pool.submit(s.run, 1) for s in solvers]]
        for s in solvers:
            ev = torch.cuda.Event()
            ev.record(s.stream)
            main.wait_event(ev)
        return its

    def states_of(group):
        if isinstance(group, rfnse.Batch):
            return [group.get_state(i)[1] for i in range(group.count)]
        return [s.get_state()[1] for s in group]

    def close_all(group):
        if isinstance(group, rfnse.Batch):
            group.close()
        else:
            for s in group:
                s.close()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    dof_per_step = sum(p.size for p, _ in inst)

    def timed(solvers, steps, warmup, profile_kind=0, clocks=None, serial=False):
        for _ in range(warmup):
            advance(solvers, serial=serial)
        torch.cuda.synchronize()
        if profile_kind:
            for s in solvers:
                s.profile(profile_kind)
        launches0 = rfnse.launch_count()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        iters = []
        barrier(world)
        torch.cuda.synchronize()
        if clocks:
            clocks.mark_on()
        wall0 = time.perf_counter()
        for k in range(steps):
            flush.fill_(float(k))                       # evict L2 between timed steps
            evs[k][0].record(main)
            iters += advance(solvers, evs[k][0], serial=serial)
            evs[k][1].record(main)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if clocks:
            clocks.mark_off()
        barrier(world)
        launches = rfnse.launch_count() - launches0
        ms = sum(a.elapsed_time(b) for a, b in evs)
        prof = None
        if profile_kind:
            tot = [0, 0.0, 0.0, 0.0]
            for s in solvers:
                n, pms, fl, by = s.profile_read()
                tot[0] += n; tot[1] += pms; tot[2] += fl; tot[3] += by
                s.profile(0)
            prof = tot
        return ms, wall, launches, iters, prof

    # headline: mixed form
    mixed = make(1)
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    # the residual's Toeplitz pass along x (double-float FFTs in the mixed form on these grids); for 1-D
    # the preconditioner and the product share one FP32 pass
    dom_kind = (rfnse.K_DF | rfnse.K_TOEP_X) if args.workload != "1d" else \
        (rfnse.K_FP32 | rfnse.K_DST | rfnse.K_LAM | rfnse.K_DSCALE | rfnse.K_TOEP_X)
    ms, wall, launches, iters_m, _ = timed(mixed, args.steps, args.warmup, clocks=clocks)
    clk = clocks.stop() if clocks else None
    mixed_states = states_of(mixed)   # after warmup + steps, for the FP64 comparison
    # the dominant kernel class, timed launch by launch in a further serial run of the same steps
    # (in the concurrent region the instances' kernels share the SMs, which stretches each launch)
    # (host-driven solvers: CUDA events cannot be recorded around single kernels inside a running graph;
    # the kernels are the same as in the device loop)
    nprof = max(1, min(args.steps, 20))
    prof_solvers = make(1, device_loop=0, batch=False)
    ms_r, _, _, _, prof = timed(prof_solvers, nprof, args.warmup, profile_kind=dom_kind, serial=True)
    for s in prof_solvers:
        s.close()
    # the other large class: the FP32 pass that ends the preconditioner and starts the product along x
    prof32 = None
    if args.workload in ("2d", "3d"):
        k32 = rfnse.K_FP32 | rfnse.K_DST | rfnse.K_DSCALE | rfnse.K_TOEP_X
        prof_solvers = make(1, device_loop=0, batch=False)
        ms_r32, _, _, _, prof32 = timed(prof_solvers, nprof, args.warmup, profile_kind=k32, serial=True)
        for s in prof_solvers:
            s.close()
    # the cooperative Arnoldi kernel (MGS, Givens, test), launched on its own by the host-driven loops
    prof_arn = None
    if args.workload in ("2d", "3d"):
        prof_solvers = make(1, device_loop=0, batch=False)
        ms_ra, _, _, _, prof_arn = timed(prof_solvers, nprof, args.warmup, profile_kind=rfnse.K_ARNOLDI, serial=True)
        for s in prof_solvers:
            s.close()
    ms_max = reduce_max(ms, world, dev)
    value = weak_value(world, dof_per_step, args.steps, ms_max)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
           "data": "synthetic (closed-form initial data of the paper's shape)",
           "config": dict(desc, precision="mixed: FP32 transforms in FGMRES, FP64 Arnoldi/Givens/residual",
                          l2="256 MiB buffer written between timed steps",
                          parallelism=(f"{world} GPU(s), instances replicated per GPU; "
                                       + ("all instances advanced by one batch call per step "
                                          "(rfnse_batch_run: one CUDA graph launch)" if use_batch else
                                          "one CUDA stream and host thread per instance" if concurrent
                                          else "instances in turn on one stream")),
                          control=("host-driven GMRES loops" if args.host_loop
                                   else "device-decided GMRES loops, one CUDA graph per solve")),
           "gpu_launches": launches,
           "iters_per_solve_mean": float(np.mean(iters_m)) if iters_m else None}

    # roofline of the two largest kernel classes, each timed launch by launch; the larger is `roofline`
    measured = ("CUDA events around every launch of the class (on its stream), serial run of "
                f"{nprof} further bench steps")
    entries = []
    if prof and prof[0] > 0 and args.workload != "1d":
        n, pms, fl, by = prof
        hbm, how = measured_hbm_gbs()
        achieved = by / (pms * 1e-3) / 1e9
        fp64eq = fl / (pms * 1e-3) / 1e12
        entries.append({"bound": "hbm", "kernel": "k_toeplitz_df<F_TOEP_X> (residual Toeplitz x-pass, "
                                                  "double-float FFTs)",
                        "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        # profiles/k_toeplitz_df_x_2d511.md
                        "traffic": TRAFFIC_DF_TOEP_X.get(args.workload), "launches": n,
                        "avg_launch_us": 1e3 * pms / n, "total_ms": pms,
                        "share_of_step_time": pms / ms_r if ms_r > 0 else None, "measured": measured,
                        "algorithmic_flops_per_launch": fl / n, "algorithmic_bytes_per_launch": by / n,
                        "fp64_equivalent_TFLOPs": fp64eq,
                        "frac_of_fp64_alu_peak": fp64eq * 1e12 / FP64_ALU_PEAK_FLOPS,
                        "peak_note": f"copy bandwidth, {how} (MEASURED_PEAKS.json).  The FFTs run in "
                                     "double-float on the FP32 pipes, so their FP64-accurate flop rate may "
                                     "exceed the native FP64 peak (152 SM x 2 FMA/clk x 2 x 2.07 GHz)"})
    if prof and prof[0] > 0 and args.workload == "1d":
        n, pms, fl, by = prof
        hbm, how = measured_hbm_gbs()
        achieved = by / (pms * 1e-3) / 1e9
        entries.append({"bound": "hbm", "kernel": "k_line_pass<float,all flags> (1-D FP32 preconditioner + "
                                                  "product)", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": None, "launches": n, "avg_launch_us": 1e3 * pms / n,
                        "total_ms": pms, "share_of_step_time": pms / ms_r if ms_r > 0 else None,
                        "measured": measured, "peak_note": f"copy bandwidth, {how}"})
    if prof32 and prof32[0] > 0:
        n, pms, fl, by = prof32
        hbm, how = measured_hbm_gbs()
        achieved = by / (pms * 1e-3) / 1e9
        entries.append({"bound": "hbm", "kernel": ("k_line_pass_fixed" if args.workload == "2d" else "k_line_pass")
                                                  + "<float,F_DST|F_DSCALE|F_TOEP_X> "
                                                  "(FP32 inverse DST x + (wI+D) + Toeplitz x)",
                        "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        # profiles/k_line_pass_fp32_fused_x_2d511.md
                        "traffic": TRAFFIC_FP32_FUSED_X.get(args.workload), "launches": n,
                        "avg_launch_us": 1e3 * pms / n, "total_ms": pms,
                        "share_of_step_time": pms / ms_r32 if ms_r32 > 0 else None, "measured": measured,
                        "algorithmic_flops_per_launch": fl / n, "algorithmic_bytes_per_launch": by / n,
                        "achieved_TFLOPs": fl / (pms * 1e-3) / 1e12,
                        "frac_of_fp32_alu_peak": fl / (pms * 1e-3) / FP32_ALU_PEAK_FLOPS,
                        "peak_note": f"copy bandwidth, {how} (MEASURED_PEAKS.json); arithmetic intensity "
                                     f"{fl / by:.1f} flop/B is below the FP32 balance point"})
    if prof_arn and prof_arn[0] > 0:
        n, pms, fl, by = prof_arn
        hbm, how = measured_hbm_gbs()
        achieved = fl / (pms * 1e-3) / 1e12
        entries.append({"bound": "alu", "kernel": "k_mgs_step (cooperative MGS + Givens + convergence test, "
                                                  "one launch per Arnoldi step)",
                        "achieved": achieved, "peak": FP64_ALU_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                        "frac": achieved * 1e12 / FP64_ALU_PEAK_FLOPS,
                        # profiles/k_mgs_step_2d511.md
                        "traffic": TRAFFIC_ARNOLDI.get(args.workload), "launches": n,
                        "avg_launch_us": 1e3 * pms / n, "total_ms": pms,
                        "share_of_step_time": pms / ms_ra if ms_ra > 0 else None, "measured": measured,
                        "algorithmic_flops_per_launch": fl / n, "algorithmic_bytes_per_launch": by / n,
                        "achieved_GBs": by / (pms * 1e-3) / 1e9, "frac_of_hbm": by / (pms * 1e-3) / 1e9 / hbm,
                        "peak_note": "FP64 FMA issue rate, 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz (1.26 TFLOP/s "
                                     "measured by --alu-probe); the kernel performs j + 2 sweeps with a grid-wide "
                                     "reduction after each, and the synchronisation between sweeps, not the FP64 "
                                     f"pipe or memory, sets its time ({how} copy bandwidth beside it)"})
    if entries:
        entries.sort(key=lambda e: -e["total_ms"])
        out["roofline"] = entries[0]
        if len(entries) > 1:
            out["roofline_second"] = entries[1]
        if len(entries) > 2:
            out["roofline_third"] = entries[2]
    if clk:
        out["clocks"] = clk

    # plain FP64 form, same protocol, and the distance between the two trajectories
    if not args.no_fp64:
        fp64 = make(0)
        ms64, _, _, iters64, _ = timed(fp64, args.steps, args.warmup)
        ms64 = reduce_max(ms64, world, dev)
        errs = []
        for ua, ub in zip(mixed_states, states_of(fp64)):
            errs.append(float(torch.linalg.vector_norm(ua - ub) / torch.linalg.vector_norm(ub)))
        out["fp64"] = {"value": world * dof_per_step * args.steps / (ms64 * 1e-3), "ms_per_step": ms64 / args.steps,
                       "iters_per_solve_mean": float(np.mean(iters64)) if iters64 else None}
        out["mixed_vs_fp64_rel_l2_after_run"] = max(errs)
        out["mixed_speedup_vs_fp64"] = ms64 / ms_max
        close_all(fp64)

    # end to end through the C ABI with host buffers: H2D of the step's inputs, D2H of its result
    if not args.no_e2e:
        e2e_solvers = make(1, batch=False)
        for s in e2e_solvers:
            s.run(2)  # reach a regular step
        hosts = []
        for s in e2e_solvers:
            up, uc, step = s.get_state()
            pin_up = torch.empty(s.N, dtype=torch.complex128, pin_memory=True)
            pin_uc = torch.empty(s.N, dtype=torch.complex128, pin_memory=True)
            pin_out = torch.empty(s.N, dtype=torch.complex128, pin_memory=True)
            pin_up.copy_(up.cpu())
            pin_uc.copy_(uc.cpu())
            hosts.append([pin_up, pin_uc, pin_out, step])
        steps_e2e = max(1, min(args.steps, 30))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        def e2e_one(s, h):
            s.set_state_host(h[1].numpy(), h[0].numpy(), h[3])     # H2D of u^{n-1}, u^n
            s.run_host(1, h[2].numpy())                            # step + D2H of u^{n+1}
            h[0], h[1], h[2] = h[1], h[2], h[0]
            h[3] += 1

        for _ in range(steps_e2e):
            if concurrent:
                for f in [pool.submit(e2e_one, s, h) for s, h in zip(e2e_solvers, hosts)]:
                    f.result()
            else:
                for s, h in zip(e2e_solvers, hosts):
                    e2e_one(s, h)
        torch.cuda.synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
        nb = sum(s.N for s in e2e_solvers) * 16
        out["e2e"] = {"value": world * dof_per_step * steps_e2e / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": 2 * nb, "d2h_bytes_per_step": nb, "steps": steps_e2e}
        for s in e2e_solvers:
            s.close()

    # the CPU oracle on the host cores (bounded sample), rank 0 at N = 1 only
    if not args.no_cpu and rank == 0 and world == 1:
        n_cpu = 30 if args.workload != "3d" else 1
        v, secs, n = oracle_sample(inst, n_cpu)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                               "sample": f"{n} time steps of the alpha={inst[0][0].alpha} instance "
                                         f"({secs:.1f} s), numpy/BLAS dense-transform oracle"}
    close_all(mixed)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batched(args):
    """The 64-instance batch: one bench step = one time step of every instance (one graph launch)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    inst, desc = workload("batched")
    main = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    dof = sum(p.size for p, _ in inst)

    def timed(precision, clocks=None):
        b = rfnse.Batch([p for p, _ in inst], precision=precision, stream=main)
        for i, (p, u0) in enumerate(inst):
            b.set_state(i, torch.from_numpy(u0.ravel().copy()).to(dev))
        b.run(max(args.warmup, 3))                  # the first steps run instance by instance
        torch.cuda.synchronize()
        l0 = rfnse.launch_count()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        its = []
        barrier(world)
        if clocks:
            clocks.mark_on()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(main)
            it, _ = b.run(1)
            evs[k][1].record(main)
            its.append(it)
        torch.cuda.synchronize()
        if clocks:
            clocks.mark_off()
        ms = sum(a.elapsed_time(e) for a, e in evs)
        launches = rfnse.launch_count() - l0
        states = [b.get_state(i)[1] for i in range(b.count)]
        b.close()
        return ms, launches, np.array(its), states

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    ms, launches, its, st_mixed = timed(1, clocks)
    clk = clocks.stop() if clocks else None
    ms = reduce_max(ms, world, dev)
    out = {"metric": METRIC, "value": weak_value(world, dof, args.steps, ms), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
           "data": "synthetic (closed-form initial data of the paper's shape, seeded parameters)",
           "config": dict(desc, precision="mixed", l2="256 MiB buffer written between timed steps",
                          parallelism=f"{world} GPU(s); one CUDA graph launch per batch step"),
           "gpu_launches": launches, "iters_per_solve_mean": float(its.mean())}
    if clk:
        out["clocks"] = clk
    if not args.no_fp64:
        ms64, _, its64, st64 = timed(0)
        ms64 = reduce_max(ms64, world, dev)
        errs = [float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(st_mixed, st64)]
        out["fp64"] = {"value": world * dof * args.steps / (ms64 * 1e-3), "ms_per_step": ms64 / args.steps,
                       "iters_per_solve_mean": float(its64.mean())}
        out["mixed_vs_fp64_rel_l2_after_run"] = max(errs)
        out["mixed_speedup_vs_fp64"] = ms64 / ms
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_adjoint(args):
    """The gradient workload (255^2, 20 steps, FP64): one bench step = a taped forward run plus its
    reverse pass (dL/du0 and dL/drho of L = sum |u^N - u_target|^2), checkpoints every 5 steps."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    p, u0, nsteps, u0t, rho_t = W.config_adjoint()
    main = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = rfnse.Solver(p.replace(rho=rho_t), precision=0, stream=main)
    target, _ = st.tape_forward(torch.from_numpy(u0t.ravel().copy()).to(dev), nsteps, 5)
    st.close()
    s = rfnse.Solver(p, precision=0, stream=main)
    x0 = torch.from_numpy(u0.ravel().copy()).to(dev)

    def one():
        uN, _ = s.tape_forward(x0, nsteps, 5)
        return s.tape_backward(2.0 * (uN - target))

    for _ in range(max(args.warmup, 3)):
        one()
    torch.cuda.synchronize()
    l0 = rfnse.launch_count()
    fw, bw = [], []
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
        clocks.mark_on()
    barrier(world)
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(main)
        uN, _ = s.tape_forward(x0, nsteps, 5)
        e1.record(main)
        g0, grho, its = s.tape_backward(2.0 * (uN - target))
        e2.record(main)
        torch.cuda.synchronize()
        fw.append(e0.elapsed_time(e1))
        bw.append(e1.elapsed_time(e2))
    if clocks:
        clocks.mark_off()
    clk = clocks.stop() if clocks else None
    launches = rfnse.launch_count() - l0
    ms = reduce_max(sum(fw) + sum(bw), world, dev)
    out = {"metric": METRIC, "value": weak_value(world, p.size * nsteps, args.steps, ms), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (closed-form initial data; target from a seeded perturbation of u0 and rho)",
           "config": {"workload": "adjoint_2d_n255_alpha1.5_rho2_dt0.005_20steps_fp64", "d": 2, "n": [255, 255],
                      "what": "one step = taped forward run + reverse pass (dL/du0, dL/drho), checkpoint every 5",
                      "l2": "256 MiB buffer written between timed steps", "parallelism": f"{world} GPU(s)"},
           "gpu_launches": launches, "forward_ms": sum(fw) / args.steps, "backward_ms": sum(bw) / args.steps,
           "backward_over_forward": sum(bw) / max(sum(fw), 1e-9), "adjoint_arnoldi_steps": its,
           "grad_rho": grho}
    if clk:
        out["clocks"] = clk
    if rank == 0:
        print(json.dumps(out), flush=True)
    s.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_comparators(args):
    """tau-GMRES against the comparators of Sec. 5 (C-GMRES with Strang's circulant, plain GMRES) on
    the same time-stepping run: 2-D 255^2, alpha = 1.5, rho = 2, dt = 0.005, tol 1e-10, mixed form."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    p, u0, _ = W.config_2d(1.5, n=255)
    main = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for pc, name in ((0, "tau-GMRES"), (1, "C-GMRES"), (2, "GMRES")):
        q = p.replace(precond=pc, restart=256 if pc == 2 else p.restart)
        s = rfnse.Solver(q, precision=1, stream=main)
        s.set_state(torch.from_numpy(u0.ravel().copy()).to(dev))
        s.run(max(args.warmup, 3))
        steps = args.steps if pc != 2 else max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        ms, its = 0.0, []
        for k in range(steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            it, _ = s.run(1)
            b.record(main)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            its.append(int(it[0]))
        res[name] = {"value": q.size * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "iters_per_solve_mean": float(np.mean(its)), "steps": steps}
        s.close()
    out = {"metric": METRIC, "value": res["tau-GMRES"]["value"], "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": res["tau-GMRES"]["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
           "data": "synthetic (closed-form initial data of the paper's shape)",
           "config": {"workload": "comparators_2d_n255_alpha1.5_rho2_dt0.005_tol1e-10", "d": 2, "n": [255, 255],
                      "what": "the same run with the sine-transform preconditioner, Strang's circulant "
                              "(Bluestein DFTs) and none (restart 256)",
                      "l2": "256 MiB buffer written between timed steps"},
           "comparators": res}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_omega(args):
    """Fig. 1: tau-GMRES iterations at the 2nd time level versus the TBAN parameter w in (0, 4] for
    alpha = 1.1:0.2:1.9 (1-D, [-20,20], rho = 2, sech(x)e^{2ix}, n = 2047, dt = 0.05, tol 1e-8, no
    restart); the line's value is the solve throughput over the whole sweep."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    main = torch.cuda.current_stream()
    omegas = [round(0.1 * k, 1) for k in range(1, 41)]
    curves, best, total_ms, nsolve = {}, {}, 0.0, 0
    n = 2047
    for alpha in (1.1, 1.3, 1.5, 1.7, 1.9):
        its = []
        for w in omegas:
            p = W.Problem(d=1, n=(n,), lo=(-20.0,), hi=(20.0,), alpha=alpha, rho=2.0, dt=0.05, tol=1e-8, omega=w,
                          restart=256)
            s = rfnse.Solver(p, precision=0, stream=main)
            u0 = torch.from_numpy(W.u0_sech_1d(p, 2.0)).to(dev)
            s.set_state(u0)
            s.run(1)
            _, u1, _ = s.get_state()
            D = (p.rho * p.dt) * torch.abs(u1) ** 2
            b = -s.apply_A(u0, D) + 2j * u0
            s.solve(D, b)                                    # warm: graph capture
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            _, it, _ = s.solve(D, b)
            e1.record(main)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            nsolve += 1
            its.append(it)
            s.close()
        curves[str(alpha)] = its
        best[str(alpha)] = omegas[int(np.argmin(its))]
    out = {"metric": METRIC, "value": n * nsolve / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": nsolve,
           "warmup": 1, "ms_per_step": total_ms / nsolve, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (the 1-D test of Sec. 5.1)",
           "config": {"workload": "omega_sweep_1d_n2047_rho2_dt0.05_tol1e-8", "what": "one step = one solve at "
                      "the 2nd time level; w = 0.1:0.1:4.0 for each alpha"},
           "omega": omegas, "iterations": curves, "best_omega": best}
    print(json.dumps(out), flush=True)


def arnoldi_probe():
    """Duration of the cooperative Arnoldi kernel per column j (CUDA events, 20 launches each)."""
    import torch
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    props = torch.cuda.get_device_properties(0)
    out = {"device": props.name, "what": "k_mgs_step: MGS against j+1 basis vectors, Givens, test"}
    for name, n in (("2d_511^2", 511 * 511), ("3d_255^3", 255 ** 3)):
        rows = {}
        for j in (0, 1, 2, 3, 4, 7):
            us, blocks = rfnse.probe_arnoldi(n, j)
            rows[str(j)] = round(us, 2)
        out[name] = {"n": n, "blocks": blocks, "us_per_step_by_j": rows}
    print(json.dumps(out), flush=True)


def alu_probe():
    import torch
    from paper_2410_03643_gb300 import build, rfnse
    build.build_library()
    props = torch.cuda.get_device_properties(0)
    out = {"device": props.name, "sms": props.multi_processor_count,
           "fp64_tflops": rfnse.probe_fma(True) / 1e12, "fp32_tflops": rfnse.probe_fma(False) / 1e12}
    out["fp32_over_fp64"] = out["fp32_tflops"] / out["fp64_tflops"]
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.alu_probe:
        alu_probe()
        return
    if args.arnoldi_probe:
        arnoldi_probe()
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "comparators":
        run_comparators(args)
    elif args.workload == "omega":
        run_omega(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
