#!/usr/bin/env python3
"""Benchmark: time to 1e-8 relative residual per backward-Euler step at 8.4M DOF.

Workload (synthetic, seeded): 1024 x 1024 cells x 8 layers (8,388,608 unknowns),
two stacked Si dies (100um Si + 10um bond each), TIM 25um and a 1mm Cu spreader in
three sublayers; 50um cells; h = 1e4 W/m^2K to 45 C; dt = 1e-4 s; 100 steps from
45 C; four random block floorplans (64 rectangles + 16 Gaussian hotspots on each Si
layer, seeds 30-33) switched every 25 steps.  Every step is solved to
||b - A theta|| <= 1e-8 ||b|| (FP64) with FP32 Chebyshev-preconditioned PCG inside
FP64 iterative refinement, the whole 100-step loop replayed as one CUDA graph with
device-side loop control.  The plain FP64 GPU path (FP64 PCG, same preconditioner)
is timed on the same trajectory.

One bench step = one full 100-step trajectory.  `value` = ms per time step.
Inputs (about 1 GB of FP32/FP64 arrays) exceed the 129 MB L2, so no L2 flush is
needed between steps.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 rel. residual (8.4M DOF) & stencil HBM GB/s, mixed vs FP64 GPU"
UNIT = "ms per backward-Euler step (8.4M DOF, rel. residual 1e-8)"
NX = NY = 1024
DT = 1e-4
N_STEPS = 100
STEPS_PER_MAP = 25
SEEDS = (30, 31, 32, 33)

# algorithmic bytes per cell of each timed kernel (reads + writes it must make)
KERNEL_BYTES = {
    # the workload's grid has one conductivity per layer: the solver's FP32 and
    # double-float kernels take the face conductances from a per-layer table
    "cheb_f32": 16,      # z_m, z_{m-1}, r (12) + z_{m+1} (4)
    "cheb_tb4": 20,      # four fused steps: z_m, z_{m-1}, r read once (12) + z_{m+4}, z_{m+3} (8)
    "cheb_tb3": 20,      # three fused steps, same traffic per launch
    "cheb_tb2": 20,      # two fused steps, same traffic per launch
    "spmv_dot_f32": 16,  # z, p_old (8) + p_new, mu (8)
    "update_f32": 28,    # x, r (read+write 16) + p, mu (8) + z (4); 1/diag from the per-layer table
    "stencil_f32": 8,    # x (4) + y (4)
    "residual_df": 24,   # theta, theta_n as hi+lo (16) + P f32 (4) + r f32 (4)
    # the same kernels reading per-face arrays (grids with a per-cell conductivity map)
    "cheb_f32_faces": 28,      # + gx gy gz (12)
    "spmv_dot_f32_faces": 28,  # + gx gy gz (12)
    "stencil_f32_faces": 20,   # + gx gy gz (12)
    "residual_df_faces": 48,   # + gx gy gz hi+lo (24)
    "cheb_bf16": 22,     # gx gy gz bf16 (6) + 16
    # plain FP64 path
    "residual_f64": 48,  # gx gy gz (24) + theta, theta_n (16) + P f32 (4) + r f32 (4)
    "stencil_f64": 48,   # gx gy gz, diagonal (32) + x (8) + y (8)
    "cheb_f64": 72,      # gx gy gz, diagonal (32) + z_m, z_{m-1}, r, 1/diag (32) + z_{m+1} (8)
    # the paper's adaptive mixed precision (Sec. 4.4)
    "ad_cheb_a3": 28,    # A3 in FP16 (8) + z_m, z_{m-1}, r, 1/diag (16) + z_{m+1} (4)
    "ad_spmv_early": 32, # D4, gx gy gz FP32 (16) + p (8) + mu (8)
    "ad_spmv_late": 48,  # D4, gx gy gz FP64 (32) + p (8) + mu (8)
    # one multigrid V-cycle on the layer table; finest level: pre-smoothing from zero
    # (b in, x out: 8), restriction (x, b in, 1/4 of a coarse b out: 9), post-smoothing
    # (b, x, 1/4 of the coarse correction in, z out: 13); every coarser level a quarter
    # of the one above: 30 x 4/3
    "mg_vcycle": 40,
    # fused Chebyshev steps on per-face arrays: z_m, z_{m-1}, r, gx, gy, gz read once (24)
    # + z_{m+S}, z_{m+S-1} written (8)
    "cheb_tbf4": 32,
    "cheb_tbf3": 32,
    "cheb_tbf2": 32,
}
DOMINANT = "cheb_tb4"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--degree", type=int, default=29, help="Chebyshev degree k (SpMVs per application)")
    ap.add_argument("--fp64-degree", type=int, default=10,
                    help="Chebyshev degree of the plain FP64 comparison arm (its own best, measured)")
    ap.add_argument("--faces-degree", type=int, default=0,
                    help="Chebyshev degree of the per-face trajectory (0: the headline's)")
    ap.add_argument("--adaptive-degree", type=int, default=6,
                    help="Chebyshev degree of the paper's adaptive scheme (its own best, measured)")
    ap.add_argument("--guess", type=int, default=3,
                    help="transient initial guess: 0 previous step (the paper's warm start), "
                         "1 linear extrapolation from the two previous steps, 2 quadratic from three, "
                         "3 cubic from four (orders capped by the steps since the last power-map switch)")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="smallest residual reduction an FP32 inner solve is asked for")
    ap.add_argument("--fuse", type=int, default=0,
                    help="Chebyshev steps per launch (0 auto = 4, 1 one step per launch, 2..4)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-stack batched section")
    ap.add_argument("--no-faces", action="store_true",
                    help="skip the trajectory on per-face arrays (conductivity map holding the layer values)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 2048x2048x10 adjoint section")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the trajectory with the paper's adaptive mixed-precision PCG")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernels", action="store_true")
    ap.add_argument("--no-ablation", action="store_true", help="skip the stencil-vs-CSR SpMV comparison")
    ap.add_argument("--no-precond", action="store_true",
                    help="skip the preconditioner comparison (Chebyshev vs multigrid, steady 512^2x8 and the "
                         "transient trajectory)")
    ap.add_argument("--polled", action="store_true",
                    help="host-polled loop instead of the CUDA graph (same kernels; for per-kernel profiling)")
    ap.add_argument("--time-steps", type=int, default=N_STEPS,
                    help="backward-Euler steps per trajectory (100 for the measured workload; "
                         "fewer only for short profiling captures)")
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not sample nvidia-smi (profiling runs under ncu)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only time each hot kernel on the full-size grid (short ncu target)")
    ap.add_argument("--reps", type=int, default=40, help="launches per kernel timing")
    ap.add_argument("--cpu-child", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks

class NoClocks:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def summary(self):
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (profiling run)"]}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if len(r) > 5 + j and r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------- workload

def workload_arrays():
    import numpy as np
    import thermal_inputs as ti
    inst = ti.c3(NX, NY, SEEDS, dtype=np.float32)
    maps = [inst.power] + list(inst.extra_power)
    return inst, maps


def config_dict(degree, polled=False, guess=2, fuse=0):
    return {"workload": "transient backward Euler, 1024x1024x8 layers (8,388,608 DOF), 2 Si dies + TIM + Cu, "
                        "dt=1e-4 s, 100 steps from 45 C, 4 floorplans switched every 25 steps",
            "nx": NX, "ny": NY, "layers": 8, "dof": NX * NY * 8, "time_steps_per_bench_step": N_STEPS,
            "tol_rel": 1e-8, "precision": "FP32 PCG + FP64 iterative refinement",
            "preconditioner": f"Chebyshev degree {degree} on the Jacobi-scaled operator (Lanczos bounds), "
                              f"up to {fuse or 4} steps per launch (temporal blocking)",
            "initial_guess": {0: "previous step T_n", 1: "linear extrapolation 2 T_n - T_(n-1)",
                              2: "quadratic extrapolation 3 T_n - 3 T_(n-1) + T_(n-2)",
                              3: "cubic extrapolation 4 T_n - 6 T_(n-1) + 4 T_(n-2) - T_(n-3)"}[guess]
                             + (", order capped by the steps since the last power-map switch" if guess >= 2 else ""),
            "loop": ("host-polled launch chunks (profiling mode)" if polled else
                     "CUDA graph, conditional WHILE nodes (no host sync inside the 100 steps)"),
            "l2": "inputs larger than L2 (about 1 GB resident vs 129 MB L2); no flush"}


# ----------------------------------------------------------------- oracle timing (CPU)

def cpu_oracle_step_ms(n_samples=1):
    """The FP64 CPU oracle as it stands: Algorithm 1 with Jacobi on the assembled CSR
    matrix of one backward-Euler step, to the same 1e-8 relative residual, single thread."""
    import numpy as np
    from oracle import discretisation as disc, krylov
    inst, maps = workload_arrays()
    st = inst.stack
    A = disc.assemble(NX, NY, st, dt=DT)
    T = np.full(inst.n, st.t_amb)
    times = []
    for s in range(n_samples):
        p = maps[(s // STEPS_PER_MAP) % len(maps)].astype(np.float64)
        b = disc.rhs_transient(NX, NY, st, p, T, DT)
        t0 = time.perf_counter()
        op = krylov.CountingOp(A)
        T, it, _, _ = krylov.pcg(op, b, krylov.jacobi(A), x0=T, tol_rel=1e-8)
        times.append((time.perf_counter() - t0) * 1e3)
    return times


def run_cpu_child():
    times = cpu_oracle_step_ms(1)
    print(json.dumps({"ms": times}))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _thread_env(n):
    return {v: str(n) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}


def cpu_baseline():
    """The oracle's step timed twice in child processes: with NumPy/SciPy allowed every
    host core, and with one thread.  SciPy's sparse product is single-threaded; the
    vector reductions go through the BLAS, which takes the threads."""
    sample = ("first backward-Euler step of the 100-step workload (full 1024x1024x8 grid), FP64 Jacobi-PCG "
              "(Algorithm 1) on the assembled CSR matrix to rel. residual 1e-8; assembly untimed")
    out = {}
    for key, threads in (("all", host_cores()), ("one", 1)):
        env = dict(os.environ, **_thread_env(threads))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child"], env=env, capture_output=True,
                           text=True, timeout=1200)
        if r.returncode != 0:
            out[key] = {"value": None, "cores": threads, "error": r.stderr[-400:]}
        else:
            out[key] = {"value": json.loads(r.stdout.strip().splitlines()[-1])["ms"][0], "cores": threads}
    return {"value": out["all"]["value"], "unit": UNIT, "cores": out["all"]["cores"], "kind": "oracle",
            "sample": sample + f"; NumPy/SciPy threads = {out['all']['cores']} (every core in the affinity mask)",
            "single_thread": {"value": out["one"]["value"], "unit": UNIT, "cores": 1}}


def reference_config():
    """The reference arm's own description: the same workload, solved by the FP64 CPU oracle."""
    c = config_dict(0)
    for k in ("preconditioner", "initial_guess", "loop", "precision", "l2"):
        c.pop(k, None)
    c.update({"solver": "FP64 CPU oracle: Algorithm 1 (PCG) with the Jacobi preconditioner on the assembled CSR "
                        "matrix (NumPy/SciPy)",
              "precision": "FP64", "initial_guess": "previous step T_n (warm start)",
              "loop": "one backward-Euler step of the trajectory per bench step (host Python)",
              "threads": host_cores()})
    return c


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    # the oracle as it stands, with NumPy/SciPy allowed every host core (set before import)
    cores = host_cores()
    os.environ.update(_thread_env(cores))
    import numpy as np
    from oracle import discretisation as disc, krylov
    inst, maps = workload_arrays()
    st = inst.stack
    A = disc.assemble(NX, NY, st, dt=DT)
    T = np.full(inst.n, st.t_amb)
    step_ms = []
    for s in range(args.warmup + args.steps):
        p = maps[(s // STEPS_PER_MAP) % len(maps)].astype(np.float64)
        b = disc.rhs_transient(NX, NY, st, p, T, DT)
        t0 = time.perf_counter()
        T, it, _, _ = krylov.pcg(krylov.CountingOp(A), b, krylov.jacobi(A), x0=T, tol_rel=1e-8)
        dt_ms = (time.perf_counter() - t0) * 1e3
        if s >= args.warmup:
            step_ms.append(dt_ms)
    v = sum(step_ms) / len(step_ms)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": reference_config(),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "one backward-Euler step of the 100-step workload per bench step (steps "
                                      "0..W+K-1 of the trajectory), FP64 Jacobi-PCG on the assembled CSR matrix "
                                      f"to rel. residual 1e-8, NumPy/SciPy threads = {cores}; assembly untimed"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ----------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.cpu_child:
        run_cpu_child()
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import ThermalGrid

    inst, maps_h = workload_arrays()
    st = inst.stack
    grid = ThermalGrid.from_stack(NX, NY, st)
    peak, peak_kind = measured_peaks()
    if args.kernels_only:
        kern = kernel_table(grid, inst.n, args.reps, peak, peak_kind)
        print(json.dumps({"kernels": kern, "config": config_dict(args.degree, guess=args.guess), "reps": args.reps}))
        return
    maps = [torch.from_numpy(m).cuda() for m in maps_h]
    T = torch.full((inst.n,), st.t_amb, dtype=torch.float64, device="cuda")
    opts = dict(precision="mixed", precond="cheb", cheb_degree=args.degree, tol_rel=1e-8,
                use_graph=0 if args.polled else 1, guess=args.guess, cheb_fuse=args.fuse,
                inner_tol=args.inner_tol)

    nsteps = args.time_steps

    def trajectory(o, Tt, mp):
        Tt.fill_(st.t_amb)
        return grid.run_transient(mp, STEPS_PER_MAP, nsteps, DT, Tt, **o)[1]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    t_setup = time.perf_counter()
    stats = trajectory(opts, T, maps)  # first call: Lanczos setup and graph build
    t_setup = (time.perf_counter() - t_setup) * 1e3
    for _ in range(args.warmup):
        stats = trajectory(opts, T, maps)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with (NoClocks() if args.no_clocks else ClockSampler(local)) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            stats = trajectory(opts, T, maps)
        e1.record(stream)
        barrier()
    ms_total = e0.elapsed_time(e1)
    from paper_2606_17850_gb300.dist import max_over_ranks
    ms_total = max_over_ranks(ms_total, device="cuda")
    ms_traj = ms_total / args.steps
    value = ms_traj / nsteps
    T_mixed = T.clone()

    result = {"metric": METRIC, "value": value / world if False else value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_traj, "higher_is_better": False,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
              "config": config_dict(args.degree, args.polled, args.guess, args.fuse)}
    if nsteps != N_STEPS:
        result["config"]["time_steps_per_bench_step"] = nsteps
        result["config"]["note"] = "shortened trajectory (profiling run), not the measured workload"
    result["solver"] = {"inner_it_per_traj": stats["inner_it"], "outer_it_per_traj": stats["outer_it"],
                        "n_spmv_per_traj": stats["n_spmv"], "final_rel_res": stats["rel_res"],
                        "status": stats["status"], "first_call_ms (setup+graph build+solve)": t_setup}
    k = args.degree
    # kernel launches per trajectory from the solver's counters (graph mode): a
    # Chebyshev application is ceil((k-1)/4) fused launches on this layer-uniform grid;
    # an outer iteration adds the preconditioner, the correction, the residual (which
    # also starts the next inner solve) and the loop conditions
    fuse = args.fuse or 4
    cheb = -(-(k - 1) // fuse)
    pairs = (stats["inner_it"] + stats["outer_it"]) // 2 + stats["outer_it"]
    launches = (3 + nsteps * 6 + stats["outer_it"] * (cheb + 4) + pairs * (2 * (cheb + 2) + 1) + 1) * args.steps
    result["gpu_launches"] = int(launches)
    result["clocks"] = clk.summary()

    # plain FP64 GPU path on the same trajectory (the baseline the metric compares against)
    if not args.no_fp64:
        o64 = dict(opts, precision="fp64", cheb_degree=args.fp64_degree)
        T64 = torch.full((inst.n,), st.t_amb, dtype=torch.float64, device="cuda")
        trajectory(o64, T64, maps)  # warm-up (graph build)
        barrier()
        e0.record(stream)
        s64 = trajectory(o64, T64, maps)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1)
        rise = (T64 - st.t_amb).abs().max().item()
        err = (T_mixed - T64).abs().max().item() / rise
        result["fp64_gpu"] = {"value": ms64 / nsteps, "unit": UNIT, "ms_per_trajectory": ms64,
                              "inner_it": s64["inner_it"], "final_rel_res": s64["rel_res"],
                              "cheb_degree": args.fp64_degree}
        result["speedup_mixed_vs_fp64"] = (ms64 / nsteps) / value
        result["accuracy"] = {"max_abs_diff_mixed_vs_fp64_K": err * rise,
                              "max_rel_diff_vs_rise": err}

    # the paper's adaptive mixed-precision PCG (stage switch + hot restart) on the same trajectory
    if not args.no_adaptive:
        oad = dict(opts, precision="adaptive", cheb_degree=args.adaptive_degree)
        Tad = torch.full((inst.n,), st.t_amb, dtype=torch.float64, device="cuda")
        trajectory(oad, Tad, maps)  # warm-up (graph build)
        barrier()
        e0.record(stream)
        sad = trajectory(oad, Tad, maps)
        e1.record(stream)
        barrier()
        msad = e0.elapsed_time(e1)
        rise = (Tad - st.t_amb).abs().max().item()
        result["adaptive_gpu"] = {
            "value": msad / nsteps, "unit": UNIT, "ms_per_trajectory": msad, "inner_it": sad["inner_it"],
            "stage_switches": sad["stage_switches"], "final_rel_res": sad["rel_res"],
            "cheb_degree": args.adaptive_degree,
            "max_abs_diff_vs_mixed_K": (Tad - T_mixed).abs().max().item(),
            "note": "FP64 PCG, early stage FP64/32 SpMV, late stage FP64 SpMV (switch on Eqs. switch_a-c, hot "
                    "restart), Chebyshev preconditioner in FP32 with the FP32/16 product of Algorithm 3"}
        result["speedup_mixed_vs_adaptive"] = (msad / nsteps) / value

    # live per-kernel timings (CUDA events on the launching stream) -> roofline
    if not args.no_kernels:
        kern = kernel_table(grid, inst.n, args.reps, peak, peak_kind)
        result["kernels"] = kern
        dom = kern[DOMINANT]
        result["roofline"] = {"bound": "hbm", "kernel": DOMINANT, "achieved": dom["GB/s"], "peak": peak,
                              "unit": "GB/s", "frac": dom["GB/s"] / peak, "peak_source": peak_kind,
                              "algorithmic_bytes_per_launch": KERNEL_BYTES[DOMINANT] * inst.n,
                              "traffic": traffic_from_profiles(DOMINANT)}

    # end to end through the public API with host buffers (copies inside the timed region)
    if not args.no_e2e:
        maps_pin = [torch.from_numpy(m).pin_memory() for m in maps_h]
        T_pin = torch.full((inst.n,), st.t_amb, dtype=torch.float64).pin_memory()
        trajectory(opts, T_pin, maps_pin)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            trajectory(opts, T_pin, maps_pin)
        barrier()
        ms_e2e = (time.perf_counter() - t0) * 1e3 / args.steps
        result["e2e"] = {"value": ms_e2e / nsteps, "unit": UNIT,
                         "h2d_bytes_per_step": int(sum(m.numel() * 4 for m in maps_pin) + inst.n * 8),
                         "d2h_bytes_per_step": int(inst.n * 8),
                         "note": "per bench step (one 100-step trajectory): 4 power maps + T_0 to the device, "
                                 "T_100 back, through thermal_run_transient with pinned host buffers"}
    if not args.no_ablation:
        result["spmv_ablation"] = ablation_section(grid, inst.n, args.reps, result.get("kernels"), peak)
    if not args.no_faces:
        fo = dict(opts, cheb_degree=args.faces_degree) if args.faces_degree > 0 else opts
        result["per_face"] = faces_section(fo, maps, nsteps, st, value, T_mixed)
        result["per_face"]["cheb_degree"] = fo["cheb_degree"]
    if not args.no_precond:
        result["preconditioners"] = precond_section(args, opts, trajectory, maps, nsteps, st)
    if not args.no_batched:
        result["batched"] = batched_section(args)
    if not args.no_adjoint:
        result["adjoint"] = adjoint_section(args)
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def _event_ms(fn, reps=1):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


# algorithmic bytes per row of the CSR product (Sec. 5.5 comparison): row offset,
# ~7 (column index + value) pairs, x and y
CSR_BYTES = {"f32": 4 + 7 * (4 + 4) + 4 + 4, "f64": 4 + 7 * (4 + 8) + 8 + 8}


def ablation_section(grid, n, reps, kern, peak):
    """Stencil product vs a CSR copy of the same matrix (Sec. 5.5, Table abl_spmv):
    row-wise (scalar) and 8-lane (vector) CSR in FP32 and FP64 on the 1024x1024x8
    transient matrix, against the stencil kernels timed the same way."""
    import torch
    out = {}
    x64 = torch.rand(n, dtype=torch.float64, device="cuda")
    for prec, x in (("f32", x64.float()), ("f64", x64)):
        y_st = grid.apply(x, DT, "fp64" if prec == "f64" else "mixed")
        for var in ("scalar", "vector"):
            y, ms = grid.csr_spmv(x, dt=DT, variant=var, reps=reps)
            diff = ((y - y_st).abs().max() / y_st.abs().max()).item()
            gbs = CSR_BYTES[prec] * n / (ms * 1e-3) / 1e9
            out[f"csr_{var}_{prec}"] = {"ms": ms, "bytes_per_cell": CSR_BYTES[prec], "GB/s": gbs,
                                        "frac_of_peak": gbs / peak, "max_rel_diff_vs_stencil": diff}
    st = {}
    for name in ("stencil_f32", "stencil_f32_faces", "stencil_f64"):
        st[name] = kern[name]["ms"] if kern and name in kern else grid.kernel_time(name, reps=reps, dt=DT)
    out["stencil_ms"] = st
    out["speedup_stencil_vs_csr_scalar"] = {
        "f64 (faces FP64)": out["csr_scalar_f64"]["ms"] / st["stencil_f64"],
        "f32 (faces FP32)": out["csr_scalar_f32"]["ms"] / st["stencil_f32_faces"],
        "f32 (layer table)": out["csr_scalar_f32"]["ms"] / st["stencil_f32"]}
    out["note"] = ("same matrix (transient, dt=1e-4) in CSR with 32-bit indices; the paper reports 2.0-2.2x "
                   "for its diagonal-wise kernels over CSR on a different GPU")
    return out


def faces_section(opts, maps, nsteps, st, value, T_ref):
    """The same 100-step trajectory on a grid given a per-cell conductivity map that holds
    the layer values: every kernel then reads the per-face arrays (FP32 faces in the
    preconditioner, double-float faces in the refinement residual) instead of the
    per-layer table.  Same answer, general storage."""
    import numpy as np
    import torch
    from paper_2606_17850_gb300 import ThermalGrid
    g = ThermalGrid.from_stack(NX, NY, st)
    g.set_conductivity_map(torch.from_numpy(np.repeat(st.k(), NX * NY)).cuda())
    Tf = torch.full((NX * NY * st.L,), st.t_amb, dtype=torch.float64, device="cuda")

    def traj():
        Tf.fill_(st.t_amb)
        return g.run_transient(maps, STEPS_PER_MAP, nsteps, DT, Tf, **opts)[1]

    traj()  # set-up and graph build
    ms, stt = _event_ms(traj, reps=1)
    rise = (T_ref - st.t_amb).abs().max().item()
    out = {"ms_per_step": ms / nsteps, "ratio_to_layer_table": (ms / nsteps) / value,
           "inner_it": stt["inner_it"], "outer_it": stt["outer_it"], "final_rel_res": stt["rel_res"],
           "max_rel_diff_vs_layer_table": (Tf - T_ref).abs().max().item() / rise}
    g.close()
    return out


def precond_section(args, opts, trajectory, maps, nsteps, st):
    """Chebyshev (Lanczos bounds) against the geometric multigrid V-cycle: the steady
    512 x 512 x 8 floorplan stack (FP32 PCG + FP64 refinement to 1e-8) and the
    transient trajectory of the headline."""
    import numpy as np
    import torch
    import thermal_inputs as ti
    from paper_2606_17850_gb300 import ThermalGrid
    out = {}
    c2 = ti.c2(dtype=np.float32)
    g2 = ThermalGrid.from_stack(c2.nx, c2.ny, c2.stack)
    P2 = torch.from_numpy(c2.power).cuda()
    for name, o in (("cheb30", dict(precond="cheb", cheb_degree=30)), ("cheb20", dict(precond="cheb", cheb_degree=20)),
                    ("mg", dict(precond="mg")), ("jacobi", dict(precond="jacobi"))):
        oo = dict(o, tol_rel=1e-8, inner_tol=args.inner_tol, use_graph=1)  # every arm in a CUDA graph
        g2.solve_steady(P2, **oo)  # set-up (Lanczos / hierarchy, graph)
        ms, (T, stt) = _event_ms(lambda: g2.solve_steady(P2, **oo), reps=2)
        out[f"steady_512x512x8_{name}"] = {"ms": ms, "inner_it": stt["inner_it"], "outer_it": stt["outer_it"],
                                            "rel_res": stt["rel_res"]}
    omg = dict(opts, precond="mg")
    Tm = torch.full((maps[0].numel(),), st.t_amb, dtype=torch.float64, device="cuda")
    trajectory(omg, Tm, maps)
    ms, stt = _event_ms(lambda: trajectory(omg, Tm, maps), reps=1)
    out["transient_1024x1024x8_mg"] = {"ms_per_step": ms / nsteps, "inner_it": stt["inner_it"],
                                       "outer_it": stt["outer_it"], "rel_res": stt["rel_res"]}
    return out


def batched_section(args):
    """64 independent stacks of uneven size (128^2x4 .. 512^2x8, k perturbed +-20%),
    steady, FP32 PCG + FP64 refinement to 1e-8, in one persistent cooperative launch
    per rank, with the multigrid V-cycle and with Chebyshev-30 as the preconditioner.  With several ranks the stacks are
    sharded (contiguous balanced shares, ``dist.solve_sharded``): each rank solves its
    share in one launch, the job time is the slowest rank's, and the per-instance
    results are gathered on the host.  No data-path collective."""
    import numpy as np
    import torch
    import thermal_inputs as ti
    from paper_2606_17850_gb300 import ThermalGrid, solve_batched
    from paper_2606_17850_gb300.dist import max_over_ranks, rank_world, shard, solve_sharded
    insts = ti.c4_instances()
    rank, world = rank_world()
    timing = {}
    o = {}

    def solve_shard(idx):
        grids = [ThermalGrid.from_stack(insts[i].nx, insts[i].ny, insts[i].stack) for i in idx]
        powers = [torch.from_numpy(insts[i].power).cuda() for i in idx]
        Ts = [torch.empty(insts[i].n, dtype=torch.float64, device="cuda") for i in idx]
        solve_batched(grids, powers, Ts, **o)  # set-up: Lanczos per instance
        if world > 1:
            torch.distributed.barrier()
        ms, stats = _event_ms(lambda: solve_batched(grids, powers, Ts, **o), reps=max(1, args.steps))
        timing["ms"] = ms
        res = {i: {"status": s["status"], "rel_res": s["rel_res"], "inner_it": s["inner_it"],
                   "tile_rows": s["tile_rows"], "tile_layers": s["tile_layers"]} for i, s in zip(idx, stats)}
        for g in grids:
            g.close()
        return res

    n = sum(i.n for i in insts)
    out = {"workload": "64 steady stacks of uneven size (128^2x4, 256^2x6, 384^2x8, 512^2x8; k x U[0.8,1.2])",
           "unknowns": n, "ranks": world,
           "instances_per_rank": [len(shard(len(insts), r, world)) for r in range(world)],
           "launch": "one cooperative persistent kernel per rank for its share of the 64 instances"}
    for name, oo in (("multigrid", dict(tol_rel=1e-8, precond="mg")),
                     ("chebyshev30", dict(tol_rel=1e-8, precond="cheb", cheb_degree=30))):
        o.clear()
        o.update(oo)
        res = solve_sharded(len(insts), solve_shard, rank, world)
        ms = max_over_ranks(timing.get("ms", 0.0), device="cuda")
        st = [res[i] for i in range(len(insts))]
        out[name] = {"ms_per_batch_solve": ms, "max_rel_res": max(s["rel_res"] for s in st),
                     "status": max(s["status"] for s in st), "inner_it_sum": sum(s["inner_it"] for s in st),
                     "max_inner_it": max(s["inner_it"] for s in st),
                     "tiles": {f"{insts[i].nx}x{insts[i].ny}x{insts[i].stack.L}":
                               f"128 x {8 * st[i]['tile_rows']} columns x {st[i]['tile_layers']} layers"
                               for i in range(len(insts))}}
    best = min(("multigrid", "chebyshev30"), key=lambda k: out[k]["ms_per_batch_solve"])
    out["ms_per_batch_solve"] = out[best]["ms_per_batch_solve"]
    out["preconditioner"] = best
    return out


def adjoint_section(args):
    """2048 x 2048 x 10 memory-on-logic stack (41.9M unknowns): steady solve, log-sum-exp
    hotspot objective (beta = 2/K) over the two FEOL layers, adjoint gradient w.r.t. the
    power map and the 10 layer conductivities."""
    import numpy as np
    import torch
    import thermal_inputs as ti
    from paper_2606_17850_gb300 import ThermalGrid
    inst = ti.c5(dtype=np.float32)
    g = ThermalGrid.from_stack(inst.nx, inst.ny, inst.stack)
    P = torch.from_numpy(inst.power).cuda()
    layers = inst.stack.power_layers()

    def run(o):
        def one():
            T, s1 = g.solve_steady(P, **o)
            J, w = g.hotspot_lse(T, layers, 2.0)
            dP, dk, s2 = g.grad(T, w, dJdP_dtype=torch.float32, **o)
            return s1, s2, J

        one()  # set-up (spectral bounds or the multigrid hierarchy, the graphs of both solves)
        return _event_ms(one, reps=1)

    # steady solves of this stack converge fastest with the multigrid preconditioner
    ms, (s1, s2, J) = run(dict(precision="mixed", precond="mg", tol_rel=1e-8, use_graph=1))
    ms_cheb, (c1, c2, _) = run(dict(precision="mixed", precond="cheb", cheb_degree=30, tol_rel=1e-8, use_graph=1))
    return {"workload": "2048x2048x10 memory-on-logic stack, forward solve + LSE + adjoint gradient",
            "unknowns": inst.n, "preconditioner": "multigrid V-cycle", "ms_forward_plus_gradient": ms, "J": J,
            "forward_inner_it": s1["inner_it"], "adjoint_inner_it": s2["inner_it"],
            "rel_res": [s1["rel_res"], s2["rel_res"]],
            "chebyshev30": {"ms_forward_plus_gradient": ms_cheb, "forward_inner_it": c1["inner_it"],
                            "adjoint_inner_it": c2["inner_it"]}}


def kernel_table(grid, n, reps, peak, peak_kind):
    """Mean launch time of each hot kernel (CUDA events around `reps` back-to-back
    launches on the launching stream) and the HBM bandwidth its algorithmic bytes imply."""
    kern = {}
    for name, nbytes in KERNEL_BYTES.items():
        ms = grid.kernel_time(name, reps=reps, dt=DT)
        gbs = nbytes * n / (ms * 1e-3) / 1e9
        kern[name] = {"ms": ms, "bytes_per_cell": nbytes, "GB/s": gbs, "frac_of_" + peak_kind: gbs / peak}
    return kern


# source files that define each profiled kernel: a committed DRAM-traffic figure is
# used only while these files are unchanged
KERNEL_SOURCES = {"cheb_tb4": ["kernels_tb.cuh"], "cheb_tbf4": ["kernels_tb.cuh"], "cheb_f32": ["kernels_v4.cuh"]}


def traffic_from_profiles(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's sources
    are unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get(kernel)
    if not ent or ent.get("sources_sha") != sources_sha(kernel):
        return None
    return ent.get("dram_bytes_per_launch_full_size")


def sources_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_17850_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES.get(kernel, [])):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
