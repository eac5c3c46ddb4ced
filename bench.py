"""Benchmark: Laplace solves/s to a 1e-10 relative residual on the 4097 x 4097 grid.

Workload (seeded, synthetic): 4097 x 4097, dx = dy = 1/4096, every edge carries
sum_{k=1..8} a_k sin(k pi s) with a_k ~ U[-1, 1], interior zero. One step solves it,
from the same initial field, with
  * red-black SOR at w_opt = 2 / (1 + sin(pi/4096)), residual tested every 100 sweeps, its
    neighbour sums paired along diagonals, (W + S) + (E + N) (LAP_SUM_DIAGONAL), and
  * the V(2,2) multigrid cycle down to 5 x 5, residual tested every cycle,
each to ||r||_2 <= 1e-10 ||r_0||_2. value = solves per second over all ranks. The ADI half
sweeps and the Jacobi sweep are timed per sweep in the same run ("kernels").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run, one process per GPU, each solving its own
replica (no data-path collective); timings are the max over ranks. `--impl reference`
times the CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = 4097
H = 1.0 / 4096
TOL = 1e-10
SOR_CHECK = 100
METRIC = "Laplace solves/s to 1e-10 residual"
WORKLOAD = "4097x4097 Laplace, sine-series Dirichlet edges, RB-SOR(w_opt) + V(2,2) multigrid"
HBM_PEAK = None  # read from MEASURED_PEAKS.json when present
# FP64 pipe: 2 operations (add, multiply or fused multiply-add) per clock per SM on GB300,
# 152 SMs, 2070 MHz maximum SM clock -> 0.629 T FP64 operations/s (nominal 1.25 TFLOP/s
# counts an fma as two flops)
FP64_OPS_PEAK = 152 * 2 * 2.070e9
# FP64 operations per point of one red-black SOR colour pass with the neighbour sum paired
# along diagonals (the timed solve): 2 adds (the point's E + N pair, then the sum with the W + S
# pair carried from the previous point of the diagonal), 1 multiply by (1-w), 1 fma; the
# multiply by 1/d = 1/4 runs on the integer pipe. In the paper's summation order the neighbour
# sum takes 3 adds: 5 operations.
SOR_OPS_PER_POINT = 4
SOR_OPS_PER_POINT_PAPER_ORDER = 5
SOR_BYTES_PER_POINT = 16  # algorithmic bytes of a sweep: read 8, write 8 bytes per point
# FP64 operations per unknown of a zebra line half sweep, form A, beta = 1 (the kernels' count):
# 1 add (right-hand side), 1 fma forward, 1 fma back, 2 for the relaxed output, plus 2 fmas in the
# first K0 = 34 positions of each 127-unknown chunk (the boundary layer): 5 + 68/127
LINE_OPS_PER_POINT = 5.54
INTERIOR = (M - 2) * (N - 2)
ORACLE_BATCH_SAMPLE = (0, 85, 170, 255)  # problems of the 256-grid batch checked against the oracle


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--latency-solves", type=int, default=30, help="extra MG solves for p50/p99")
    ap.add_argument("--serving-requests", type=int, default=10000,
                    help="requests served across the load levels of the serving workload")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is
    unchanged since the capture (the sha256 of its source file and of the device helpers
    it includes is recorded beside the number)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    csrc = os.path.join(ROOT, "paper_2208_02427_gb300", "csrc")
    try:
        h = hashlib.sha256()
        for name in ("point_kernels.cu", "lap_device.cuh"):
            h.update(open(os.path.join(csrc, name), "rb").read())
        digest = h.hexdigest()[:16]
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
                return float(parts[2])
    except OSError:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if bus_id:
                cmd += ["-i", bus_id]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        rows = []
        for line in open(self.file.name):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def bus_id(dev):
    import torch
    p = torch.cuda.get_device_properties(dev)
    try:
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except AttributeError:
        return None


# ---- the oracle on the host (cpu_baseline and the reference arm) ----------------------

def oracle_sample(psi, sor_sweeps: int, sor_total: int, threads: int = 0):
    """Time the oracle on a bounded sample of one step's work: sor_sweeps calls of its
    red-black SOR sweep on one buffer (scaled to sor_total, the sweeps this input needs), and
    its whole V(2,2) multigrid solve to 1e-10 (run in full). With threads > 1 the SOR sweeps
    run in the threaded timing wrapper (bitwise the oracle's sweeps; rows split across host
    threads). Returns the baseline and the oracle's multigrid solution."""
    import ctypes as C

    import numpy as np

    import oracle as ora
    from paper_2208_02427_gb300 import workloads as wl
    w = wl.w_opt_sor(M, N)
    buf = np.ascontiguousarray(psi, dtype=np.float64).copy()
    t0 = time.perf_counter()
    if threads > 1:
        buf = ora.mt_sor_rb_sweeps(buf, w, sor_sweeps, 1.0, threads)
    else:
        ptr = buf.ctypes.data_as(C.POINTER(C.c_double))
        lib = ora.lib()
        for _ in range(sor_sweeps):
            lib.ora_sor_sweep(M, N, 1.0, w, ora.RB, ptr, None)
    t_sor = (time.perf_counter() - t0) / sor_sweeps
    t0 = time.perf_counter()
    sol, info = ora.solve(psi, method=ora.MG, ordering=ora.RB, dx=H, dy=H, tol=TOL, max_iter=100)
    t_mg = time.perf_counter() - t0
    solve_s = t_sor * sor_total + t_mg
    cores = max(1, threads)
    return {"value": 2.0 / solve_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{sor_sweeps} RB-SOR sweeps ({t_sor*1e3:.1f} ms each, "
                      f"{'threaded over ' + str(threads) + ' host threads' if threads > 1 else 'single-threaded'}) "
                      f"scaled to {sor_total} sweeps, + the whole V(2,2) multigrid solve to 1e-10 "
                      f"({info['iters']} cycles, {t_mg:.2f} s, single-threaded) of the C oracle "
                      f"on the 4097^2 input",
            "seconds_per_solve_pair": solve_s, "mg_cycles": info["iters"]}, sol


def _oracle_batched_problem(job):
    """One problem of the batched workload solved by the oracle's V(2,2) multigrid to 1e-10
    (run in a spawned worker process); returns its wall time and cycle count."""
    m, n, seed = job
    import oracle as ora
    from paper_2208_02427_gb300 import workloads as wl
    psi = wl.random_ring(m, n, seed=seed)
    t0 = time.perf_counter()
    _, info = ora.solve(psi, method=ora.MG, ordering=ora.RB, dx=1.0, dy=1.0, tol=TOL, max_iter=100)
    return time.perf_counter() - t0, info["iters"]


def oracle_batched_sample(count=4096, every=16):
    """The batched workload's oracle baseline: every `every`-th problem of the 4096 solved by
    the oracle, one problem per worker process over all host cores (spawned: the parent holds
    a CUDA context). solves/s = problems / wall time of the pool."""
    import multiprocessing as mp

    from paper_2208_02427_gb300 import workloads as wl
    shapes = wl.batch_shapes(count, seed=wl.SEED_BASE + 2)
    jobs = [(m, n, wl.SEED_BASE + 2 + 10 * k) for k, (m, n) in enumerate(shapes)][::every]
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_batched_problem, jobs[:cores])  # workers import and build once
        t0 = time.perf_counter()
        res = pool.map(_oracle_batched_problem, jobs)
        wall = time.perf_counter() - t0
    return {"value": len(jobs) / wall, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(jobs)} of the {count} problems (every {every}th), V(2,2) to 1e-10, "
                      f"one problem per process over {cores} host processes; "
                      f"{sum(t for t, _ in res):.2f} s of single-core oracle time in {wall:.2f} s",
            "max_cycles": max(c for _, c in res)}


def oracle_serving_estimate(work, gpu_solves_per_s):
    """The serving workload's oracle baseline, extrapolated: for each request size of the
    saturation run, one oracle RB-SOR sweep and one V(2,2) cycle (with its residual norm) are
    timed once on one host core; a request costs its unit times the iterations the GPU ran for it
    (the oracle's red-black and multigrid iterates follow the same counts), plus one residual norm
    per 50 SOR sweeps (the server's test period). Mixed-precision requests are charged as the
    oracle's FP64 multigrid."""
    import numpy as np

    import oracle as ora
    from paper_2208_02427_gb300 import workloads as wl
    units = {}
    for m, n in sorted({(m, n) for m, n, _, _ in work}):
        psi = wl.random_interior(wl.random_ring(m, n, seed=7), seed=8)
        t0 = time.perf_counter()
        reps = max(1, int(2e6 // (m * n)))
        for _ in range(reps):
            ora.sor_sweep(psi, 1.9, 1.0, ora.RB)
        sweep = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            ora.defect_norm(psi, 1.0)
        norm = (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        ora.solve(psi, method=ora.MG, ordering=ora.RB, tol=0.0, max_iter=1)
        cycle = time.perf_counter() - t0
        units[(m, n)] = (sweep + norm / 50.0, cycle + norm)
    seconds = sum(units[(m, n)][0 if method == "sor" else 1] * max(1, it)
                  for m, n, method, it in work)
    cores = os.cpu_count() or 1
    value = len(work) / seconds if seconds > 0 else None
    return {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"extrapolated: the {len(work)} requests of the saturation run, each charged "
                      f"its size's oracle RB-SOR sweep (+ a norm per 50 sweeps) or V(2,2) cycle "
                      f"(+ norm), timed once per size on one host core, times the GPU's iteration "
                      f"count; {len(units)} sizes, {seconds:.1f} s of oracle time",
            "all_cores_ideal": {"value": value * cores if value else None, "cores": cores,
                                "how": "the single-core estimate with requests spread evenly over "
                                       "all host cores (not run)"},
            "gpu_over_oracle_single_core": gpu_solves_per_s / value if value else None}


# Sweeps of this input to 1e-10 (RB-SOR tested every 100 sweeps; in either summation order the
# oracle's RB-SOR iterates are bitwise identical to the GPU's in that order, and both orders stop
# at the same test, so the oracle needs the same count).
SOR_SWEEPS_TO_TOL = 15600


def reference_arm(args):
    from paper_2208_02427_gb300 import replicas
    from paper_2208_02427_gb300 import workloads as wl
    rank, size, _ = replicas.world()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    psi = wl.sine_edges(M, N, seed=wl.SEED_BASE + 1)
    samples, wall = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s, _ = oracle_sample(psi, 4, SOR_SWEEPS_TO_TOL)
        if k >= args.warmup:
            samples.append(s)
            wall.append(time.perf_counter() - t0)
    value = statistics.median(s["value"] for s in samples)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # the wall time of each sampled step as it ran; the value is extrapolated from it
            "ms_per_step": statistics.median(wall) * 1e3,
            "value_is_extrapolated": True,
            "extrapolation": "value = 2 solves / (seconds per sampled oracle RB-SOR sweep x "
                             f"{SOR_SWEEPS_TO_TOL} sweeps + seconds of the whole oracle multigrid "
                             "solve); each step runs 4 SOR sweeps and the whole multigrid solve",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": "4097x4097", "tol": TOL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": samples[0]["sample"] + " (each step one such sample; "
                                       "the SOR part is extrapolated from the sampled sweeps)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- our arm ----------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch
    from paper_2208_02427_gb300 import binding as b
    from paper_2208_02427_gb300 import replicas
    from paper_2208_02427_gb300 import workloads as wl

    rank, size, local = replicas.init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    lap = b.Laplace(device=local)
    psi_host = wl.sine_edges(M, N, seed=wl.SEED_BASE + 1)
    init = b.to_field(psi_host, dev)
    work = b.field(M, N, dev)
    w_sor = wl.w_opt_sor(M, N)
    sor_kw = dict(method="sor", w=w_sor, tol=TOL, check_every=SOR_CHECK, max_iter=200000,
                  sum_order="diagonal")
    mg_kw = dict(method="mg", tol=TOL, nu1=2, nu2=2, coarsest_min=5, max_iter=100)

    def step(record=None):
        out = {}
        for name, kw in (("sor", sor_kw), ("mg", mg_kw)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                work.copy_(init)
                e0.record(stream)
                info = lap.solve(work, H, H, stream=stream, **kw)
                e1.record(stream)
            stream.synchronize()
            if info["status"] != "converged":
                raise RuntimeError(f"{name} did not converge: {info}")
            out[name] = dict(info, ms=e0.elapsed_time(e1))
        return out

    for _ in range(args.warmup):
        step()
    replicas.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(bus_id(dev))
    launches0 = b.kernel_launches()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    per_step = [step() for _ in range(args.steps)]
    t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    launches = b.kernel_launches() - launches0
    clk = clocks.stop()
    replicas.barrier()
    local_ms = t_start.elapsed_time(t_end)
    total_ms = replicas.reduce_scalar(local_ms, "max")
    solves = replicas.reduce_scalar(2.0 * args.steps, "sum")
    value = solves / (total_ms / 1e3)

    # ---- dominant kernel: one red-black SOR colour pass, inside the solve's graphs -------
    # The solve replays check periods (100 sweeps + the residual norm + the device-side test)
    # as one CUDA graph. Timing one-period solves of 200 and 2200 sweeps the same way and
    # differencing leaves 2000 in-graph sweeps (4000 colour passes): the per-launch time of
    # the kernel as it runs inside the timed step.
    fma_rate = lap.fp64_rate()  # measured FP64 fma issue rate of this device (probe kernel)

    def sor_period_ms(sweeps, reps=3, **extra):
        kw = dict(sor_kw, tol=0.0, max_iter=sweeps, check_every=sweeps, **extra)
        times = []
        for r in range(2 + reps):  # two warm-ups: the period graph is captured on first use
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                work.copy_(init)
                e0.record(stream)
                lap.solve(work, H, H, stream=stream, **kw)
                e1.record(stream)
            stream.synchronize()
            if r >= 2:
                times.append(e0.elapsed_time(e1))
        return statistics.median(times)

    t_short, t_long = sor_period_ms(200), sor_period_ms(2200)
    launch_s = (t_long - t_short) / 1e3 / (2 * 2000)
    # the same in the paper's summation order (rb_colour_kernel), for comparison
    launch_paper_s = (sor_period_ms(2200, sum_order="paper") -
                      sor_period_ms(200, sum_order="paper")) / 1e3 / (2 * 2000)
    pts_per_launch = INTERIOR / 2
    ops = SOR_OPS_PER_POINT * pts_per_launch / launch_s
    # the algorithmic bytes of a red-black sweep are 16 per point (read and write each point
    # once); a colour pass updates half the points: 16 B x pts_per_launch per launch
    hbm_gbs = SOR_BYTES_PER_POINT * pts_per_launch / launch_s / 1e9
    peaks = measured_peaks()
    traffic = recorded_traffic("rb_diag_kernel")
    pipe_busy = recorded_traffic("rb_diag_kernel:fp64_pipe_active")
    sor_step_ms = statistics.median(s["sor"]["ms"] for s in per_step)
    sor_sweeps = per_step[-1]["sor"]["iters"]
    roofline = {"bound": "alu",
                "kernel": "rb_diag_kernel (SOR, one colour, neighbour sums paired along diagonals)",
                "achieved": ops / 1e12, "peak": fma_rate / 1e12, "unit": "Top/s",
                "frac": ops / fma_rate, "traffic": traffic,
                "peak_source": "measured live: lap_fp64_rate, FP64 fma chains on register "
                               "operands over 4 blocks x 256 threads per SM",
                "peak_derived": FP64_OPS_PEAK / 1e12,
                "frac_of_derived": ops / FP64_OPS_PEAK,
                "ops_per_point": SOR_OPS_PER_POINT, "points_per_launch": pts_per_launch,
                "ops_issued_per_point": SOR_OPS_PER_POINT + 1.0 / 6,  # + a fresh pair per 6-point walk
                "ncu_fp64_pipe_active": pipe_busy,
                "ms_per_launch": launch_s * 1e3,
                "ms_per_launch_how": "in-graph: (one-period solve of 2200 sweeps - one of 200) / "
                                     "4000 colour passes, CUDA events on the solve stream",
                "step_check": {"sor_solve_ms": sor_step_ms, "passes": 2 * sor_sweeps,
                               "passes_x_ms_per_launch": 2 * sor_sweeps * launch_s * 1e3},
                "hbm_view": {"achieved_gbs": hbm_gbs, "peak_gbs": peaks.get("hbm_gbs"),
                             "frac": hbm_gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                             "bytes_per_point_per_sweep": SOR_BYTES_PER_POINT},
                "paper_order_kernel": {
                    "kernel": "rb_colour_kernel (SOR, one colour, (E + W) + (N + S))",
                    "ms_per_launch": launch_paper_s * 1e3,
                    "ops_per_point": SOR_OPS_PER_POINT_PAPER_ORDER,
                    "achieved": SOR_OPS_PER_POINT_PAPER_ORDER * pts_per_launch / launch_paper_s / 1e12,
                    "frac": SOR_OPS_PER_POINT_PAPER_ORDER * pts_per_launch / launch_paper_s / fma_rate,
                    "traffic": recorded_traffic("rb_colour_kernel")}}

    # ---- other hot-path kernels, per sweep ------------------------------------------------
    def kernel_ms(fn, reps):
        with torch.cuda.stream(stream):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    def alu_entry(ms, ops_pp, bytes_pp):
        s_ = ms / 1e3
        return {"ms": ms, "fp64_ops_per_point": ops_pp,
                "achieved_top_s": ops_pp * INTERIOR / s_ / 1e12,
                "frac_of_measured_fp64": ops_pp * INTERIOR / s_ / fma_rate,
                "alg_bytes_per_point": bytes_pp, "gbs": bytes_pp * INTERIOR / s_ / 1e9,
                "hbm_frac": (bytes_pp * INTERIOR / s_ / 1e9 / peaks["hbm_gbs"]
                             if peaks.get("hbm_gbs") else None)}

    other = b.field(M, N, dev)
    other.copy_(init)
    kernels = {}
    ms = kernel_ms(lambda: b.smooth(work, w=1.0, nsweeps=1, dx=H, dy=H, stream=stream), 50)
    # GS at beta = 1 without a source term: the three adds of the neighbour sum (the multiply
    # by 1/4 runs on the integer pipe)
    kernels["gs_sweep"] = alu_entry(ms, 3, 16)
    # line relaxation, form A at beta = 1: LINE_OPS_PER_POINT FP64 operations per unknown;
    # 24 algorithmic bytes per point (per zebra colour the other colour's lines read, the
    # line read and written)
    ms = kernel_ms(lambda: lap.line_sweep(work, 1.3, "A", 0, H, H, stream=stream), 10)
    kernels["adi_x_half"] = alu_entry(ms, LINE_OPS_PER_POINT, 24)
    ms = kernel_ms(lambda: lap.line_sweep(work, 1.3, "A", 1, H, H, stream=stream), 10)
    kernels["adi_y_half"] = alu_entry(ms, LINE_OPS_PER_POINT, 24)
    ms = kernel_ms(lambda: b.jacobi_sweep(init, other, H, H, stream=stream), 20)
    kernels["jacobi_sweep_with_ring_copy"] = {"ms": ms}

    # ---- latency distribution of multigrid solves ----------------------------------------
    lat = []
    for _ in range(args.latency_solves):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            work.copy_(init)
            e0.record(stream)
            lap.solve(work, H, H, stream=stream, **mg_kw)
            e1.record(stream)
        stream.synchronize()
        lat.append(e0.elapsed_time(e1))
    lat.sort()
    latency = {"mg_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                         "n": len(lat)},
               "sor_ms": {"p50": statistics.median(s["sor"]["ms"] for s in per_step), "n": len(per_step)}}

    # ---- line relaxation to 1e-10: zebra SLOR by x-lines (form A) at its optimum ------------
    # Zebra ADI (x-lines then y-lines) is not accelerated by w on fine grids (its iteration
    # count grows like h^-2, about 1e6 iterations here); zebra SLOR is consistently ordered,
    # so at Young's optimum it converges like h^-1 and reaches 1e-10 in bounded time.
    w_slor = wl.w_opt_slor(M, N)
    slor_kw = dict(method="slor", w=w_slor, line_form="A", tol=TOL, check_every=SOR_CHECK,
                   max_iter=400000)
    with torch.cuda.stream(stream):
        work.copy_(init)
        lap.solve(work, H, H, stream=stream, **dict(slor_kw, tol=0.0, max_iter=2 * SOR_CHECK))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        work.copy_(init)
        e0.record(stream)
        slor_info = lap.solve(work, H, H, stream=stream, **slor_kw)
        e1.record(stream)
    stream.synchronize()
    slor_ms = e0.elapsed_time(e1)
    line_solve = {"method": "zebra line SOR by x-lines, form A (Eqs. 8-9), residual tested every "
                            f"{SOR_CHECK} sweeps", "w": w_slor, "iters": slor_info["iters"],
                  "status": slor_info["status"], "ms": slor_ms, "solves_per_s": 1e3 / slor_ms,
                  "r_final_over_r0": slor_info["r_final"] / slor_info["r0"],
                  "ms_per_sweep": slor_ms / max(1, slor_info["iters"]),
                  "adi": "zebra ADI is not run to 1e-10: not accelerated by w on this grid (h^-2 "
                         "growth of its iteration count, about 1e6 iterations); its half sweeps "
                         "are timed under kernels"}

    # ---- mixed precision: FP32 V-cycles inside FP64 defect correction ---------------------
    def timed_solve(field, src, kw, h):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            field.copy_(src)
            e0.record(stream)
            info = lap.solve(field, h, h, stream=stream, **kw)
            e1.record(stream)
        stream.synchronize()
        return info, e0.elapsed_time(e1)

    def exact_solution(psi):
        """The exact discrete solution of the 5-point system for the ring of psi (beta = 1):
        a DST-I diagonalises the interior operator (host, FP64; measurement only)."""
        import scipy.fft
        n_, m_ = psi.shape
        rhs = np.zeros((n_ - 2, m_ - 2))
        rhs[:, 0] += psi[1:-1, 0]
        rhs[:, -1] += psi[1:-1, -1]
        rhs[0, :] += psi[0, 1:-1]
        rhs[-1, :] += psi[-1, 1:-1]
        lx = 4.0 * np.sin(np.arange(1, m_ - 1) * np.pi / (2 * (m_ - 1))) ** 2
        ly = 4.0 * np.sin(np.arange(1, n_ - 1) * np.pi / (2 * (n_ - 1))) ** 2
        uh = scipy.fft.dstn(rhs, type=1, norm="ortho", workers=-1) / (lx[None, :] + ly[:, None])
        out = psi.copy()
        out[1:-1, 1:-1] = scipy.fft.idstn(uh, type=1, norm="ortho", workers=-1)
        return out

    def mixed_vs_fp64(psi_np, h, reps, keep):
        src = b.to_field(psi_np, dev)
        mixed_kw = dict(mg_kw, method="mg_mixed", inner_cycles=1)
        fp32_kw = dict(mg_kw, method="mg_fp32", tol=1e-5)
        out = {}
        fields = {}
        for name, kw in (("fp64", mg_kw), ("mixed", mixed_kw), ("fp32_only_tol_1e-5", fp32_kw)):
            f = b.field(src.shape[1], src.shape[0], dev)
            for _ in range(3):  # warm-up: graphs captured, small-level tail chosen
                timed_solve(f, src, kw, h)
            times, info = [], None
            for _ in range(reps):
                info, ms = timed_solve(f, src, kw, h)
                times.append(ms)
            out[name] = {"ms_median": statistics.median(times), "iters": info["iters"],
                         "status": info["status"], "r_final_over_r0": info["r_final"] / info["r0"]}
            fields[name] = f
        want = exact_solution(psi_np)
        scale = float(np.abs(want).max())
        for name, f in fields.items():
            got = f.cpu().numpy()
            out[name]["max_err_vs_exact_over_max"] = float(np.abs(got - want).max()) / scale
            keep[name] = got  # compared with the oracle's solution in the CPU-baseline leg
        del want
        diff = (fields["mixed"] - fields["fp64"]).abs().max().item()
        out["speedup"] = out["fp64"]["ms_median"] / out["mixed"]["ms_median"]
        out["max_abs_diff_vs_fp64_over_max"] = diff / fields["fp64"].abs().max().item()
        return out

    mixed = {"method": "V(2,2) in FP32 (smoother, residual, restriction, interpolation) inside "
                       "FP64 defect correction; FP64 residual, update and coarsest solve",
             "error": "max |psi - psi_exact| / max |psi_exact|, psi_exact the exact discrete "
                      "solution (DST-I, host FP64)",
             "error_vs_oracle": "max |psi - psi_oracle| / max |psi_oracle|, psi_oracle the oracle's "
                                "FP64 V(2,2) solution to the same 1e-10 (computed in the CPU-"
                                "baseline leg)"}
    kept = {"grid_4097": {}, "grid_8193": {}, "batch_256x1025": {}}
    mixed["grid_4097"] = mixed_vs_fp64(psi_host, H, 5, kept["grid_4097"])
    psi_8193 = wl.sine_edges(8193, 8193, seed=wl.SEED_BASE + 1)
    mixed["grid_8193"] = mixed_vs_fp64(psi_8193, 1.0 / 8192, 3, kept["grid_8193"])

    def mixed_batch(count=256, side=1025, reps=3):
        pristine = [b.to_field(wl.sine_edges(side, side, seed=wl.SEED_BASE + 3 + k), dev)
                    for k in range(count)]
        work_ = [f.clone() for f in pristine]
        batch_ = b.Batch(work_, 1.0 / (side - 1), 1.0 / (side - 1))  # descriptors marshalled once
        out = {"problems": count, "side": side}
        for name, method in (("fp64", "mg"), ("mixed", "mg_mixed")):
            kw = dict(mg_kw, method=method)
            times, res = [], None
            for rep in range(8 + reps):  # warm-ups: plan, graphs, the configuration's choice
                for f, g in zip(work_, pristine):
                    f.copy_(g)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = lap.solve_batched(batch_, stream=stream, **kw)
                e1.record(stream)
                stream.synchronize()
                if rep >= 8:
                    times.append(e0.elapsed_time(e1))
            if not all(r["status"] == "converged" for r in res):
                raise RuntimeError(f"batch {name}: not all problems converged")
            ms = statistics.median(times)
            out[name] = {"ms": ms, "solves_per_s": count / (ms / 1e3),
                         "max_cycles": max(r["iters"] for r in res)}
            kept["batch_256x1025"][name] = [work_[k].cpu().numpy() for k in ORACLE_BATCH_SAMPLE]
        out["speedup"] = out["fp64"]["ms"] / out["mixed"]["ms"]
        return out

    mixed["batch_256x1025"] = mixed_batch()
    batch_inputs = [wl.sine_edges(1025, 1025, seed=wl.SEED_BASE + 3 + k) for k in ORACLE_BATCH_SAMPLE]

    # ---- the paper's chamber problem (25 x 17, Eq. 4), its stopping rule (Eq. 16) ---------
    # Iteration counts the paper prints for it (Results and Discussion), context only: its
    # figures of the geometry are missing, so the boundary is a reading of the text.
    paper_counts = {"jacobi": 1194, "gs_lex": 624, "slorb_w1.25": 55, "adi_b_w1.30": 33, "mg_v22": 6}

    def chamber_section(reps=20):
        psi0 = wl.chamber()
        src = b.to_field(psi0, dev)
        f = b.field(psi0.shape[1], psi0.shape[0], dev)
        cases = [("jacobi", dict(method="jacobi")), ("gs_lex", dict(method="gs_lex")),
                 ("gs_rb", dict(method="gs")), ("sor_lex_w1.75", dict(method="sor_lex", w=1.75)),
                 ("sor_rb_w1.75", dict(method="sor", w=1.75)),
                 ("slorb_w1.25", dict(method="slor", w=1.25, line_form="B")),
                 ("adi_b_w1.30", dict(method="adi", w=1.3, line_form="B")),
                 ("mg_v22", dict(method="mg", nu1=2, nu2=2))]
        out = {"grid": "25x17, dx = dy = 0.25 m, psi = 1 on wall AB, 0 elsewhere",
               "stopping": "max|psi^{k+1} - psi^k| <= 1e-9 tested every iteration (Eq. 16)",
               "orderings": "*_lex: the paper's lexicographic order; gs_rb, sor_rb: red-black; "
                            "slorb, adi: zebra lines (the paper's counts are for successive "
                            "lines, which the oracle reproduces: 49 and 31)",
               "timing": "host wall clock around lap_solve (launches, graph replays and the "
                         "per-iteration host check included), median over 20 solves"}
        for name, kw in cases:
            kw = dict(kw, norm="maxdelta", tol=1e-9, max_iter=100000)
            times, info = [], None
            for r in range(reps + 2):
                with torch.cuda.stream(stream):
                    f.copy_(src)
                stream.synchronize()
                t0 = time.perf_counter()
                info = lap.solve(f, 0.25, 0.25, stream=stream, **kw)
                t1 = time.perf_counter()
                if r >= 2:
                    times.append((t1 - t0) * 1e6)
            us = statistics.median(times)
            out[name] = {"iters": info["iters"], "status": info["status"], "us_per_solve": us,
                         "solves_per_s": 1e6 / us, "paper_iters": paper_counts.get(name)}
        return out

    chamber = chamber_section()

    # ---- batched uneven grids: 4096 problems, sides 2^k+1 (k = 5..9), aspect <= 4 ---------
    def batched_workload(count=4096, sample=128):
        shapes = wl.batch_shapes(count, seed=wl.SEED_BASE + 2)
        pristine = [b.to_field(wl.random_ring(m, n, seed=wl.SEED_BASE + 2 + 10 * k), dev)
                    for k, (m, n) in enumerate(shapes)]
        work = [f.clone() for f in pristine]
        batch = b.Batch(work, 1.0, 1.0)  # descriptors marshalled once, outside the timing
        points = sum((m - 2) * (n - 2) for m, n in shapes)
        out = {"problems": count, "interior_points": points,
               "shapes": "m, n in {33, 65, 129, 257, 513}, aspect <= 4, ring U[0,1], interior 0"}

        def time_batch(method, warm, reps, **extra):
            # warm-ups: the plan, the candidates' graphs and the choice by timing (each call's
            # cycles with every problem running time one candidate configuration)
            times, res = [], None
            for rep in range(warm + reps):
                for f, g in zip(work, pristine):
                    f.copy_(g)
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = lap.solve_batched(batch, stream=stream, **dict(mg_kw, method=method, **extra))
                e1.record(stream)
                stream.synchronize()
                if rep >= warm:
                    times.append(e0.elapsed_time(e1))
            if not all(r["status"] == "converged" for r in res):
                raise RuntimeError(f"batched {method}: not all problems converged")
            return statistics.median(times), res

        for name, method in (("fp64", "mg"), ("mixed", "mg_mixed")):
            ms, res = time_batch(method, 8, 3)
            out[name] = {"ms": ms, "solves_per_s": count / (ms / 1e3),
                         "max_cycles": max(r["iters"] for r in res),
                         "configuration": lap.last_batch_config()}
        # the FP32 tilings one by one (tail and item size still chosen by timing): what the
        # choice between them is worth
        out["mixed_by_tiling"] = {}
        for tiling, label in ((1, "tiles_512x128x64"), (2, "tiles_1024x128x64"),
                              (3, "tiles_512x128x32"), (-1, "one_kernel_per_pass")):
            ms, _ = time_batch("mg_mixed", 6, 3, tiling=tiling)
            out["mixed_by_tiling"][label] = {"ms": ms, "configuration": lap.last_batch_config()}
        # one CTA per work item against persistent launches (resident CTAs looping over the
        # items), the other knobs still chosen by timing
        out["by_launch"] = {}
        for name, method in (("fp64", "mg"), ("mixed", "mg_mixed")):
            for persistent, label in ((-1, "one_cta_per_item"), (1, "persistent")):
                ms, _ = time_batch(method, 6, 3, persistent=persistent)
                out["by_launch"][f"{name}_{label}"] = {"ms": ms,
                                                       "configuration": lap.last_batch_config()}
        # one problem at a time through lap_solve, on a sample
        kw = dict(mg_kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for f, g in zip(work[:sample], pristine[:sample]):
            f.copy_(g)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for f in work[:sample]:
            lap.solve(f, 1.0, 1.0, stream=stream, **kw)
        e1.record(stream)
        stream.synchronize()
        per = e0.elapsed_time(e1) / sample
        out["fp64_one_at_a_time"] = {"ms_per_solve": per, "solves_per_s": 1e3 / per,
                                     "sample": f"first {sample} problems"}
        out["mixed_batched_over_fp64_one_at_a_time"] = out["mixed"]["solves_per_s"] / (1e3 / per)
        out["mixed_batched_over_fp64_batched"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
        return out

    batched = batched_workload()

    # ---- serving: Poisson arrivals, continuous batching under a 40 GB budget ---------------
    def serving_workload(total_requests=args.serving_requests, burst=400):
        rng = np.random.default_rng(wl.SEED_BASE + 4)

        def draw(count):
            out = []
            for _ in range(count):
                m, n = (2 ** int(round(np.log2(v - 1))) + 1
                        for v in np.exp(rng.uniform(np.log(33), np.log(2049), size=2)))
                tol = float(np.exp(rng.uniform(np.log(1e-10), np.log(1e-6))))
                method = "mg_mixed" if rng.uniform() < 0.5 else "sor"
                out.append((m, n, tol, method, int(rng.integers(1 << 30))))
            return out

        def pct(v, q):
            v = sorted(v)
            return 1e3 * v[min(len(v) - 1, int(q * len(v)))] if v else None

        def run(reqs, rate):
            srv = b.Server(lap, hbm_budget=40 << 30, max_running=512, sor_sweeps=50)
            fields = [b.to_field(wl.random_ring(m, n, seed), dev) for m, n, _, _, seed in reqs]
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs))) if rate else np.zeros(len(reqs))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ids, lat, nxt, steps = {}, {"mg_mixed": [], "sor": []}, 0, 0
            work_done = []  # (m, n, method, iterations) per finished request
            finished = 0
            while finished < len(reqs):
                now = time.perf_counter() - t0
                while nxt < len(reqs) and arrivals[nxt] <= now:
                    m, n, tol, method, _ = reqs[nxt]
                    w = wl.w_opt_sor(m, n) if method == "sor" else 1.0
                    rid = srv.submit(fields[nxt], 1.0, 1.0, method=method, w=w, tol=tol, max_iter=10 ** 6)
                    ids[rid] = (arrivals[nxt], method, m, n)
                    nxt += 1
                if not ids:
                    time.sleep(max(0.0, min(arrivals[nxt] - now, 0.01)))
                    continue
                srv.step(stream)
                steps += 1
                done = time.perf_counter() - t0
                # the step's completion list: the requests its convergence tests retired
                for rid, res in srv.drain():
                    if res["status"] != "converged":
                        raise RuntimeError(f"served request did not converge: {res}")
                    arrived, method, m, n = ids.pop(rid)
                    lat[method].append(done - arrived)
                    work_done.append((m, n, method, res["iters"]))
                    finished += 1
            total = time.perf_counter() - t0
            srv.close()
            del fields
            both = lat["mg_mixed"] + lat["sor"]
            return {"requests": len(reqs), "seconds": total, "solves_per_s": len(reqs) / total,
                    "steps": steps, "p50_ms": pct(both, 0.5), "p99_ms": pct(both, 0.99),
                    "by_class": {k: {"requests": len(v), "p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99)}
                                 for k, v in lat.items()},
                    "_work": work_done}

        sat = run(draw(burst), 0.0)
        serving_work.extend(sat["_work"])
        loads = (0.1, 0.3, 0.5, 0.7, 0.9, 1.2)
        # equal arrival windows per load level, sized so that the levels together serve about
        # total_requests requests
        window = total_requests / (sat["solves_per_s"] * sum(loads))
        out = {"workload": "m, n log-uniform in [33, 2049] snapped to 2^k+1; tol log-uniform in "
                           "[1e-10, 1e-6]; 50% mixed-precision V(2,2) / 50% RB-SOR(w_opt, 50 sweeps "
                           "per step); ring U[0,1]; 40 GB budget; host-side latency arrival -> the "
                           "step whose completion list holds the request",
               "saturation": sat, "arrival_window_s": window, "loads": {}}
        for load in loads:
            rate = load * sat["solves_per_s"]
            count = max(20, int(rate * window))
            out["loads"][f"{load:.1f}"] = run(draw(count), rate)
        for v in [out["saturation"], *out["loads"].values()]:
            v.pop("_work", None)
        out["requests_total"] = sat["requests"] + sum(v["requests"] for v in out["loads"].values())
        return out

    serving_work = []  # the saturation run's requests: (m, n, method, iterations)
    serving = serving_workload()

    # ---- end to end through the public API with host buffers -----------------------------
    pinned = torch.from_numpy(psi_host.copy()).pin_memory()
    out_host = torch.empty_like(pinned).pin_memory()
    # one untimed pass: the library's device copy of the field and its graphs are made here
    for kw in (sor_kw, mg_kw):
        out_host.copy_(pinned)
        lap.solve_host(out_host, H, H, stream=stream, **kw)
    torch.cuda.synchronize(dev)
    e2e_steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for kw in (sor_kw, mg_kw):
            out_host.copy_(pinned)
            lap.solve_host(out_host, H, H, stream=stream, **kw)
    e2e_s = replicas.reduce_scalar(time.perf_counter() - t0, "max")
    field_bytes = M * N * 8
    e2e = {"value": replicas.reduce_scalar(2.0 * e2e_steps, "sum") / e2e_s, "unit": "solves/s",
           "h2d_bytes_per_step": 2 * field_bytes, "d2h_bytes_per_step": 2 * field_bytes,
           "api": "lap_solve_host: pinned host field in, the library's copies and solve, "
                  "host field out; host wall clock, the host-side reset of the input included"}

    cpu = None
    if rank == 0:
        # The CPU-baseline leg: the oracle timed on the host cores on a bounded sample (SOR
        # sweeps scaled, the multigrid solve whole), single-threaded and with the SOR sweeps
        # threaded over every host core; its multigrid solutions (4097^2, 8193^2, four
        # problems of the 1025^2 batch) are the reference of the mixed-precision errors.
        import oracle as ora
        ora.build()
        sor_iters = per_step[0]["sor"]["iters"]
        cpu, sol = oracle_sample(psi_host, 30, sor_iters)
        cores = os.cpu_count() or 1
        cpu_mt, _ = oracle_sample(psi_host, 30, sor_iters, threads=cores)
        cpu["all_cores"] = {k: v for k, v in cpu_mt.items() if k != "seconds_per_solve_pair"}

        def rel(a, ref):
            return float(np.abs(a - ref).max() / np.abs(ref).max())

        mixed["grid_4097"]["oracle"] = {name: rel(got, sol) for name, got in kept["grid_4097"].items()}
        t0 = time.perf_counter()
        sol8, info8 = ora.solve(psi_8193, method=ora.MG, ordering=ora.RB, dx=1.0 / 8192, dy=1.0 / 8192,
                                tol=TOL, max_iter=100)
        mixed["grid_8193"]["oracle"] = {name: rel(got, sol8) for name, got in kept["grid_8193"].items()}
        mixed["grid_8193"]["oracle"]["oracle_cycles"] = info8["iters"]
        mixed["grid_8193"]["oracle"]["oracle_seconds"] = time.perf_counter() - t0
        del sol8
        bo = {"fp64": [], "mixed": []}
        for k, x in enumerate(batch_inputs):
            ref, _ = ora.solve(x, method=ora.MG, ordering=ora.RB, dx=1.0 / 1024, dy=1.0 / 1024,
                               tol=TOL, max_iter=100)
            for name in bo:
                bo[name].append(rel(kept["batch_256x1025"][name][k], ref))
        mixed["batch_256x1025"]["oracle"] = {name: max(v) for name, v in bo.items()}
        mixed["batch_256x1025"]["oracle"]["sample"] = f"problems {list(ORACLE_BATCH_SAMPLE)}"
        batched["cpu_baseline"] = oracle_batched_sample()
        serving["cpu_baseline"] = oracle_serving_estimate(serving_work, serving["saturation"]["solves_per_s"])
        for key in ("grid_4097", "grid_8193", "batch_256x1025"):
            o = mixed[key]["oracle"]
            o["mixed_within_1e-10"] = o["mixed"] <= 1e-10

    lap.close()
    replicas.finish()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": size, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "4097x4097", "dx": H, "tol": TOL,
                   "norm": "L2 of the scaled residual, relative to the initial one",
                   "sor_w": w_sor, "sor_check_every": SOR_CHECK,
                   "sor_sum_order": "diagonal pairs (W + S) + (E + N)",
                   "mg": "V(2,2), RB Gauss-Seidel, "
                   "full weighting, bilinear, 11 levels to 5x5, exact coarsest solve",
                   "l2": "inputs larger than L2: field 134 MB + multigrid hierarchy",
                   "parallelism": f"replicas x{size}"},
        "methods": {k: {"iters": per_step[-1][k]["iters"],
                        "ms_median": statistics.median(s[k]["ms"] for s in per_step),
                        "r_final_over_r0": per_step[-1][k]["r_final"] / per_step[-1][k]["r0"]}
                    for k in ("sor", "mg")},
        "roofline": roofline, "kernels": kernels, "latency": latency, "line_relaxation": line_solve,
        "cpu_baseline": {k: v for k, v in cpu.items() if k != "seconds_per_solve_pair"},
        "mixed_precision": mixed, "chamber_25x17": chamber, "batched": batched, "serving": serving, "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
