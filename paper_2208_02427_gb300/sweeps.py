"""Run one hot-path kernel family repeatedly on a seeded grid and print its device time.

    python -m paper_2208_02427_gb300.sweeps --method sor --m 4097 --n 4097 --iters 20

Methods: jacobi, gs, sor (one red-black sweep = 2 launches), sor_diag (one sweep with the
neighbour sums paired along diagonals, inside a one-sweep solve), residual, adi-x, adi-y
(zebra half sweeps), restrict, prolong, mg (one V(2,2) cycle), mg_mixed (one FP32
V(2,2) cycle inside one FP64 defect-correction step), batched / batched_mixed (one cycle
of --count uneven grids, 33..513 per side, through lap_solve_batched), step (one step of
bench.py: RB-SOR at w_opt and V(2,2) multigrid to 1e-10 on the grid). Used for profiling
a single kernel under ncu: small launch counts, the same kernels the solver runs.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as b
from . import workloads as wl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--method", default="sor")
    ap.add_argument("--m", type=int, default=4097)
    ap.add_argument("--n", type=int, default=4097)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--w", type=float, default=None)
    ap.add_argument("--count", type=int, default=4096, help="problems for batched methods")
    ap.add_argument("--tail", type=int, default=0,
                    help="V-cycle small-level tail size (0 = timed choice, -1 = none)")
    ap.add_argument("--unfused", action="store_true",
                    help="FP32 cycle: one kernel per pass instead of the tile kernels")
    ap.add_argument("--tiling", type=int, default=0,
                    help="batched mixed: FP32 tile variant 1..3, -1 = one kernel per pass, 0 = timed")
    ap.add_argument("--item-points", type=int, default=0,
                    help="batched: points per work item (0 = timed)")
    ap.add_argument("--persistent", type=int, default=0,
                    help="batched: 1 = persistent launches, -1 = one CTA per item, 0 = timed")
    ap.add_argument("--no-graphs", action="store_true",
                    help="direct launches (kernels inside conditional graphs cannot be profiled "
                         "one by one)")
    a = ap.parse_args()
    m, n = a.m, a.n
    h = 1.0 / (m - 1)
    psi = wl.sine_edges(m, n)
    lap = b.Laplace()
    if a.no_graphs:
        lap.set_graphs(False)
    u = b.to_field(psi)
    other = b.field(m, n)
    mc, nc = (m - 1) // 2 + 1, (n - 1) // 2 + 1
    qc, ec = b.field(mc, nc), b.field(mc, nc)
    w = a.w if a.w is not None else wl.w_opt_sor(m, n)
    ops = {
        "jacobi": lambda: b.jacobi_sweep(u, other, h, h),
        "gs": lambda: b.smooth(u, w=1.0, nsweeps=1, dx=h, dy=h),
        "sor": lambda: b.smooth(u, w=w, nsweeps=1, dx=h, dy=h),
        "sor_diag": lambda: lap.solve(u, h, h, method="sor", w=w, tol=0.0, max_iter=1,
                                      sum_order="diagonal"),
        "residual": lambda: lap.residual(u, h, h),
        "adi-x": lambda: lap.line_sweep(u, 1.3, "A", 0, h, h),
        "adi-y": lambda: lap.line_sweep(u, 1.3, "A", 1, h, h),
        "restrict": lambda: b.restrict(u, qc, other, ec=ec, dx=h, dy=h),
        "prolong": lambda: b.prolong_add(u, ec, h, h),
        "mg": lambda: lap.solve(u, h, h, method="mg", tol=0.0, max_iter=1, tail_size=a.tail),
        "mg_mixed": lambda: lap.solve(u, h, h, method="mg_mixed", tol=0.0, max_iter=1,
                                      tail_size=a.tail, unfused=a.unfused),
    }
    if a.method == "step":
        # one step of the benchmark: RB-SOR at w_opt (tested every 100 sweeps, neighbour sums
        # paired along diagonals) and the V(2,2) multigrid, each to ||r|| <= 1e-10 ||r0|| from the
        # same initial field
        init = u.clone()

        def step():
            u.copy_(init)
            lap.solve(u, h, h, method="sor", w=w, tol=1e-10, check_every=100, max_iter=200000,
                      sum_order="diagonal")
            u.copy_(init)
            lap.solve(u, h, h, method="mg", tol=1e-10, nu1=2, nu2=2, coarsest_min=5, max_iter=100)

        ops["step"] = step
    if a.method.startswith("batched"):
        shapes = wl.batch_shapes(a.count, seed=wl.SEED_BASE + 2)
        fields = [b.to_field(wl.random_ring(bm, bn, seed=wl.SEED_BASE + 2 + 10 * k))
                  for k, (bm, bn) in enumerate(shapes)]
        meth = "mg_mixed" if a.method == "batched_mixed" else "mg"
        ops[a.method] = lambda: lap.solve_batched(fields, 1.0, 1.0, method=meth, tol=0.0,
                                                  max_iter=1, tail_size=a.tail,
                                                  unfused=a.unfused, tiling=a.tiling,
                                                  item_points=a.item_points,
                                                  persistent=a.persistent)
    fn = ops[a.method]
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.iters):
        fn()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"method": a.method, "m": m, "n": n, "iters": a.iters,
                      "ms_per_iter": e0.elapsed_time(e1) / a.iters}))
    lap.close()


if __name__ == "__main__":
    main()
