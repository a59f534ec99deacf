"""Throughput of one DG operator apply (GDoF/s), the operator half of the
benchmark metric, for a workload's mesh on one GPU.

python -m paper_2107_07776_gb300.applybench [--workload tgv32] [--cells N ...]
        [--op momentum|poisson] [--precision fp64|fp64_native|fp32]
        [--launches K] [--warmup W] [--profile]

The operator is dg_apply_momentum (mass 1/(gamma dt), viscosity 1/(2 Re),
advection 1/2, advecting field = the workload's initial velocity) or
dg_apply_poisson (alpha = 1/(c gamma dt)^2) on a seeded N(0,1) source, in the
launch configuration the solver uses (after dg_autotune).  "fp64" is the
float-float FP64 arithmetic, "fp64_native" the FP64 pipe, "fp32" the
multigrid levels' single-precision apply.  Each timed launch is bracketed by
CUDA events on the launching stream with a 512 MiB buffer written before it
(L2 is 135 MB).  --profile brackets the timed launches with
cudaProfilerStart/Stop so `ncu --profile-from-start off` captures exactly
those.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import statistics

import workloads as W

from . import binding as b


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tgv32", choices=sorted(W.WORKLOADS))
    ap.add_argument("--op", default="momentum", choices=["momentum", "poisson"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp64_native", "fp32"])
    ap.add_argument("--cells", type=int, nargs="+", default=None,
                    help="cells per axis (the workload's mesh scaled; default: its own)")
    ap.add_argument("--launches", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="run this kernel variant (0-7) for every operator instead of the tuned choice")
    ap.add_argument("--profile", action="store_true")
    args = ap.parse_args(argv)

    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    if args.cells:
        cells = args.cells * w.dim if len(args.cells) == 1 else args.cells
        w = w.scaled(tuple(cells))
    mesh = b.Mesh.from_workload(w)
    if not args.no_autotune:
        b.dg_autotune(mesh.handle)
    if args.variant is not None:
        b.dg_mesh_set_variant(mesh.handle, args.variant)
    b.dg_mesh_set_fp64_arith(mesh.handle, 1 if args.precision == "fp64_native" else 0)
    dt = torch.float32 if args.precision == "fp32" else torch.float64
    g = b.GAMMA
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    if args.op == "momentum":
        X = mesh.node_coords(0).cpu().numpy()
        Xp = mesh.node_coords(1).cpu().numpy()
        u0h, _ = W.initial_state(w, X, Xp)
        ubar = torch.tensor(u0h.reshape(-1), device=dev).to(dt)
        n = mesh.n_dofs_u
        co = b.momentum_coeffs(1.0 / (g * w.dt), 1.0 / (2 * w.Re), 0.5)
        f = b.dg_apply_momentum_f32 if dt == torch.float32 else b.dg_apply_momentum
        x = torch.tensor(W.random_vector(n, 1), device=dev).to(dt)
        y = torch.empty_like(x)
        call = lambda: f(mesh.handle, co, ubar, x, y, sp)  # noqa: E731
    else:
        n = mesh.n_dofs_p
        alpha = 1.0 / (w.c ** 2 * (g * w.dt) ** 2)
        f = b.dg_apply_poisson_f32 if dt == torch.float32 else b.dg_apply_poisson
        x = torch.tensor(W.random_vector(n, 2), device=dev).to(dt)
        y = torch.empty_like(x)
        call = lambda: f(mesh.handle, alpha, x, y, sp)  # noqa: E731
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        call()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.launches)]
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.start()
    for i, (a, c) in enumerate(evs):
        flush.fill_(i & 0xFF)
        a.record(stream)
        call()
        c.record(stream)
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.stop()
    ms = [a.elapsed_time(c) for a, c in evs]
    med = statistics.median(ms)
    print(json.dumps({"workload": w.name, "op": args.op, "precision": args.precision,
                      "dofs": n, "launches": args.launches, "ms_median": med,
                      "ms_mean": statistics.mean(ms), "gdofs": n / (med * 1e-3) / 1e9}))
    mesh.close()


if __name__ == "__main__":
    main()
