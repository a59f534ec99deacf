"""Benchmark of the DG TR-BDF2 hot path on one GB300 (replicas on N GPUs).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload tgv32] [--mode apply|step]

mode "apply" (the matrix-free operator pass): one step = one FP64 momentum
apply (all velocity components, advecting field = the workload's initial
velocity) + one FP64 pressure Helmholtz apply, on inputs resident in HBM;
value = (velocity + pressure DoFs) / time per step in GDoF/s.

Timing: W untimed warm-up steps; K timed steps, each bracketed by CUDA events
on the launching stream, with a 512 MiB buffer written between steps (L2 is
135 MB) so every step starts cold; barrier + synchronize on both sides; max
over ranks.  e2e: the same step through the C ABI from pinned host buffers,
host<->device copies inside the timed region.  roofline: the dominant
kernel's algorithmic flops per launch / its CUDA-event duration against the
FP64 FMA peak.  cpu_baseline / --impl reference: the oracle (assembled
block operators, OpenMP) on the host cores over a bounded sample of cells.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "GDoF/s DG operator apply; s per TR-BDF2 step (mixed+learned vs FP64)"
FP64_PEAK_TFLOPS = 1.253   # measured FP64 FMA throughput of GB300
FP32_PEAK_TFLOPS = 76.5    # measured FP32 FMA throughput


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "fallback": True}


# ---------------------------------------------------------------- flop model
def apply_flops_per_cell(dim: int, N: int, adv: bool) -> float:
    """Algorithmic FP64 flops of one scalar operator application per cell
    (sum factorisation on the collocated basis, every face evaluated once):
    gradient and transposed gradient sweeps 2 d N^(d+1) FMA, mass N^d FMA,
    d faces per cell with N^(d-1) points each needing traces and normal
    derivatives of both sides (4N FMA), the flux (10) and the test-side
    distribution to both cells (4N FMA); advection adds the advective flux
    (2 per node and direction) and the normal advecting-field traces with
    the LF speed (2N + 5 per face point).  FMA = 2 flops."""
    NB, NF = N ** dim, N ** (dim - 1)
    fma = 2 * dim * N ** (dim + 1) + NB + dim * NF * (8 * N + 10)
    if adv:
        fma += 2 * dim * NB + dim * NF * (2 * N + 5)
    return 2.0 * fma


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap,power.draw"

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch

    from paper_2107_07776_gb300 import binding as b

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    mesh = b.Mesh.from_workload(w)
    d, nu_s = w.dim, mesh.n_dofs_u // w.dim
    X = mesh.node_coords(0).cpu().numpy()
    if w.name.startswith("tgv"):
        ub_h = W.tgv3d_u(*X)
    elif w.name == "channel":
        ub_h = W.channel_u0(*X)
    else:
        ub_h = np.zeros((d, nu_s))
    ub = torch.tensor(ub_h.reshape(-1), dtype=torch.float64, device=dev)
    src_u = torch.tensor(W.random_vector(mesh.n_dofs_u, 1), device=dev)
    src_p = torch.tensor(W.random_vector(mesh.n_dofs_p, 2), device=dev)
    dst_u = torch.empty_like(src_u)
    dst_p = torch.empty_like(src_p)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    g = b.GAMMA
    co = b.momentum_coeffs(1.0 / (g * w.dt), 1.0 / (2 * w.Re), 0.5)
    alpha = 1.0 / (w.c ** 2 * (g * w.dt) ** 2)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step():
        b.dg_apply_momentum(mesh.handle, co, ub, src_u, dst_u, sp)
        b.dg_apply_poisson(mesh.handle, alpha, src_p, dst_p, sp)

    launches_per_step = 2
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            e0, e1, e2 = ev[i]
            e0.record(stream)
            b.dg_apply_momentum(mesh.handle, co, ub, src_u, dst_u, sp)
            e1.record(stream)
            b.dg_apply_poisson(mesh.handle, alpha, src_p, dst_p, sp)
            e2.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [e0.elapsed_time(e2) for e0, _, e2 in ev]
    mom_ms = [e0.elapsed_time(e1) for e0, e1, _ in ev]
    pois_ms = [e1.elapsed_time(e2) for _, e1, e2 in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    dofs = mesh.n_dofs_u + mesh.n_dofs_p
    value = dofs * world / (ms_per_step * 1e-3) / 1e9

    # ---- end to end through the C ABI with pinned host buffers ----
    hu = torch.empty(mesh.n_dofs_u, dtype=torch.float64, pin_memory=True)
    hp = torch.empty(mesh.n_dofs_p, dtype=torch.float64, pin_memory=True)
    hu.copy_(src_u.cpu())
    hp.copy_(src_p.cpu())
    ou = torch.empty_like(hu, pin_memory=True)
    op = torch.empty_like(hp, pin_memory=True)
    torch.cuda.synchronize()
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    for i in range(args.steps):
        src_u.copy_(hu, non_blocking=True)
        src_p.copy_(hp, non_blocking=True)
        step()
        ou.copy_(dst_u, non_blocking=True)
        op.copy_(dst_p, non_blocking=True)
    e_b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e_a.elapsed_time(e_b) / args.steps
    e2e = {"value": dofs * world / (e2e_ms * 1e-3) / 1e9, "unit": "GDoF/s",
           "h2d_bytes_per_step": 8 * dofs, "d2h_bytes_per_step": 8 * dofs}

    # ---- roofline of the dominant kernel (FP64 momentum apply) ----
    mom_avg = statistics.mean(mom_ms)
    n_cells = mesh.n_cells
    fl = d * n_cells * apply_flops_per_cell(d, w.degree + 1, True)
    achieved = fl / (mom_avg * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "scalar_op_kernel (momentum, FP64)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": args.traffic,
            "peak_source": "measured FP64 FMA probe on GB300 (DESIGN.md)",
            "momentum_gdofs": mesh.n_dofs_u / (mom_avg * 1e-3) / 1e9,
            "poisson_gdofs": mesh.n_dofs_p / (statistics.mean(pois_ms) * 1e-3) / 1e9}
    return dict(value=value, ms_per_step=ms_per_step, clocks=clk.summary(), e2e=e2e,
                roofline=roof, gpu_launches=launches_per_step * args.steps,
                workload=w, mesh_cells=n_cells, dofs=dofs)


# ---------------------------------------------------------------- oracle arm
def oracle_apply_rate(w, budget_s: float = 15.0, max_cells: int = 2048):
    """Oracle (assembled block operators, OpenMP over the host cores) applied
    to a sample of the workload's cells: GDoF/s of the same apply pass."""
    from oracle.dg import Mesh as OMesh, lib as olib
    om = OMesh(w.dim, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree,
               map=w.map, map_param=list(w.map_param))
    rng = np.random.default_rng(0)
    ncell = min(max_cells, om.n_cells)
    cells = np.sort(rng.choice(om.n_cells, ncell, replace=False))
    ub = W.random_vector(w.dim * om.n_u, 3)
    x = W.random_vector(om.n_u, 4)
    xp = W.random_vector(om.n_p, 5)
    M, A, C = (om.assemble("mass_u", cells=cells), om.assemble("sipg_u", cells=cells),
               om.assemble("adv_u", ub, cells=cells))
    Mp, K = om.assemble("mass_p", cells=cells), om.assemble("sipg_p", cells=cells)
    t0 = time.perf_counter()
    reps = 0
    while True:
        for _ in range(w.dim):
            M.apply(x); A.apply(x); C.apply(x)
        Mp.apply(xp); K.apply(xp)
        reps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / reps
    dofs = ncell * (w.dim * om.nb_u + om.nb_p)
    return {"value": dofs / dt / 1e9, "unit": "GDoF/s", "cores": int(olib().ora_num_threads()),
            "kind": "oracle",
            "sample": f"{ncell} of {om.n_cells} cells' rows of the assembled momentum "
                      f"(mass+SIP+LF, {w.dim} components) and pressure Helmholtz operators, "
                      f"block-sparse apply, {reps} repetitions in {budget_s:.0f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv32", choices=sorted(W.WORKLOADS))
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the dominant kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w = W.WORKLOADS[args.workload]
    cfg = {"workload": f"{w.name}: {w.dim}D {'x'.join(map(str, w.n))} cells, DG Q{w.degree}/"
                       f"Q{w.degree - 1}, Re {w.Re:g}, c {w.c:g}, dt {w.dt:g}",
           "step": "FP64 momentum apply (3 components, LF advection with the initial "
                   "velocity) + FP64 pressure Helmholtz apply",
           "l2": "512 MiB buffer written between timed steps",
           "parallelism": f"replicas x{args.gpus}"}
    if args.impl == "reference":
        if rank != 0:
            return
        cb = oracle_apply_rate(w, budget_s=max(2.0, 20.0 / max(1, args.steps)))
        ms = (w.n_dofs_u + w.n_dofs_p) / (cb["value"] * 1e9) * 1e3
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GDoF/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "GDoF/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if rank != 0:
        return
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_apply_rate(w)
    line = {"metric": METRIC, "value": r["value"], "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "clocks": r["clocks"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "roofline": r["roofline"], "cpu_baseline": cb}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
