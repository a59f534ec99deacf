"""Benchmark of the DG TR-BDF2 hot path on one GB300 (replicas on N GPUs).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload channel] [--secondary tgv32] [--solver mixed+learned]

One step = one TR-BDF2 step (Section 2: two momentum predictors solved by
Jacobi-GMRES, two pressure Helmholtz solves by flexible CG with h/p
multigrid, RHS assembly, projections and updates) on the workload's state,
all inside the CUDA library, inputs resident in HBM.  value = (velocity +
pressure DoFs) advanced per second (GDoF/s); ms_per_step = time per step.

The headline workload is the wall-bounded channel: 256x64x64 tanh-graded
hexahedra, Q2/Q1 (85 M velocity + 8.4 M pressure DoFs), Re 5000, dt 5e-4.
Solvers: "mixed+learned" (default; FP32 multigrid inside the FP64 outer
Krylov solves plus the learned initial guess, trained during an untimed
phase of --train-steps steps, inference only while timed), "mixed" (the
same with the linearly extrapolated guess) and "plain" (FP64 multigrid,
extrapolated guess).  Every solver takes the same train + warm-up + K
steps from the same initial state, so all time the same window of the flow
and end at the same time level: "error_vs_fp64" is the relative L2
difference of u and p between each solver and "plain" there (all solve to a
relative residual of 1e-8).  A smaller secondary workload (3D periodic
Taylor-Green vortex, 32^3 Q2/Q1) is reported the same way under
"secondary".

Timing: W untimed warm-up steps; K timed steps, each bracketed by CUDA
events on the launching stream, a 512 MiB buffer written between steps (L2
is 129 MB; the channel's vectors are 0.7 GB each anyway); barrier +
synchronize on both sides; max over ranks (replicas: no collective inside
a step).  e2e: the same step through the C ABI from pinned host buffers,
host<->device copies of u and p inside the timed region.  apply: GDoF/s of
each operator apply alone (CUDA events, same launch configuration as in the
step).  roofline: the momentum apply (the dominant kernel pair of the
step) -- algorithmic FP64 flops per launch / its CUDA-event duration,
against the float-float ceiling that bounds it (the FP32-pipe instruction
rate divided by the 15 instructions of one float-float multiply-add), with
its FP64-pipe and HBM fractions beside it.  cpu_baseline and --impl
reference: the oracle (assembled operators, sparse direct solves) on the
host cores -- full TR-BDF2 steps on a small mesh of the same workload,
named in its config, and the assembled momentum apply at the full 32^3
Taylor-Green size.
"""
from __future__ import annotations

import argparse
import hashlib
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
DTYPE = ("f64 storage and Krylov; df64 (float-float, 48-bit significand) operator "
         "arithmetic; fp32 multigrid preconditioner; bf16/fp32 learned guess")
# FP64 FMA peak of GB300: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz = 1.259
# TFLOP/s from the unit counts; an FMA-chain probe measured 1.253
FP64_PEAK_TFLOPS = 1.253
FP32_PEAK_TFLOPS = 76.5    # measured FP32 FMA throughput
# FP64-equivalent ceiling of float-float arithmetic: one fused multiply-add
# (df_fma) costs 15 FP32-pipe instructions; 152 SMs x 128 lanes x 2.07 GHz
# / 15 x 2 flop
FLOAT_FLOAT_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 15 * 2 / 1e12

# Untimed steps before the warm-up (the learned guess trains on them).
TRAIN_STEPS = {"tg2d": 50, "tgv32": 200, "tgv48": 200, "channel": 40, "mms64": 20}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one momentum
# apply (all its launches) from an ncu capture of the benchmark's launch
# configuration, with the SHA-256 (first 16 hex digits) of the kernel
# sources it was taken on: the figure is reported only while those sources
# are unchanged (kernel_sources_sha()), and null otherwise.
NCU_TRAFFIC = {
    # one dg_apply_momentum call on the channel (both split passes, the face and
    # the components-interleaved cell kernel): 6.8453 GB read + 3.2710 GB written
    "channel": {6: {"bytes": 10116279808, "sha": "31c3d70f105d3815"}},
}
KERNEL_SOURCES = ("dg_apply.cu", "dg_apply_kernel.cuh", "dg_split_kernel.cuh",
                  "dg_common.cuh", "dg_df64.cuh", "dg_faces.cuh")


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2107_07776_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def apply_flops_per_cell(dim: int, N: int, adv: bool) -> float:
    """Algorithmic flops of one scalar operator application per cell (sum
    factorisation on the collocated basis, every face once): gradient and
    transposed gradient sweeps 2 d N^(d+1) FMA, mass N^d, d faces per cell
    with N^(d-1) points needing traces and normal derivatives of both sides
    (4N), the flux (10) and the distribution to both cells (4N); advection
    adds 2 per node and direction plus the advecting-field traces and LF
    speed (2N + 5 per face point).  FMA = 2 flops."""
    NB, NF = N ** dim, N ** (dim - 1)
    fma = 2 * dim * N ** (dim + 1) + NB + dim * NF * (8 * N + 10)
    if adv:
        fma += 2 * dim * NB + dim * NF * (2 * N + 5)
    return 2.0 * fma


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,power.draw")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

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
        for l in self.lines:
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


def job_rate(total_ms_local: float, steps: int, dofs_per_rank: int, world: int, device=None):
    """Whole-job throughput of weakly scaled replicas: every rank advances
    dofs_per_rank DoFs per step, and the job's time is the slowest rank's
    (max over ranks, one all-reduce after the timed region).  Returns
    (ms per step, GDoF/s of all ranks together)."""
    total = float(total_ms_local)
    if world > 1:
        import torch
        t = torch.tensor([total], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total = float(t.item())
    ms = total / steps
    return ms, dofs_per_rank * world / (ms * 1e-3) / 1e9


def step_params(b, w, precond, guess, tol=1e-8, f=None, mg_degree=0):
    prm = b.dg_step_params()
    prm.dt, prm.gamma, prm.extrapolate = w.dt, 0.0, 1
    if f is not None:  # time-independent forcing at every stage time
        prm.f_n = prm.f_ng = prm.f_n1 = f.data_ptr()
    prm.mom = b.solve_opts(b.DG_SYS_MOMENTUM, tol=tol, max_iter=500, restart=30,
                           precond=b.DG_PC_JACOBI, guess=guess)
    prm.helm = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=tol, max_iter=500, precond=precond,
                            guess=guess, mg_degree=mg_degree)
    return prm


SOLVERS = {
    # name: (Helmholtz preconditioner, initial guess, learned, smoother degree)
    # (each with the Chebyshev degree that was fastest for it on the 32^3
    # Taylor-Green vortex: the learned guess pays more when iterations are
    # dearer; the trilinear workload states degree 4 and runs it for all)
    "mixed+learned": ("DG_PC_MG_FP32", "DG_GUESS_LEARNED", True, 8),
    "mixed": ("DG_PC_MG_FP32", "DG_GUESS_EXTRAP", False, 5),
    "plain": ("DG_PC_MG_FP64", "DG_GUESS_EXTRAP", False, 5),
}
FIXED_MG_DEGREE = {"mms64": 4}


def smoother_degree(w, name, args):
    if w.name in FIXED_MG_DEGREE:
        return FIXED_MG_DEGREE[w.name]
    if name == args.solver and args.mg_degree:
        return args.mg_degree
    return SOLVERS[name][3]


def rel_l2(a, b) -> float:
    return float((a - b).norm().item() / max(b.norm().item(), 1e-300))


def run_solvers(args, b, w, mesh, dev, world, nsteps, keep_main):
    """Every solver of SOLVERS (the main one first, with the clock sampler)
    from the workload's initial state: train + warm-up + nsteps steps, the
    last nsteps timed one by one.  Returns per-solver timings and the final
    states (the main solver's handle too when keep_main)."""
    import torch

    X = mesh.node_coords(0).cpu().numpy()
    Xp = mesh.node_coords(1).cpu().numpy()
    u0h, p0h = W.initial_state(w, X, Xp)
    fh = W.forcing(w, X)
    fdev = None if fh is None else torch.tensor(fh.reshape(-1), dtype=torch.float64, device=dev)
    u0 = torch.tensor(u0h.reshape(-1), dtype=torch.float64, device=dev)
    p0 = torch.tensor(p0h, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    train = args.train_steps if args.train_steps is not None else TRAIN_STEPS.get(w.name, 40)
    order = [args.solver] + [n for n in SOLVERS if n != args.solver]
    out = {}
    for name in order:
        main = name == args.solver
        pc, guess, learned, _ = SOLVERS[name]
        deg = smoother_degree(w, name, args)
        s = b.dg_solver_create(mesh.handle, w.Re, w.c)
        u, p = u0.clone(), p0.clone()
        prm = step_params(b, w, getattr(b, pc), getattr(b, guess), f=fdev, mg_degree=deg)
        if learned:  # untimed training phase, then inference only
            b.dg_guess_configure(s, enable=1, train=1, systems=1, lr=1e-3, seed=1)
        for _ in range(train):
            b.trbdf2_step(s, prm, u, p)
        if learned:
            b.dg_guess_configure(s, enable=1, train=0, systems=1, lr=1e-3, seed=1)
        for _ in range(args.warmup):
            b.trbdf2_step(s, prm, u, p)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(dev.index)
        if main:
            clk.__enter__()
        launches0 = b.dg_kernel_launches()
        iters = []
        for i in range(nsteps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            info = b.trbdf2_step(s, prm, u, p)
            ev[i][1].record(stream)
            iters.append([x.iterations for x in info])
        launches = b.dg_kernel_launches() - launches0
        torch.cuda.synchronize()
        if main:
            clk.__exit__(None, None, None)
        if world > 1:
            torch.distributed.barrier()
        r = {"ms": [a.elapsed_time(c) for a, c in ev], "iters": iters, "launches": launches,
             "mg_degree": deg, "u": u.clone(), "p": p.clone(), "clocks": clk.summary()}
        if main and keep_main:
            r["handle"] = (s, prm, u, p)
        else:
            b.dg_solver_destroy(s)
        out[name] = r
    plain = out["plain"]
    for name, r in out.items():
        r["error_vs_fp64"] = {"u": rel_l2(r["u"], plain["u"]), "p": rel_l2(r["p"], plain["p"])}
    return out, (u0, p0, stream, flush)


def summarise(w, res, steps, train):
    return {name: {"ms_per_step": statistics.mean(r["ms"]), "mg_degree": r["mg_degree"],
                   "iterations_per_step": np.array(r["iters"]).mean(axis=0).round(2).tolist(),
                   "error_vs_fp64": r["error_vs_fp64"]}
            for name, r in res.items()} | {
        "window": f"{train} untimed training steps + warm-up, then {steps} timed steps from "
                  f"t = 0 (dt {w.dt:g}); errors at that final time"}


def workload_label(w) -> str:
    return (f"{w.name}: {w.dim}D {'x'.join(map(str, w.n))} cells, DG Q{w.degree}/Q{w.degree - 1}, "
            f"{w.n_dofs_u + w.n_dofs_p} DoFs, Re {w.Re:g}, c {w.c:g}, dt {w.dt:g}")


def run_ours(args, rank, world):
    import torch

    from paper_2107_07776_gb300 import binding as b

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    mesh = b.Mesh.from_workload(w)
    autotune = None
    if not args.no_autotune:
        b.dg_autotune(mesh.handle)
        autotune = json.loads(b.dg_autotune_report(mesh.handle))
    train = args.train_steps if args.train_steps is not None else TRAIN_STEPS.get(w.name, 40)
    res, (u0, p0, stream, flush) = run_solvers(args, b, w, mesh, dev, world, args.steps, True)
    main = res[args.solver]
    dofs = mesh.n_dofs_u + mesh.n_dofs_p
    ms_per_step, value = job_rate(sum(main["ms"]), args.steps, dofs, world, dev)
    solvers = summarise(w, res, args.steps, train)

    # ---- end to end through the C ABI with pinned host buffers ----
    s, prm, u_main, p_main = main["handle"]
    # the host copies continue the main run's state (its solver history and
    # learned guess belong to that trajectory)
    hu = u_main.cpu().pin_memory()
    hp = p_main.cpu().pin_memory()
    u, p = torch.empty_like(u0), torch.empty_like(p0)

    def e2e_step():
        u.copy_(hu, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        b.trbdf2_step(s, prm, u, p)
        hu.copy_(u, non_blocking=True)
        hp.copy_(p, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e_b.record(stream)
    torch.cuda.synchronize()
    b.dg_solver_destroy(s)
    for r in res.values():
        r.pop("u"), r.pop("p"), r.pop("handle", None)
    e2e_ms = e_a.elapsed_time(e_b) / args.steps
    # the transfers alone (the same copies, no step), for the split of e2e
    e_a.record(stream)
    for _ in range(3):
        u.copy_(hu, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        hu.copy_(u, non_blocking=True)
        hp.copy_(p, non_blocking=True)
    e_b.record(stream)
    torch.cuda.synchronize()
    copy_ms = e_a.elapsed_time(e_b) / 3
    nbytes = 8 * dofs
    e2e = {"value": dofs * world / (e2e_ms * 1e-3) / 1e9, "unit": "GDoF/s",
           "ms_per_step": e2e_ms, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "copies_alone_ms_per_step": copy_ms}
    apply, apply_ms = time_applies(args, b, w, mesh, dev, stream, flush, u0)
    roof = roofline(w, mesh, autotune, apply_ms)
    secondary = None
    if args.secondary and args.secondary != args.workload:
        w2 = W.WORKLOADS[args.secondary]
        mesh2 = b.Mesh.from_workload(w2)
        if not args.no_autotune:
            b.dg_autotune(mesh2.handle)
        res2, _ = run_solvers(args, b, w2, mesh2, dev, world, args.steps, False)
        ms2 = statistics.mean(res2[args.solver]["ms"])
        train2 = args.train_steps if args.train_steps is not None else TRAIN_STEPS.get(w2.name, 40)
        secondary = {"workload": workload_label(w2), "ms_per_step": ms2,
                     "value": (mesh2.n_dofs_u + mesh2.n_dofs_p) / (ms2 * 1e-3) / 1e9,
                     "unit": "GDoF/s", "solvers": summarise(w2, res2, args.steps, train2)}
        mesh2.close()
    study = None if args.no_guess_study else guess_study(b)
    return dict(value=value, ms_per_step=ms_per_step, clocks=main["clocks"], e2e=e2e,
                roofline=roof, gpu_launches=main["launches"], solvers=solvers, apply=apply,
                dofs=dofs, autotune=autotune, secondary=secondary, guess_study=study,
                iterations=np.array(main["iters"]).mean(axis=0).round(2).tolist())


def guess_study(b):
    """The learned initial guess over a long run (48^3 Q2/Q1 Taylor-Green
    vortex, 400 steps: the nets train during the first 200 and only infer
    during the last 200) against the extrapolated guess on the same steps,
    FP32 multigrid Helmholtz: Krylov iterations per solve and ms per step
    over the evaluated steps, for the pressure net alone and for both nets."""
    from paper_2107_07776_gb300 import guessstudy as gs
    w = W.TGV48
    base, ub, pb = gs.run(w, 400, 200, False, 1, b.DG_PC_MG_FP32, 1e-8)
    out = {"workload": workload_label(w), "steps": 400, "train_steps": 200,
           "extrapolated": {k: base[k] for k in ("iterations_per_solve", "ms_per_step")}}
    for systems, name in ((1, "learned_pressure"), (3, "learned_both")):
        lrn, ul, pl = gs.run(w, 400, 200, True, systems, b.DG_PC_MG_FP32, 1e-8)
        out[name] = {k: lrn[k] for k in ("iterations_per_solve", "ms_per_step")}
        out[name]["step_time_vs_extrapolated"] = lrn["ms_per_step"] / base["ms_per_step"]
        out[name]["final_u_rel_diff"] = float(np.linalg.norm(ul - ub) / np.linalg.norm(ub))
    return out


def time_applies(args, b, w, mesh, dev, stream, flush, u0):
    """GDoF/s of each operator apply alone, in the launch configuration the
    solver uses (CUDA events on the launching stream, L2 flushed before each
    launch); FP64 float-float, FP64 native and FP32."""
    import torch

    g = b.GAMMA
    co = b.momentum_coeffs(1.0 / (g * w.dt), 1.0 / (2 * w.Re), 0.5)
    alpha = 1.0 / (w.c ** 2 * (g * w.dt) ** 2)
    xu = torch.tensor(W.random_vector(mesh.n_dofs_u, 1), device=dev)
    xp = torch.tensor(W.random_vector(mesh.n_dofs_p, 2), device=dev)
    yu, yp = torch.empty_like(xu), torch.empty_like(xp)
    xu32, xp32, u032 = xu.float(), xp.float(), u0.float()
    yu32, yp32 = torch.empty_like(xu32), torch.empty_like(xp32)
    sp = stream.cuda_stream
    calls = {
        "momentum_fp64": (lambda: b.dg_apply_momentum(mesh.handle, co, u0, xu, yu, sp), mesh.n_dofs_u),
        "poisson_fp64": (lambda: b.dg_apply_poisson(mesh.handle, alpha, xp, yp, sp), mesh.n_dofs_p),
        "momentum_fp32": (lambda: b.dg_apply_momentum_f32(mesh.handle, co, u032, xu32, yu32, sp),
                          mesh.n_dofs_u),
        "poisson_fp32": (lambda: b.dg_apply_poisson_f32(mesh.handle, alpha, xp32, yp32, sp),
                         mesh.n_dofs_p),
    }
    calls["momentum_fp64_native"] = calls["momentum_fp64"]
    calls["poisson_fp64_native"] = calls["poisson_fp64"]
    apply_ms = {}
    for name, (fn, n) in calls.items():
        b.dg_mesh_set_fp64_arith(mesh.handle, 1 if name.endswith("native") else 0)
        for _ in range(3):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for a, c in evs:
            flush.fill_(1)
            a.record(stream)
            fn()
            c.record(stream)
        torch.cuda.synchronize()
        apply_ms[name] = statistics.mean(a.elapsed_time(c) for a, c in evs)
    b.dg_mesh_set_fp64_arith(mesh.handle, 0)
    apply = {k + "_gdofs": round(calls[k][1] / (v * 1e-3) / 1e9, 4) for k, v in apply_ms.items()}
    pk, _ = peaks()
    apply["hbm_frac"] = {
        "momentum_fp32": (12 * mesh.n_dofs_u / (apply_ms["momentum_fp32"] * 1e-3) / 1e9) / pk["hbm_gbs"],
        "poisson_fp32": (8 * mesh.n_dofs_p / (apply_ms["poisson_fp32"] * 1e-3) / 1e9) / pk["hbm_gbs"],
        "momentum_fp64": (24 * mesh.n_dofs_u / (apply_ms["momentum_fp64"] * 1e-3) / 1e9) / pk["hbm_gbs"],
        "poisson_fp64": (16 * mesh.n_dofs_p / (apply_ms["poisson_fp64"] * 1e-3) / 1e9) / pk["hbm_gbs"]}
    return apply, apply_ms


def roofline(w, mesh, autotune, apply_ms):
    """The momentum apply with advection in float-float arithmetic: the
    step's dominant kernel pair, bound by FP32-pipe issue."""
    pk, src = peaks()
    fl = w.dim * mesh.n_cells * apply_flops_per_cell(w.dim, w.degree + 1, True)
    t = apply_ms["momentum_fp64"] * 1e-3
    achieved = fl / t / 1e12
    variant, face_once = None, False
    for r in autotune or []:
        if r.get("op") == "momentum+advection" and r.get("precision") == "f64":
            variant = r["chosen_variant"]
            face_once = bool(r.get("face_once", [0] * 8)[variant])
    if w.map == 2:
        kname = ("general_op_kernel<double,df64> (momentum apply on trilinear cells; flop model of "
                 "the affine operator, a lower bound of the work)")
    elif face_once:
        cell = "cell_split_nc_kernel" if variant == 6 else "cell_split_kernel"
        kname = (f"face_flux_kernel + {cell}<double,df64> (momentum apply, face-once form, "
                 "float-float FP64 arithmetic)")
    else:
        kname = "scalar_op_kernel<double,df64> (momentum apply, float-float FP64 arithmetic)"
    sha = kernel_sources_sha()
    rec = NCU_TRAFFIC.get(w.name, {}).get(variant) if variant is not None else None
    traffic = rec["bytes"] if rec and rec.get("sha") == sha else None
    alg_bytes = 24 * mesh.n_dofs_u
    return {"bound": "alu", "kernel": kname, "variant": variant,
            "achieved": achieved, "peak": FLOAT_FLOAT_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FLOAT_FLOAT_PEAK_TFLOPS,
            "peak_source": "float-float ceiling from the unit counts and clock: 152 SMs x 128 FP32 "
                           "lanes x 2.07 GHz / 15 FP32 instructions per df64 multiply-add x 2 flop "
                           "= 5.37 TFLOP/s (FP64-equivalent)",
            "flop_per_launch": fl, "launch_ms": apply_ms["momentum_fp64"],
            "fp64_pipe_frac": achieved / FP64_PEAK_TFLOPS,
            "hbm_achieved_gbs": alg_bytes / t / 1e9, "hbm_peak_gbs": pk["hbm_gbs"],
            "hbm_frac": alg_bytes / t / 1e9 / pk["hbm_gbs"], "peak_file": src,
            "traffic": traffic, "traffic_algorithmic": alg_bytes, "kernel_sources_sha": sha}


# ---------------------------------------------------------------- oracle
def oracle_step_rate(w, budget_s: float = 15.0, cells=None):
    """The oracle's TR-BDF2 step (assembled operators, sparse direct solves)
    on a small mesh of the same workload (the channel keeps its aspect:
    4:1:1); GDoF/s = that mesh's DoFs / s per step."""
    from oracle.dg import Mesh as OMesh, lib as olib
    from oracle.trbdf2 import Stepper
    if cells is None:
        cells = (8, 2, 2) if w.name == "channel" else (4,) * w.dim
    ws = w.scaled(tuple(cells))
    om = OMesh(ws.dim, list(ws.n), list(ws.lo), list(ws.hi), list(ws.periodic), ws.degree,
               map=ws.map, map_param=list(ws.map_param))
    X, Xp = om.node_coords(), om.node_coords(True)
    u, p = W.initial_state(ws, X, Xp)
    uh = u.copy()
    fh = W.forcing(ws, X)
    force = None if fh is None else (lambda t: fh)
    t0 = time.perf_counter()
    st = Stepper(om, ws.Re, c=ws.c)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    steps = 0
    while steps == 0 or time.perf_counter() - t0 < budget_s:
        u, p, uh = st.step(u, p, uh, steps * ws.dt, ws.dt, f=force)
        steps += 1
    dt = (time.perf_counter() - t0) / steps
    dofs = ws.n_dofs_u + ws.n_dofs_p
    return {"value": dofs / dt / 1e9, "unit": "GDoF/s", "cores": int(olib().ora_num_threads()),
            "kind": "oracle", "ms_per_step": dt * 1e3, "mesh": workload_label(ws),
            "sample": f"{steps} oracle TR-BDF2 steps on the {'x'.join(map(str, ws.n))} mesh of "
                      f"the {w.name} workload ({dofs} DoFs; measured there, not extrapolated; "
                      f"constant operators assembled once in {setup:.1f} s, not timed; per step: "
                      f"advection assembly on the OpenMP threads and sparse LU solves to machine "
                      f"precision, which SuperLU runs on one thread)"}


def oracle_apply_rate(w, budget_s: float = 5.0):
    """The oracle's momentum operator (assembled cell blocks, OpenMP block
    product) applied to the 3 velocity components at the workload's full
    size: GDoF/s = velocity DoFs / s per apply (assembly not timed)."""
    from oracle.dg import BlockOp, Mesh as OMesh, lib as olib
    om = OMesh(w.dim, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree,
               map=w.map, map_param=list(w.map_param))
    X, Xp = om.node_coords(), om.node_coords(True)
    ub = W.initial_state(w, X, Xp)[0]
    if not np.any(ub):
        ub = W.forcing(w, X)
    g = 2.0 - math.sqrt(2.0)
    t0 = time.perf_counter()
    M = om.assemble("mass_u")
    blocks = (1.0 / (g * w.dt)) * M.blocks
    blocks += (1.0 / (2 * w.Re)) * om.assemble("sipg_u").blocks
    blocks += 0.5 * om.assemble("adv_u", ub.reshape(-1)).blocks
    op = BlockOp(blocks, M.cols, M.nt, M.ns, M.ncol_cells)
    setup = time.perf_counter() - t0
    x = W.random_vector(w.dim * om.n_u, 1).reshape(w.dim, -1)
    t0, reps = time.perf_counter(), 0
    while reps == 0 or time.perf_counter() - t0 < budget_s:
        for c in range(w.dim):
            op.apply(x[c])
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    return {"value": w.dim * om.n_u / dt / 1e9, "unit": "GDoF/s",
            "cores": int(olib().ora_num_threads()), "ms_per_apply": dt * 1e3,
            "sample": f"oracle momentum operator (assembled 27x27 blocks, 7 per cell row) applied "
                      f"{reps} times to the {w.dim} components at the full {workload_label(w)} "
                      f"size ({w.dim * om.n_u} DoFs; assembly {setup:.1f} s, not timed)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="channel", choices=sorted(W.WORKLOADS))
    ap.add_argument("--secondary", default="tgv32",
                    help="a second, smaller workload reported under 'secondary' ('' for none)")
    ap.add_argument("--solver", default="mixed+learned", choices=sorted(SOLVERS))
    ap.add_argument("--train-steps", type=int, default=None,
                    help="untimed steps before the warm-up (the learned guess trains on them); "
                         "default per workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-guess-study", action="store_true",
                    help="skip the 400-step learned-guess study on the 48^3 vortex")
    ap.add_argument("--mg-degree", type=int, default=0,
                    help="Chebyshev degree of the multigrid smoother for --solver (0: its default)")
    ap.add_argument("--oracle-budget", type=float, default=30.0,
                    help="seconds of oracle steps in the reference arm")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w = W.WORKLOADS[args.workload]
    cfg = {"workload": workload_label(w),
           "step": "one TR-BDF2 step: 2 Jacobi-GMRES(30) momentum solves + 2 multigrid-FCG "
                   "Helmholtz solves to 1e-8 relative residual, RHS, projections, updates",
           "solver": args.solver,
           "l2": "512 MiB buffer written between timed steps; working set > L2",
           "parallelism": f"replicas x{args.gpus}"}
    if args.impl == "reference":
        if rank != 0:
            return
        cb = oracle_step_rate(w, budget_s=args.oracle_budget)
        cfg_ref = dict(cfg, workload=cb["mesh"] + f" (a sample of {w.name}; the oracle runs on "
                                                  f"the host cores)")
        apply = oracle_apply_rate(W.TGV32)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GDoF/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": cb["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 (CPU oracle)", "data": "synthetic",
                "config": cfg_ref, "cpu_baseline": dict(cb, apply=apply),
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
        cb = oracle_step_rate(w)
        cb["apply"] = oracle_apply_rate(W.TGV32)
    line = {"metric": METRIC, "value": r["value"], "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE,
            "data": "synthetic", "config": cfg, "clocks": r["clocks"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "iterations_per_step": r["iterations"],
            "solvers": r["solvers"], "apply": r["apply"], "roofline": r["roofline"],
            "secondary": r["secondary"], "guess_study": r["guess_study"],
            "autotune": r["autotune"], "cpu_baseline": cb}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
