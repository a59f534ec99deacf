"""Benchmark of the DG TR-BDF2 hot path on one GB300 (replicas on N GPUs).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload tgv32] [--solver mixed|plain]

One step = one TR-BDF2 step (Section 2: two momentum predictors solved by
Jacobi-GMRES, two pressure Helmholtz solves by flexible CG with h/p multigrid,
RHS assembly, projections and updates) on the workload's state, all inside
the CUDA library; inputs resident in HBM.  value = (velocity + pressure
DoFs) advanced per second (GDoF/s); ms_per_step = the time per TR-BDF2 step.
"mixed+learned" (default): FP32 multigrid inside the FP64 outer Krylov
solves and the learned initial guess (trained in an untimed phase of
--train-steps steps before the warm-up, inference only while timed);
"mixed": the same with the linearly extrapolated guess; "plain": FP64
multigrid and the extrapolated guess.  The other solvers' times per step are
reported in "compare"; every solver first takes the same --train-steps +
--warmup untimed steps, so all of them time the same window of the flow.  Solves stop at a relative residual of 1e-8.

Timing: W untimed warm-up steps; K timed steps, each bracketed by CUDA events
on the launching stream, with a 512 MiB buffer written between steps (L2 is
135 MB) so every step starts cold; barrier + synchronize on both sides; max
over ranks (replicas: no collective inside a step).  e2e: the same step
through the C ABI from pinned host buffers, host<->device copies of u and p
inside the timed region.  apply: GDoF/s of each operator apply alone (CUDA
events over K launches, same launch configuration as inside the step).
roofline: the dominant kernel (FP64 momentum apply) as algorithmic flops per
launch / its CUDA-event duration against the FP64 FMA peak.  cpu_baseline
and --impl reference: the oracle's TR-BDF2 step on a reduced mesh of the
same workload, on the host cores.
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
# FP64 FMA peak of GB300: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz = 1.259
# TFLOP/s from the unit counts; an FMA-chain probe measured 1.253
FP64_PEAK_TFLOPS = 1.253
FP32_PEAK_TFLOPS = 76.5    # measured FP32 FMA throughput
# FP64-equivalent ceiling of float-float arithmetic: one fused multiply-add
# (df_fma) costs 15 FP32-pipe instructions; 152 SMs x 128 lanes x 2.07 GHz
# / 15 x 2 flop
FLOAT_FLOAT_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 15 * 2 / 1e12


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel, the float-float momentum apply, from an ncu capture of
# the bench's launch configuration; to be re-captured whenever the kernel
# changes
# (face-once form: flux kernel + cell kernel of one apply)
NCU_TRAFFIC_BYTES = {"tgv32": 42662656 + 7026688 + 85345536 + 7072256}


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
    # (each with the Chebyshev degree that was fastest for it on tgv32:
    # the learned guess pays more when iterations are dearer)
    "mixed+learned": ("DG_PC_MG_FP32", "DG_GUESS_LEARNED", True, 8),
    "mixed": ("DG_PC_MG_FP32", "DG_GUESS_EXTRAP", False, 5),
    "plain": ("DG_PC_MG_FP64", "DG_GUESS_EXTRAP", False, 5),
}


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
    X = mesh.node_coords(0).cpu().numpy()
    Xp = mesh.node_coords(1).cpu().numpy()
    u0h, p0h = W.initial_state(w, X, Xp)
    fh = W.forcing(w, X)
    fdev = None if fh is None else torch.tensor(fh.reshape(-1), dtype=torch.float64, device=dev)
    u0 = torch.tensor(u0h.reshape(-1), dtype=torch.float64, device=dev)
    p0 = torch.tensor(p0h, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    def timed_steps(name, nsteps, nwarm, sample_clocks=False):
        # every solver takes the same untimed steps (training phase of the
        # learned guess + warm-up) so all time the same window of the flow
        pc, guess, learned, deg = SOLVERS[name]
        if name == args.solver and args.mg_degree:
            deg = args.mg_degree
        pc, guess = getattr(b, pc), getattr(b, guess)
        s = b.dg_solver_create(mesh.handle, w.Re, w.c)
        u, p = u0.clone(), p0.clone()
        prm = step_params(b, w, pc, guess, f=fdev, mg_degree=deg)
        if learned:  # untimed training phase, then inference only
            b.dg_guess_configure(s, enable=1, train=1, systems=1, lr=1e-3, seed=1)
        for _ in range(args.train_steps):
            b.trbdf2_step(s, prm, u, p)
        if learned:
            b.dg_guess_configure(s, enable=1, train=0, systems=1, lr=1e-3, seed=1)
        iters = []
        for _ in range(nwarm):
            b.trbdf2_step(s, prm, u, p)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(dev.index)
        if sample_clocks:
            clk.__enter__()
        launches0 = b.dg_kernel_launches()
        for i in range(nsteps):
            flush.fill_(i & 0xFF)
            if sample_clocks and args.profile_step and i == 0:
                torch.cuda.profiler.start()
            ev[i][0].record(stream)
            info = b.trbdf2_step(s, prm, u, p)
            ev[i][1].record(stream)
            if sample_clocks and args.profile_step and i == 0:
                torch.cuda.profiler.stop()
            iters.append([x.iterations for x in info])
        launches = b.dg_kernel_launches() - launches0
        torch.cuda.synchronize()
        if sample_clocks:
            clk.__exit__(None, None, None)
        if world > 1:
            torch.distributed.barrier()
        ms = [a.elapsed_time(c) for a, c in ev]
        return ms, iters, clk.summary(), launches, (s, prm, u, p)

    ms, iters, clocks, launches, (s_main, prm_main, u_main, p_main) = timed_steps(args.solver, args.steps,
                                                                  args.warmup, True)
    dofs = mesh.n_dofs_u + mesh.n_dofs_p
    ms_per_step, value = job_rate(sum(ms), args.steps, dofs, world, dev)
    compare = {}
    for other in SOLVERS:
        if other == args.solver:
            continue
        ms_o, iters_o, _, _, (s_o, _, _, _) = timed_steps(other, max(3, args.steps // 2), args.warmup)
        b.dg_solver_destroy(s_o)
        compare[other] = {"ms_per_step": statistics.mean(ms_o), "mg_degree": SOLVERS[other][3],
                          "iterations_per_step": np.array(iters_o).mean(axis=0).round(2).tolist()}

    # ---- end to end through the C ABI with pinned host buffers ----
    s, prm = s_main, prm_main
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
    e2e_ms = e_a.elapsed_time(e_b) / args.steps
    nbytes = 8 * dofs
    e2e = {"value": dofs * world / (e2e_ms * 1e-3) / 1e9, "unit": "GDoF/s",
           "ms_per_step": e2e_ms, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # ---- operator applies alone (same launch configuration as in the step) ----
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
    apply = {k: (calls[k][1] / (v * 1e-3) / 1e9) for k, v in apply_ms.items()}
    apply = {k + "_gdofs": round(v, 4) for k, v in apply.items()}
    fl = w.dim * mesh.n_cells * apply_flops_per_cell(w.dim, w.degree + 1, True)
    achieved = fl / (apply_ms["momentum_fp64"] * 1e-3) / 1e12
    pk, src = peaks()
    face_once = False
    for r in autotune or []:
        if r.get("op") == "momentum+advection" and r.get("precision") == "f64":
            face_once = bool(r["face_once"][r["chosen_variant"]])
    if w.map == 2:
        kname = ("general_op_kernel<double,df64> (momentum apply on trilinear cells; flop model of "
                 "the affine operator, a lower bound of the work)")
    elif face_once:
        kname = ("face_flux_kernel + cell_split_kernel<double,df64> (momentum apply, face-once form, "
                 "float-float FP64 arithmetic)")
    else:
        kname = "scalar_op_kernel<double,df64> (momentum apply, float-float FP64 arithmetic)"
    roof = {"bound": "alu", "kernel": kname,
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": (args.traffic if args.traffic is not None
                        else (NCU_TRAFFIC_BYTES.get(w.name) if face_once else None)),
            "traffic_algorithmic": 24 * mesh.n_dofs_u,
            "frac_of_float_float_ceiling": achieved / FLOAT_FLOAT_PEAK_TFLOPS,
            "peak_source": "FP64 FMA: 152 SMs x 2 FMA/clk x 2.07 GHz (1.259), measured 1.253",
            "hbm_frac_poisson_fp32": (8 * mesh.n_dofs_p / (apply_ms["poisson_fp32"] * 1e-3) / 1e9)
                                     / pk["hbm_gbs"]}
    it = np.array(iters)
    return dict(value=value, ms_per_step=ms_per_step, clocks=clocks, e2e=e2e, roofline=roof,
                gpu_launches=launches,
                iterations=it.mean(axis=0).round(2).tolist(), compare=compare, apply=apply,
                dofs=dofs, autotune=autotune)


# ---------------------------------------------------------------- oracle
def oracle_step_rate(w, budget_s: float = 15.0, n_small: int = 4):
    """The oracle's TR-BDF2 step (assembled operators, sparse direct solves)
    on an n_small^d mesh of the same workload; GDoF/s = DoFs / s per step."""
    from oracle.dg import Mesh as OMesh, lib as olib
    from oracle.trbdf2 import Stepper
    ws = w.scaled(tuple([n_small] * w.dim))
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
            "kind": "oracle", "ms_per_step": dt * 1e3,
            "sample": f"{steps} oracle TR-BDF2 steps on the {'x'.join(map(str, ws.n))} mesh of "
                      f"the same workload ({dofs} DoFs; constant operators assembled once in "
                      f"{setup:.1f} s, not timed; per step: advection assembly on the OpenMP "
                      f"threads and sparse LU solves to machine precision, which SuperLU runs on "
                      f"one thread)"}


def oracle_apply_rate(w, n_small: int = 16, budget_s: float = 5.0):
    """The oracle's momentum operator (assembled cell blocks, OpenMP block
    product) applied to the 3 velocity components on an n_small^d mesh of
    the workload: GDoF/s = velocity DoFs / s per apply."""
    from oracle.dg import BlockOp, Mesh as OMesh, lib as olib
    ws = w.scaled(tuple(min(n_small, n) for n in w.n))
    om = OMesh(ws.dim, list(ws.n), list(ws.lo), list(ws.hi), list(ws.periodic), ws.degree,
               map=ws.map, map_param=list(ws.map_param))
    X, Xp = om.node_coords(), om.node_coords(True)
    ub = W.initial_state(ws, X, Xp)[0]
    if not np.any(ub):
        ub = W.forcing(ws, X)
    g = 2.0 - math.sqrt(2.0)
    M, A, C = om.assemble("mass_u"), om.assemble("sipg_u"), om.assemble("adv_u", ub.reshape(-1))
    op = BlockOp(1.0 / (g * ws.dt) * M.blocks + 1.0 / (2 * ws.Re) * A.blocks + 0.5 * C.blocks,
                 M.cols, M.nt, M.ns, M.ncol_cells)
    x = W.random_vector(ws.dim * om.n_u, 1).reshape(ws.dim, -1)
    t0, reps = time.perf_counter(), 0
    while reps == 0 or time.perf_counter() - t0 < budget_s:
        for c in range(ws.dim):
            op.apply(x[c])
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    return {"value": ws.dim * om.n_u / dt / 1e9, "unit": "GDoF/s", "cores": int(olib().ora_num_threads()),
            "sample": f"oracle momentum operator (assembled blocks) applied {reps} times to the "
                      f"{ws.dim} components on the {'x'.join(map(str, ws.n))} mesh "
                      f"({ws.dim * om.n_u} DoFs)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv32", choices=sorted(W.WORKLOADS))
    ap.add_argument("--solver", default="mixed+learned", choices=sorted(SOLVERS))
    ap.add_argument("--train-steps", type=int, default=200,
                    help="untimed steps before the warm-up (the learned guess trains on them)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the dominant kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--mg-degree", type=int, default=0,
                    help="Chebyshev degree of the multigrid smoother for --solver (0: its default)")
    ap.add_argument("--profile-step", action="store_true",
                    help="bracket the first timed step with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w = W.WORKLOADS[args.workload]
    cfg = {"workload": f"{w.name}: {w.dim}D {'x'.join(map(str, w.n))} cells, DG Q{w.degree}/"
                       f"Q{w.degree - 1}, Re {w.Re:g}, c {w.c:g}, dt {w.dt:g}",
           "step": "one TR-BDF2 step: 2 Jacobi-GMRES(30) momentum solves + 2 multigrid-FCG "
                   "Helmholtz solves to 1e-8 relative residual, RHS, projections, updates",
           "solver": args.solver,
           "l2": "512 MiB buffer written between timed steps",
           "parallelism": f"replicas x{args.gpus}"}
    if args.impl == "reference":
        if rank != 0:
            return
        budget = max(5.0, 120.0 / max(1, args.steps + args.warmup))
        cb = oracle_step_rate(w, budget_s=budget)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GDoF/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": (w.n_dofs_u + w.n_dofs_p) / (cb["value"] * 1e9) * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg, "cpu_baseline": cb,
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
        cb["apply"] = oracle_apply_rate(w)
    line = {"metric": METRIC, "value": r["value"], "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "clocks": r["clocks"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "iterations_per_step": r["iterations"],
            "compare": r["compare"], "apply": r["apply"], "roofline": r["roofline"],
            "autotune": r["autotune"], "mg_degree": args.mg_degree or SOLVERS[args.solver][3], "cpu_baseline": cb}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
