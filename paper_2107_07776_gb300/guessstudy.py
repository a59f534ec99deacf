"""The learned initial guess against the extrapolated one over a long run:
train on the first half of the steps, evaluate on the second half.

python -m paper_2107_07776_gb300.guessstudy [--workload tgv48] [--steps 400]
        [--train 200] [--systems 3] [--precond mg_fp32] [--tol 1e-8]

Two solvers advance the same initial state of the workload (48^3 Q2/Q1
Taylor-Green vortex by default) through the same TR-BDF2 steps:
  extrapolated  every stage solve starts from 2 x_{k-1} - x_{k-2};
  learned       the per-cell MLP adds its correction (systems: bit 0 pressure
                Helmholtz, bit 1 momentum).  It trains (one Adam step per
                solve, on that solve's converged solution) during the first
                --train steps and only infers afterwards.
Both solve every stage to the same relative residual, so the answers agree
to that tolerance; the comparison is the number of Krylov iterations per
solve and the time per step (CUDA events, initial residual norms), averaged
over the evaluation steps.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

import workloads as W

from . import binding as b


def run(w, steps: int, train: int, learned: bool, systems: int, precond: int, tol: float):
    import torch

    dev = torch.device("cuda", 0)
    mesh = b.Mesh.from_workload(w)
    b.dg_autotune(mesh.handle)
    X = mesh.node_coords(0).cpu().numpy()
    Xp = mesh.node_coords(1).cpu().numpy()
    u0h, p0h = W.initial_state(w, X, Xp)
    u = torch.tensor(u0h.reshape(-1), dtype=torch.float64, device=dev)
    p = torch.tensor(p0h, dtype=torch.float64, device=dev)
    fh = W.forcing(w, X)
    f = None if fh is None else torch.tensor(fh.reshape(-1), dtype=torch.float64, device=dev)
    s = b.dg_solver_create(mesh.handle, w.Re, w.c)
    guess = b.DG_GUESS_LEARNED if learned else b.DG_GUESS_EXTRAP
    prm = b.dg_step_params()
    prm.dt, prm.gamma, prm.extrapolate = w.dt, 0.0, 1
    prm.mom = b.solve_opts(b.DG_SYS_MOMENTUM, tol=tol, max_iter=1000, restart=30,
                           precond=b.DG_PC_JACOBI, guess=guess)
    prm.helm = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=tol, max_iter=1000, precond=precond, guess=guess)
    if f is not None:
        prm.f_n = prm.f_ng = prm.f_n1 = f.data_ptr()
    stream = torch.cuda.current_stream(dev)
    rows = []
    try:
        for k in range(steps):
            if learned and k == 0:
                b.dg_guess_configure(s, enable=1, train=1, systems=systems, lr=1e-3, seed=1)
            if learned and k == train:
                b.dg_guess_configure(s, enable=1, train=0, systems=systems, lr=1e-3, seed=1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = b.trbdf2_step(s, prm, u, p)
            e1.record(stream)
            torch.cuda.synchronize()
            rows.append(([i.iterations for i in info], [i.res0 for i in info], e0.elapsed_time(e1)))
        stats = b.dg_guess_get_stats(s) if learned else None
    finally:
        b.dg_solver_destroy(s)
        mesh.close()
    ev = rows[train:]
    its = np.array([r[0] for r in ev], dtype=float)
    res0 = np.array([r[1] for r in ev], dtype=float)
    out = {"iterations_per_solve": its.mean(axis=0).round(3).tolist(),
           "initial_residual": res0.mean(axis=0).tolist(),
           "ms_per_step": statistics.mean(r[2] for r in ev),
           "u_final_norm": float(torch.linalg.vector_norm(u).item()),
           "p_final_norm": float(torch.linalg.vector_norm(p).item())}
    if stats is not None:
        out["train_steps"] = int(stats.train_steps)
        out["last_loss"] = float(stats.last_loss)
    return out, u.cpu().numpy(), p.cpu().numpy()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tgv48", choices=sorted(W.WORKLOADS))
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--systems", type=int, default=3)
    ap.add_argument("--precond", default="mg_fp32", choices=["mg_fp32", "mg_fp64", "jacobi"])
    ap.add_argument("--tol", type=float, default=1e-8)
    args = ap.parse_args(argv)
    if not 0 < args.train < args.steps:
        ap.error("need 0 < --train < --steps")
    pc = {"mg_fp32": b.DG_PC_MG_FP32, "mg_fp64": b.DG_PC_MG_FP64, "jacobi": b.DG_PC_JACOBI}[args.precond]
    w = W.WORKLOADS[args.workload]
    base, ub, pb = run(w, args.steps, args.train, False, args.systems, pc, args.tol)
    lrn, ul, pl = run(w, args.steps, args.train, True, args.systems, pc, args.tol)
    line = {"workload": w.name, "steps": args.steps, "train_steps": args.train,
            "evaluated_steps": args.steps - args.train, "systems": args.systems,
            "precond": args.precond, "tol": args.tol, "extrapolated": base, "learned": lrn,
            "iterations_ratio": (np.array(base["iterations_per_solve"]).sum()
                                 / max(np.array(lrn["iterations_per_solve"]).sum(), 1e-30)),
            "step_time_ratio": base["ms_per_step"] / lrn["ms_per_step"],
            "final_u_rel_diff": float(np.linalg.norm(ul - ub) / np.linalg.norm(ub)),
            "final_p_rel_diff": float(np.linalg.norm(pl - pb) / np.linalg.norm(pb))}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
