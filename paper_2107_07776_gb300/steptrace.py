"""Where one TR-BDF2 step's time goes, for a workload on one GPU.

python -m paper_2107_07776_gb300.steptrace [--workload channel] [--train 6] [--traced 5]

Builds the workload's autotuned mesh and the benchmark's default solver
(FP32 multigrid Helmholtz with the learned initial guess, smoother degree 8),
takes --train untimed steps with the guess training, then --traced steps
with the library's phase tracing on (CUDA events at the phase boundaries;
dg_solver_set_tracing) and prints the mean milliseconds per step of each
phase as one JSON line.  Finally it takes one more step between
cudaProfilerStart and cudaProfilerStop, so that

    ncu --metrics gpu__time_duration.sum --clock-control none \\
        --profile-from-start off --csv --log-file launches.csv \\
        python -m paper_2107_07776_gb300.steptrace --workload channel

lists exactly the kernel launches of one step.
"""
from __future__ import annotations

import argparse
import json

import workloads as W

from . import binding as b


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="channel", choices=sorted(W.WORKLOADS))
    ap.add_argument("--train", type=int, default=6)
    ap.add_argument("--traced", type=int, default=5)
    ap.add_argument("--mg-degree", type=int, default=8)
    args = ap.parse_args(argv)

    import torch

    torch.cuda.set_device(0)
    w = W.WORKLOADS[args.workload]
    mesh = b.Mesh.from_workload(w)
    b.dg_autotune(mesh.handle)
    X = mesh.node_coords(0).cpu().numpy()
    Xp = mesh.node_coords(1).cpu().numpy()
    u0, p0 = W.initial_state(w, X, Xp)
    u = torch.tensor(u0.reshape(-1), dtype=torch.float64, device="cuda")
    p = torch.tensor(p0, dtype=torch.float64, device="cuda")
    fh = W.forcing(w, X)
    f = None if fh is None else torch.tensor(fh.reshape(-1), dtype=torch.float64, device="cuda")
    s = b.dg_solver_create(mesh.handle, w.Re, w.c)
    try:
        prm = b.dg_step_params()
        prm.dt, prm.gamma, prm.extrapolate = w.dt, 0.0, 1
        if f is not None:
            prm.f_n = prm.f_ng = prm.f_n1 = f.data_ptr()
        prm.mom = b.solve_opts(b.DG_SYS_MOMENTUM, tol=1e-8, max_iter=500, restart=30,
                               precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_LEARNED)
        prm.helm = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-8, max_iter=500,
                                precond=b.DG_PC_MG_FP32, guess=b.DG_GUESS_LEARNED,
                                mg_degree=args.mg_degree)
        b.dg_guess_configure(s, enable=1, train=1, systems=1)
        for _ in range(args.train):
            b.trbdf2_step(s, prm, u, p)
        b.dg_guess_configure(s, enable=1, train=0, systems=1)
        b.dg_solver_set_tracing(s, 1)
        for _ in range(args.traced):
            info = b.trbdf2_step(s, prm, u, p)
        phases, n = b.dg_solver_get_trace(s)
        b.dg_solver_set_tracing(s, 0)
        print(json.dumps({"workload": w.name, "phase_ms_per_step": {k: v / max(n, 1) for k, v in phases.items()},
                          "iterations": [i.iterations for i in info]}))
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        b.trbdf2_step(s, prm, u, p)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    finally:
        b.dg_solver_destroy(s)


if __name__ == "__main__":
    main()
