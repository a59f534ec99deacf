"""Convergence study of the Arnold-Beltrami-Childress flow on the GPU (Section
4.1: 3D periodic cube [0,2pi]^3, Re = 1, T = 3.2, Q2/Q1 and Q3/Q2).

python -m paper_2107_07776_gb300.abcstudy [--degree 2] [--scaling hyperbolic]
        [--cells 8 16 32] [--tol 1e-10]

Each row starts from the closed form at t = 0 (and its value at
t = -(1-gamma) dt as the stage-1 history), takes ceil(T/dt) TR-BDF2 steps
through the library (Jacobi-GMRES momentum, FP64 multigrid Helmholtz, both
to the relative residual --tol) and reports the relative L2 errors of u and
p and the relative H1 error of u against the closed form at the final time,
by the cells' (k+1)-point Gauss-Legendre rule at the nodes (the collocated
basis makes the nodes the quadrature points).  Hyperbolic scaling halves dt
with each doubling of the cells (C = 1.63 on the coarsest mesh: dt 0.32 for
Q2, 0.21 for Q3, as printed); parabolic scaling quarters it (mu = 2: dt 0.32
and 0.14 on 8^3).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

import workloads as W

from . import binding as b

T_FINAL = 3.2
DT0 = {(2, "hyperbolic"): 0.32, (3, "hyperbolic"): 0.21,
       (2, "parabolic"): 0.32, (3, "parabolic"): 0.14}


def abc_gradient(x, y, z, t, Re):
    """d u_i / d x_j of the closed form, [i][j]."""
    e = math.exp(-t / Re)
    zero = np.zeros_like(x)
    return [[zero, -np.sin(y) * e, np.cos(z) * e],
            [np.cos(x) * e, zero, -np.sin(z) * e],
            [-np.sin(x) * e, np.cos(y) * e, zero]]


def nodal_errors(w, mesh, u, p, t):
    """Relative L2 errors of u and p and relative H1 (seminorm) error of u at
    the nodes of a uniform periodic mesh, Gauss-Legendre weights."""
    k = w.degree
    n = w.n[0]
    h = (w.hi[0] - w.lo[0]) / n
    X = mesh.node_coords(0).cpu().numpy()
    Xp = mesh.node_coords(1).cpu().numpy()
    xg, wg = np.polynomial.legendre.leggauss(k + 1)
    wu = np.einsum("i,j,k->kji", wg, wg, wg).reshape(-1) * (h / 2) ** 3
    xq, wq = np.polynomial.legendre.leggauss(k)
    wp = np.einsum("i,j,k->kji", wq, wq, wq).reshape(-1) * (h / 2) ** 3
    ncell = mesh.n_cells
    wu = np.tile(wu, ncell)
    wp = np.tile(wp, ncell)
    ue = W.abc_u(*X, t, w.Re)
    pe = W.abc_p(*Xp, t, w.Re)
    uh = u.reshape(3, -1)
    eu = math.sqrt(sum((wu * (uh[i] - ue[i]) ** 2).sum() for i in range(3)) /
                   sum((wu * ue[i] ** 2).sum() for i in range(3)))
    ep = math.sqrt((wp * (p - pe) ** 2).sum() / (wp * pe ** 2).sum())
    # gradient of the discrete field by 1D differentiation along each axis
    nodes = (xg + 1) / 2
    Dm = np.zeros((k + 1, k + 1))
    for j in range(k + 1):
        c = np.zeros(k + 1)
        c[j] = 1.0
        lag = np.polynomial.polynomial.Polynomial.fit(nodes, c, k, domain=[0, 1], window=[0, 1])
        Dm[:, j] = lag.deriv()(nodes)
    G = abc_gradient(*X, t, w.Re)
    num = den = 0.0
    for i in range(3):
        v = uh[i].reshape(ncell, k + 1, k + 1, k + 1) / h   # (cell, z, y, x)
        grads = [np.einsum("qa,czya->czyq", Dm, v), np.einsum("qa,czax->czqx", Dm, v),
                 np.einsum("qa,caxy->cqxy", Dm, v)]
        for j in range(3):
            num += (wu * (grads[j].reshape(-1) - G[i][j]) ** 2).sum()
            den += (wu * G[i][j] ** 2).sum()
    return eu, ep, math.sqrt(num / den)


def run_row(N, degree, dt, tol=1e-10, stream=None):
    import torch
    w = W.ABC.scaled((N, N, N), degree=degree, dt=dt)
    mesh = b.Mesh.from_workload(w)
    X = mesh.node_coords(0).cpu().numpy()
    Xp = mesh.node_coords(1).cpu().numpy()
    u = torch.tensor(W.abc_u(*X, 0.0, w.Re).reshape(-1), dtype=torch.float64, device="cuda")
    p = torch.tensor(W.abc_p(*Xp, 0.0, w.Re), dtype=torch.float64, device="cuda")
    uh = torch.tensor(W.abc_u(*X, -(1 - b.GAMMA) * dt, w.Re).reshape(-1), dtype=torch.float64,
                      device="cuda")
    s = b.dg_solver_create(mesh.handle, w.Re, w.c)
    steps = math.ceil(T_FINAL / dt - 1e-9)
    iters = []
    try:
        b.dg_solver_set_history(s, uh)
        prm = b.dg_step_params()
        prm.dt, prm.gamma, prm.extrapolate = dt, 0.0, 1
        prm.mom = b.solve_opts(b.DG_SYS_MOMENTUM, tol=tol, max_iter=5000, restart=30,
                               precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_EXTRAP)
        prm.helm = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=tol, max_iter=500,
                                precond=b.DG_PC_MG_FP64, guess=b.DG_GUESS_EXTRAP)
        t0 = time.perf_counter()
        for _ in range(steps):
            info = b.trbdf2_step(s, prm, u, p)
            iters.append([i.iterations for i in info])
        wall = time.perf_counter() - t0
    finally:
        b.dg_solver_destroy(s)
    t = steps * dt
    eu, ep, eh1 = nodal_errors(w, mesh, u.cpu().numpy(), p.cpu().numpy(), t)
    mesh.close()
    return {"cells": N, "degree": degree, "dt": dt, "steps": steps, "t": t, "l2_u": eu,
            "h1_u": eh1, "l2_p": ep, "s_per_step": wall / steps,
            "iterations_per_step": np.array(iters).mean(axis=0).round(2).tolist()}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--scaling", default="hyperbolic", choices=["hyperbolic", "parabolic"])
    ap.add_argument("--cells", type=int, nargs="+", default=[8, 16, 32])
    ap.add_argument("--tol", type=float, default=1e-10)
    args = ap.parse_args(argv)
    dt = DT0[(args.degree, args.scaling)]
    rows = []
    for i, N in enumerate(args.cells):
        f = N / args.cells[0]
        rows.append(run_row(N, args.degree, dt / (f if args.scaling == "hyperbolic" else f * f),
                            args.tol))
    for a, c in zip(rows, rows[1:]):
        r = math.log(c["cells"] / a["cells"])
        c["rate_l2_u"] = math.log(a["l2_u"] / c["l2_u"]) / r
        c["rate_h1_u"] = math.log(a["h1_u"] / c["h1_u"]) / r
        c["rate_l2_p"] = math.log(a["l2_p"] / c["l2_p"]) / r
    print(json.dumps({"workload": "abc", "scaling": args.scaling, "Re": 1.0, "T": T_FINAL,
                      "rows": rows}))


if __name__ == "__main__":
    main()
