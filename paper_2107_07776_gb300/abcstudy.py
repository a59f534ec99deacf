"""Convergence study of the Arnold-Beltrami-Childress flow on the GPU (Section
4.1: 3D periodic cube [0,2pi]^3, Re = 1, T = 3.2, Q2/Q1 and Q3/Q2).

python -m paper_2107_07776_gb300.abcstudy [--degree 2] [--scaling hyperbolic]
        [--cells 8 16 32] [--tol 1e-10]

Each row starts from the closed form at t = 0 (and its value at
t = -(1-gamma) dt as the stage-1 history), takes ceil(T/dt) TR-BDF2 steps
through the library (Jacobi-GMRES momentum, FP64 multigrid Helmholtz, both
to the relative residual --tol) and reports the relative L2 errors of u and
p and the relative H1 error of u against the closed form at the final time,
by a (k+3)-point Gauss-Legendre rule per direction.  Hyperbolic scaling halves dt
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


def _lagrange_at(n1, m):
    """Values and derivatives on [0,1] of the nodal basis on the n1
    Gauss-Legendre points at the m-point Gauss-Legendre rule, and its
    weights."""
    nodes = (np.polynomial.legendre.leggauss(n1)[0] + 1) / 2
    xq, wq = np.polynomial.legendre.leggauss(m)
    pts = (xq + 1) / 2
    I = np.ones((m, n1))
    Dq = np.zeros((m, n1))
    for j in range(n1):
        for l in range(n1):
            if l != j:
                I[:, j] *= (pts - nodes[l]) / (nodes[j] - nodes[l])
        for l in range(n1):
            if l == j:
                continue
            t = np.full(m, 1.0 / (nodes[j] - nodes[l]))
            for r in range(n1):
                if r != j and r != l:
                    t *= (pts - nodes[r]) / (nodes[j] - nodes[r])
            Dq[:, j] += t
    return I, Dq, pts, wq / 2


def nodal_errors(w, mesh, u, p, t):
    """Relative L2 errors of u and p and relative H1 (seminorm) error of u on
    a uniform periodic mesh, by a (k+3)-point Gauss-Legendre rule per
    direction (the discrete fields interpolated from their nodes)."""
    k, n = w.degree, w.n[0]
    h = (w.hi[0] - w.lo[0]) / n
    m = k + 3
    ncell = n ** 3
    c = np.arange(ncell)
    ci = [c % n, (c // n) % n, c // (n * n)]

    def points(pts):
        # physical coordinates (cell, s, r, q) of the rule's points
        g = [w.lo[a] + (ci[a][:, None] + pts[None, :]) * h for a in range(3)]
        return (np.broadcast_to(g[0][:, None, None, :], (ncell, m, m, m)),
                np.broadcast_to(g[1][:, None, :, None], (ncell, m, m, m)),
                np.broadcast_to(g[2][:, :, None, None], (ncell, m, m, m)))

    def at_points(v, n1, I, D=(None, None, None)):
        v = v.reshape(ncell, n1, n1, n1)  # (cell, z, y, x)
        A = [I if D[a] is None else D[a] for a in range(3)]
        return np.einsum("sz,ry,qx,czyx->csrq", A[2], A[1], A[0], v)

    Iu, Du, pts, wq = _lagrange_at(k + 1, m)
    W3 = np.einsum("s,r,q->srq", wq, wq, wq)[None] * h ** 3
    X = points(pts)
    ue = W.abc_u(*X, t, w.Re)
    G = abc_gradient(*X, t, w.Re)
    uh = u.reshape(3, -1)
    e2 = n2 = g2 = d2 = 0.0
    for i in range(3):
        ui = at_points(uh[i], k + 1, Iu)
        e2 += (W3 * (ui - ue[i]) ** 2).sum()
        n2 += (W3 * ue[i] ** 2).sum()
        for j in range(3):
            D = [None, None, None]
            D[j] = Du / h
            gj = at_points(uh[i], k + 1, Iu, D)
            g2 += (W3 * (gj - G[i][j]) ** 2).sum()
            d2 += (W3 * G[i][j] ** 2).sum()
    Ip, _, _, _ = _lagrange_at(k, m)
    pe = W.abc_p(*X, t, w.Re)
    ph = at_points(p, k, Ip)
    ep = math.sqrt((W3 * (ph - pe) ** 2).sum() / (W3 * pe ** 2).sum())
    return math.sqrt(e2 / n2), ep, math.sqrt(g2 / d2)


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
