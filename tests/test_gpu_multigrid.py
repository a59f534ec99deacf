"""h/p multigrid preconditioning of the pressure Helmholtz systems: the
flexible CG with an FP32 (mixed precision) or FP64 V-cycle reaches the same
solution as the oracle's direct solve, on meshes that exercise p-coarsening
(k = 3, 4), h-coarsening along some axes only (odd cell counts), walls,
tanh grading, trilinear cells and 2D, and needs far fewer iterations than Jacobi."""
import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh as OMesh
from oracle.trbdf2 import Stepper, solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    (3, (8, 8, 8), (0, 0, 0), (1.0, 1.0, 1.0), (True, True, True), 2, 0, (0, 0, 0)),
    (3, (6, 4, 5), (0, 0, 0), (1.0, 0.7, 0.9), (True, False, True), 3, 0, (0, 0, 0)),
    (3, (4, 8, 4), (0, 0, 0), (2.0, 1.0, 1.0), (True, False, False), 2, 1, (0.0, 1.5, 1.5)),
    (2, (16, 12), (0, 0), (1.0, 1.0), (False, True), 4, 0, (0, 0, 0)),
    # trilinear cells: rediscretised levels on the coarsened vertex lattice
    (3, (8, 6, 4), (0, 0, 0), (1.0, 1.0, 1.0), (False, False, False), 3, 2, (0.03, 0, 0)),
    (2, (12, 8), (0, 0), (1.0, 1.0), (True, True), 2, 2, (0.05, 0, 0)),
]


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("fp32", [True, False])
def test_mg_pcg_matches_direct_solve(ci, fp32):
    from paper_2107_07776_gb300 import binding as b
    dim, n, lo, hi, per, k, mp, prm = CASES[ci]
    gm = b.Mesh(dim, n, lo, hi, per, k, mp, prm)
    om = OMesh(dim, list(n), list(lo), list(hi), list(per), k, map=mp, map_param=list(prm))
    s = b.dg_solver_create(gm.handle, 100.0, 1e3)
    try:
        for alpha in (2.9, 0.05):
            rhs = W.random_vector(om.n_p, 40 + ci)
            x = torch.zeros(om.n_p, dtype=torch.float64, device="cuda")
            pc = b.DG_PC_MG_FP32 if fp32 else b.DG_PC_MG_FP64
            o = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-12, max_iter=200, precond=pc)
            info = b.dg_solve_stage(s, None, alpha, None, torch.tensor(rhs, device="cuda"), x, o)
            ref = solve(Stepper(om, 100.0).helmholtz_matrix(alpha), rhs, spd=True)
            err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
            assert err < 1e-9, (alpha, err, info.iterations)
            assert info.iterations < 40, info.iterations
    finally:
        b.dg_solver_destroy(s)


@pytest.mark.parametrize("fp32", [True, False])
def test_mg_on_levels_larger_than_one_launch_wave(fp32):
    """Q3/Q2 on 32^3 trilinear cells: the finest pressure level (884,736
    DoFs) exceeds one wave of the capped grid-stride launches, so every
    transfer kernel must cover all of its level; MG-FCG converges as on the
    small meshes."""
    from paper_2107_07776_gb300 import binding as b
    w = W.MMS64.scaled((32, 32, 32))
    gm = b.Mesh.from_workload(w)
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        alpha = 1.0 / (w.c ** 2 * (b.GAMMA * w.dt) ** 2)
        rhs = torch.tensor(W.random_vector(gm.n_dofs_p, 5), device="cuda")
        x = torch.zeros_like(rhs)
        pc = b.DG_PC_MG_FP32 if fp32 else b.DG_PC_MG_FP64
        o = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-8, max_iter=60, precond=pc)
        info = b.dg_solve_stage(s, None, alpha, None, rhs, x, o)
        assert info.iterations < 20, info.iterations
    finally:
        b.dg_solver_destroy(s)


def test_mg_beats_jacobi_on_tgv32():
    from paper_2107_07776_gb300 import binding as b
    w = W.TGV32
    gm = b.Mesh.from_workload(w)
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        alpha = 1.0 / (w.c ** 2 * (b.GAMMA * w.dt) ** 2)
        rhs = torch.tensor(W.random_vector(gm.n_dofs_p, 5), device="cuda")
        its = {}
        for pc in (b.DG_PC_JACOBI, b.DG_PC_MG_FP32, b.DG_PC_MG_FP64):
            x = torch.zeros_like(rhs)
            o = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-8, max_iter=5000, precond=pc)
            its[pc] = b.dg_solve_stage(s, None, alpha, None, rhs, x, o).iterations
        assert its[b.DG_PC_MG_FP32] * 5 < its[b.DG_PC_JACOBI], its
        assert abs(its[b.DG_PC_MG_FP32] - its[b.DG_PC_MG_FP64]) <= 2, its
    finally:
        b.dg_solver_destroy(s)
