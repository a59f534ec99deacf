"""The comparison projection schemes of Section 2 (Bell-Colella-Glaz and
Guermond-Quartapelle BDF2) on the GPU (dg_projection_step) against the
oracle's ProjectionStepper: step by step at 1e-8 relative L2 with both sides
solving to 1e-13, on the 2D Taylor-Green table's first mesh (C = 1.63, the
fully nonlinear BCG predictor) and on a walled, graded 3D mesh with
tangential wall data and forcing; plus the paper's tables as a band."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh as OMesh
from oracle.projection import ProjectionStepper
from oracle.trbdf2 import Stepper, interpolate, l2_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def params(b, scheme, dt, fixed_point=0, fields=None):
    prm = b.dg_projection_params()
    prm.scheme, prm.dt = scheme, dt
    prm.mom = b.solve_opts(b.DG_SYS_MOMENTUM, tol=1e-13, max_iter=5000, restart=30,
                           precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_GIVEN)
    prm.helm = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-13, max_iter=5000,
                            precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_GIVEN)
    prm.fixed_point, prm.fixed_point_tol = fixed_point, 1e-10
    for k, v in (fields or {}).items():
        setattr(prm, k, v.data_ptr() if v is not None else None)
    return prm


@pytest.mark.parametrize("scheme", ["bcg", "bdf2"])
def test_taylor_green_table_mesh_matches_oracle(scheme):
    from paper_2107_07776_gb300 import binding as b
    N, dt, Re = 8, 0.64, 100.0
    om = OMesh(2, [N, N], [0, 0], [2 * math.pi] * 2, [True, True], 2)
    gm = b.Mesh(2, (N, N), (0, 0), (2 * math.pi, 2 * math.pi), (True, True), 2)
    fp = 300 if scheme == "bcg" else 0
    ps = ProjectionStepper(Stepper(om, Re), scheme, fixed_point=fp, fixed_point_tol=1e-10)
    ou = interpolate(om, lambda x, y: W.paper_tg_u(x, y, 0.0, Re))
    op = interpolate(om, lambda x, y: W.paper_tg_p(x, y, 0.0, Re), p_space=True)
    oup = interpolate(om, lambda x, y: W.paper_tg_u(x, y, -dt, Re))
    code = b.DG_SCHEME_BCG if scheme == "bcg" else b.DG_SCHEME_BDF2
    s = b.dg_solver_create(gm.handle, Re, 1e3)
    try:
        u, p = dev(ou.reshape(-1)), dev(op)
        b.dg_solver_set_history(s, dev(oup.reshape(-1)))
        t = 0.0
        for n in range(5):
            info = b.dg_projection_step(s, params(b, code, dt, fp), u, p)
            assert all(i.status == 0 for i in info)
            ou, op, oup = ps.step(ou, op, oup, t, dt)
            t += dt
            if scheme == "bcg":
                assert abs(b.dg_solver_get_fixed_point(s)[0] - ps.fixed_point_iterations) <= 1
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, n
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, n
        # Section 4.1's table, first row: 0.48 (BCG) and 0.28 (BDF2), factor 2
        ug = u.cpu().numpy().reshape(2, -1)
        e2 = n2 = 0.0
        for i in range(2):
            ex = lambda x, y, i=i: W.paper_tg_u(x, y, t, Re)[i]
            e2 += l2_error(om, ug[i], ex, relative=False) ** 2
            n2 += l2_error(om, 0 * ug[i], ex, relative=False) ** 2
        paper = 0.48 if scheme == "bcg" else 0.28
        assert paper / 2 < math.sqrt(e2 / n2) < paper * 2
    finally:
        b.dg_solver_destroy(s)


@pytest.mark.parametrize("scheme,fp", [("bcg", 0), ("bcg", 40), ("bdf2", 0)])
def test_walled_graded_mesh_with_data_and_forcing(scheme, fp):
    from paper_2107_07776_gb300 import binding as b
    n, lo, hi, per = (3, 4, 3), (0, 0, 0), (2.0, 1.0, 1.0), (True, False, False)
    gm = b.Mesh(3, n, lo, hi, per, 2, 1, (0.0, 1.5, 1.5))
    om = OMesh(3, list(n), list(lo), list(hi), list(per), 2, map=1, map_param=[0.0, 1.5, 1.5])
    X = om.node_coords()
    uD = lambda t: np.stack([np.sin(X[1] + t) * (1 + X[2]),
                             0.3 * X[1] * (1 - X[1]) * (1 + 0.5 * X[0]) * (1 + t),
                             0.1 * X[2] * (1 - X[2]) * (1 + X[1]) * (1 + t)])
    f = lambda t: (1 + t) * W.mms_forcing(*X)
    rng = np.random.default_rng(5)
    ou = rng.standard_normal((3, om.n_u)) * 0.1
    op = rng.standard_normal(om.n_p) * 0.1
    oup = ou + 0.01 * rng.standard_normal((3, om.n_u))
    ps = ProjectionStepper(Stepper(om, 50.0, c=30.0), scheme, fixed_point=fp,
                           fixed_point_tol=1e-10)
    code = b.DG_SCHEME_BCG if scheme == "bcg" else b.DG_SCHEME_BDF2
    s = b.dg_solver_create(gm.handle, 50.0, 30.0)
    dt = 0.02
    try:
        u, p = dev(ou.reshape(-1)), dev(op)
        b.dg_solver_set_history(s, dev(oup.reshape(-1)))
        t = 0.0
        for k in range(3):
            fld = dict(uD=dev(uD(t + dt).reshape(-1)), f_n=dev(f(t).reshape(-1)),
                       f_n1=dev(f(t + dt).reshape(-1)))
            b.dg_projection_step(s, params(b, code, dt, fp, fld), u, p)
            ou, op, oup = ps.step(ou, op, oup, t, dt, uD=uD, f=f)
            t += dt
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, k
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, k
    finally:
        b.dg_solver_destroy(s)
