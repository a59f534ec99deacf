"""The 3D Arnold-Beltrami-Childress workload on the GPU (Section 4.1, Eq.
abc; Re = 1, periodic cube): full TR-BDF2 steps against the oracle on
reduced meshes (Q2 and Q3), the study's error measure against the oracle's,
and the paper's hyperbolic-scaling table (Q2/Q1, C = 1.63) as a band."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh as OMesh
from oracle.trbdf2 import GAMMA, Stepper, interpolate, l2_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("N,k,dt", [(4, 2, 0.32), (3, 3, 0.21)])
def test_abc_steps_match_oracle(N, k, dt):
    from paper_2107_07776_gb300 import binding as b
    from paper_2107_07776_gb300.abcstudy import nodal_errors
    w = W.ABC.scaled((N, N, N), degree=k, dt=dt)
    gm = b.Mesh.from_workload(w)
    om = OMesh(3, [N] * 3, list(w.lo), list(w.hi), [True] * 3, k)
    X, Xp = om.node_coords(), om.node_coords(True)
    ou, op = W.abc_u(*X, 0.0, w.Re), W.abc_p(*Xp, 0.0, w.Re)
    ouh = W.abc_u(*X, -(1 - GAMMA) * dt, w.Re)
    st = Stepper(om, w.Re, c=w.c, direct_max=0)
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        u, p = dev(ou.reshape(-1)), dev(op)
        b.dg_solver_set_history(s, dev(ouh.reshape(-1)))
        prm = b.dg_step_params()
        prm.dt, prm.gamma, prm.extrapolate = dt, 0.0, 1
        prm.mom = b.solve_opts(b.DG_SYS_MOMENTUM, tol=1e-13, max_iter=20000, restart=30,
                               precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_EXTRAP)
        prm.helm = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-13, max_iter=5000,
                                precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_EXTRAP)
        t = 0.0
        for n in range(3):
            info = b.trbdf2_step(s, prm, u, p)
            assert all(i.status == 0 for i in info)
            ou, op, ouh = st.step(ou, op, ouh, t, dt)
            t += dt
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, n
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, n
        # the study's error measure against the oracle's: both a
        # (k+3)-point Gauss rule per direction
        eu, ep, _ = nodal_errors(w, gm, u.cpu().numpy(), p.cpu().numpy(), t)
        e2 = n2 = 0.0
        for i in range(3):
            ex = lambda x, y, z, i=i: W.abc_u(x, y, z, t, w.Re)[i]
            e2 += l2_error(om, ou[i], ex, relative=False) ** 2
            n2 += l2_error(om, 0 * ou[i], ex, relative=False) ** 2
        assert abs(eu / math.sqrt(e2 / n2) - 1) < 1e-6, (eu, math.sqrt(e2 / n2))
        eo = l2_error(om, op, lambda x, y, z: W.abc_p(x, y, z, t, w.Re), p_space=True)
        assert abs(ep / eo - 1) < 1e-6, (ep, eo)
    finally:
        b.dg_solver_destroy(s)


def test_abc_paper_table_hyperbolic_band():
    """Section 4.1's ABC table (Q2/Q1, C = 1.63, T = 3.2): relative L2 errors
    of u 0.0078 (8^3, dt 0.32) and 0.0022 (16^3, dt 0.16), H1 0.019 and
    0.0054.  The paper leaves solver tolerances, quadrature and penalty
    scale unstated, so the check is a band (factor 3) and a convergence rate
    near 2."""
    from paper_2107_07776_gb300.abcstudy import run_row
    r8 = run_row(8, 2, 0.32)
    r16 = run_row(16, 2, 0.16)
    for r, l2, h1 in ((r8, 0.0078, 0.019), (r16, 0.0022, 0.0054)):
        assert l2 / 3 < r["l2_u"] < l2 * 3, r
        assert h1 / 3 < r["h1_u"] < h1 * 3, r
    rate = math.log2(r8["l2_u"] / r16["l2_u"])
    assert 1.4 < rate < 2.8, (r8, r16)
