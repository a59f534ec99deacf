"""Stage solves and full TR-BDF2 steps on the GPU against the oracle
(Sections 2-3), plus host-side failure injection and checkpoint/resume.

Both sides solve to a relative residual of 1e-13 here, so the step-by-step
difference is bounded by the conditioning times that residual; the bound
used, 1e-8 relative L2, is the tolerance stated for full steps."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh as OMesh
from oracle.trbdf2 import GAMMA, Stepper, interpolate

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def opts(b, system, tol=1e-13, precond=None, guess=None, max_iter=5000):
    if precond is None:
        precond = b.DG_PC_JACOBI
    return b.solve_opts(system, tol=tol, max_iter=max_iter, restart=30, precond=precond,
                        guess=b.DG_GUESS_ZERO if guess is None else guess)


@pytest.mark.parametrize("walls", [False, True])
def test_stage_solves_match_direct_solve(walls):
    from paper_2107_07776_gb300 import binding as b
    per = (True, not walls, not walls)
    gm = b.Mesh(3, (4, 3, 5), (0, 0, 0), (1, 1, 1), per, 2)
    om = OMesh(3, [4, 3, 5], [0, 0, 0], [1, 1, 1], list(per), 2)
    s = b.dg_solver_create(gm.handle, 100.0, 1e3)
    try:
        ub = W.random_vector(3 * om.n_u, 5)
        rhs = W.random_vector(3 * om.n_u, 6)
        co = b.momentum_coeffs(1.0 / (GAMMA * 0.01), 1.0 / 200, 0.5)
        x = torch.zeros(3 * om.n_u, dtype=torch.float64, device="cuda")
        info = b.dg_solve_stage(s, co, 0.0, dev(ub), dev(rhs), x, opts(b, b.DG_SYS_MOMENTUM))
        assert info.res_final <= 1e-13 * np.linalg.norm(rhs) * 1.01
        st = Stepper(om, 100.0)
        from oracle.trbdf2 import MomentumCoeffs
        A = st.momentum_matrix(MomentumCoeffs(co.mass, co.visc, co.adv), ub.reshape(3, -1))
        ref = st.solve_momentum(A, rhs.reshape(3, -1)).reshape(-1)
        assert rel_l2(x.cpu().numpy(), ref) < 1e-10
        # Helmholtz, Jacobi-preconditioned CG
        rp = W.random_vector(om.n_p, 7)
        xp = torch.zeros(om.n_p, dtype=torch.float64, device="cuda")
        info = b.dg_solve_stage(s, None, 2.9, None, dev(rp), xp, opts(b, b.DG_SYS_HELMHOLTZ))
        assert info.iterations > 1
        from oracle.trbdf2 import solve
        refp = solve(st.helmholtz_matrix(2.9), rp, spd=True)
        assert rel_l2(xp.cpu().numpy(), refp) < 1e-9
    finally:
        b.dg_solver_destroy(s)


def step_params(b, dt, fields=None, extrapolate=1, tol=1e-13):
    prm = b.dg_step_params()
    prm.dt, prm.gamma, prm.extrapolate = dt, 0.0, extrapolate
    prm.mom = opts(b, b.DG_SYS_MOMENTUM, tol=tol, guess=b.DG_GUESS_EXTRAP)
    prm.helm = opts(b, b.DG_SYS_HELMHOLTZ, tol=tol, guess=b.DG_GUESS_EXTRAP)
    if fields:
        for k, v in fields.items():
            setattr(prm, k, v.data_ptr() if v is not None else None)
    return prm


def test_tg2d_workload_steps_match_oracle():
    """The 2D Taylor-Green workload: 10 steps, every step compared."""
    from paper_2107_07776_gb300 import binding as b
    w = W.TG2D
    gm = b.Mesh.from_workload(w)
    om = OMesh(2, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree)
    nu = 1.0 / w.Re
    u0 = interpolate(om, lambda x, y: W.tg2d_u(x, y, 0.0, nu))
    p0 = interpolate(om, lambda x, y: W.tg2d_p(x, y, 0.0, nu), p_space=True)
    uh0 = interpolate(om, lambda x, y: W.tg2d_u(x, y, -(1 - GAMMA) * w.dt, nu))
    st = Stepper(om, w.Re, c=w.c)
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        u, p = dev(u0.reshape(-1)), dev(p0)
        b.dg_solver_set_history(s, dev(uh0.reshape(-1)))
        ou, op, ouh = u0, p0, uh0
        for n in range(w.steps):
            info = b.trbdf2_step(s, step_params(b, w.dt), u, p)
            assert all(i.status == 0 for i in info)
            ou, op, ouh = st.step(ou, op, ouh, n * w.dt, w.dt)
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, n
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, n
    finally:
        b.dg_solver_destroy(s)


@pytest.mark.parametrize("tuning", ["autotune", 6, 7])
def test_periodic_3d_taylor_green_benchmark_path_matches_oracle(tuning):
    """The benchmark's solver path on the 3D periodic Taylor-Green vortex
    (Section 4.1's Taylor-Green case; 32^3 in the benchmark, 4^3 here):
    Q2/Q1, an autotuned (or face-once / Q1 tensor-product) mesh, the
    FP32 multigrid Helmholtz preconditioner and the learned initial guess
    (training on, both nets), 6 steps each compared with the oracle.  Both
    sides solve to 1e-13, so the mixed-precision preconditioner and the
    guess change the path, not the answer (1e-8 relative L2)."""
    from paper_2107_07776_gb300 import binding as b
    w = W.TGV32.scaled((4, 4, 4), Re=400.0, dt=0.02)
    gm = b.Mesh.from_workload(w)
    if tuning == "autotune":
        b.dg_autotune(gm.handle)
    else:
        b.dg_mesh_set_variant(gm.handle, tuning)
    om = OMesh(3, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree)
    X, Xp = om.node_coords(), om.node_coords(True)
    u0, p0 = W.initial_state(w, X, Xp)
    st = Stepper(om, w.Re, c=w.c)
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        b.dg_guess_configure(s, enable=1, train=1, systems=3)
        u, p = dev(u0.reshape(-1)), dev(p0)
        ou, op, ouh = u0, p0, u0
        prm = step_params(b, w.dt)
        prm.mom = opts(b, b.DG_SYS_MOMENTUM, guess=b.DG_GUESS_LEARNED)
        prm.helm = opts(b, b.DG_SYS_HELMHOLTZ, precond=b.DG_PC_MG_FP32,
                        guess=b.DG_GUESS_LEARNED)
        for n in range(6):
            info = b.trbdf2_step(s, prm, u, p)
            assert all(i.status == 0 for i in info)
            ou, op, ouh = st.step(ou, op, ouh, n * w.dt, w.dt)
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, n
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, n
        assert b.dg_guess_get_stats(s).train_steps > 0
    finally:
        b.dg_solver_destroy(s)


def test_fully_nonlinear_stages_match_oracle_at_c3():
    """Section 2's fully nonlinear momentum stages (Picard iterations on the
    implicit advecting field), which the paper needs at larger Courant
    numbers: the 8x8 Q2/Q1 Taylor-Green vortex at C = 3 (dt = 1.18, the
    first row of Section 4.1's C = 3 table; ceil(3.2/dt) = 3 steps), lagged
    starting fields, Picard to a relative change of 1e-10 on both sides.
    Every step matches the oracle at 1e-8, the Picard counts agree (to one
    iteration at the stopping threshold), and the final velocity error lies
    in the table's band (factor 2 of 0.39)."""
    from paper_2107_07776_gb300 import binding as b
    from oracle.trbdf2 import l2_error
    N, dt, Re = 8, 1.18, 100.0
    om = OMesh(2, [N, N], [0, 0], [2 * math.pi] * 2, [True, True], 2)
    gm = b.Mesh(2, (N, N), (0, 0), (2 * math.pi, 2 * math.pi), (True, True), 2)
    st = Stepper(om, Re, extrapolate=False, fixed_point=400, fixed_point_tol=1e-10)
    ou = interpolate(om, lambda x, y: W.paper_tg_u(x, y, 0.0, Re))
    op = interpolate(om, lambda x, y: W.paper_tg_p(x, y, 0.0, Re), p_space=True)
    ouh = ou
    s = b.dg_solver_create(gm.handle, Re, 1e3)
    try:
        u, p = dev(ou.reshape(-1)), dev(op)
        prm = step_params(b, dt, extrapolate=0)
        prm.fixed_point, prm.fixed_point_tol = 400, 1e-10
        t = 0.0
        for n in range(3):
            info = b.trbdf2_step(s, prm, u, p)
            assert all(i.status == 0 for i in info)
            ou, op, ouh = st.step(ou, op, ouh, t, dt)
            t += dt
            its = b.dg_solver_get_fixed_point(s)
            assert all(abs(a - c) <= 1 for a, c in zip(its, st.fixed_point_iterations)), \
                (its, st.fixed_point_iterations)
            assert min(its) > 2
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, n
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, n
        ug = u.cpu().numpy().reshape(2, -1)
        e2 = n2 = 0.0
        for i in range(2):
            ex = lambda x, y, i=i: W.paper_tg_u(x, y, t, Re)[i]
            e2 += l2_error(om, ug[i], ex, relative=False) ** 2
            n2 += l2_error(om, 0 * ug[i], ex, relative=False) ** 2
        assert 0.39 / 2 < math.sqrt(e2 / n2) < 0.39 * 2
    finally:
        b.dg_solver_destroy(s)


def test_fixed_point_option_is_validated():
    from paper_2107_07776_gb300 import binding as b
    gm = b.Mesh(2, (4, 4), (0, 0), (1.0, 1.0), (True, True), 2)
    s = b.dg_solver_create(gm.handle, 10.0, 1e3)
    try:
        u = torch.zeros(gm.n_dofs_u, dtype=torch.float64, device="cuda")
        p = torch.zeros(gm.n_dofs_p, dtype=torch.float64, device="cuda")
        prm = step_params(b, 0.1)
        prm.fixed_point, prm.fixed_point_tol = 5, 0.0
        with pytest.raises(b.DGError):
            b.trbdf2_step(s, prm, u, p)
    finally:
        b.dg_solver_destroy(s)


def test_step_waits_for_inputs_filled_on_the_callers_stream():
    """u, p and the history are filled on a non-blocking torch stream behind
    a ~25 ms spin, and the solver is told that stream (dg_solver_set_stream):
    its calls must wait for those copies, and the first two steps still
    match the oracle."""
    from paper_2107_07776_gb300 import binding as b
    w = W.TG2D
    gm = b.Mesh.from_workload(w)
    om = OMesh(2, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree)
    nu = 1.0 / w.Re
    u0 = interpolate(om, lambda x, y: W.tg2d_u(x, y, 0.0, nu)).reshape(-1)
    p0 = interpolate(om, lambda x, y: W.tg2d_p(x, y, 0.0, nu), p_space=True)
    uh0 = interpolate(om, lambda x, y: W.tg2d_u(x, y, -(1 - GAMMA) * w.dt, nu)).reshape(-1)
    hosts = [torch.tensor(v).pin_memory() for v in (u0, p0, uh0)]
    u, p, uh = (torch.full(h.shape, float("nan"), dtype=torch.float64, device="cuda")
                for h in hosts)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        b.dg_solver_set_stream(s, side)
        with torch.cuda.stream(side):
            torch.cuda._sleep(50_000_000)
            for d, h in zip((u, p, uh), hosts):
                d.copy_(h, non_blocking=True)
        b.dg_solver_set_history(s, uh)
        st = Stepper(om, w.Re, c=w.c)
        ou, op, ouh = u0.reshape(2, -1), p0, uh0.reshape(2, -1)
        for n in range(2):
            b.trbdf2_step(s, step_params(b, w.dt), u, p)
            ou, op, ouh = st.step(ou, op, ouh, n * w.dt, w.dt)
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, n
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, n
    finally:
        b.dg_solver_destroy(s)


@pytest.mark.parametrize("geom", ["graded", "trilinear"])
@pytest.mark.parametrize("extrapolate", [1, 0])
def test_walled_step_with_data_and_forcing_matches_oracle(extrapolate, geom):
    """3D, periodic in x, Dirichlet walls in y and z with time-dependent
    tangential wall data and forcing, on a tanh-graded mesh (Q2) or on sine-perturbed
    trilinear cells (Q3): 3 steps compared."""
    from paper_2107_07776_gb300 import binding as b
    n, lo, hi, per = (3, 4, 3), (0, 0, 0), (2.0, 1.0, 1.0), (True, False, False)
    k, mp, prm = (2, 1, [0.0, 1.5, 1.5]) if geom == "graded" else (3, 2, [0.03, 0.0, 0.0])
    gm = b.Mesh(3, n, lo, hi, per, k, mp, tuple(prm))
    om = OMesh(3, list(n), list(lo), list(hi), list(per), k, map=mp, map_param=prm)
    X = om.node_coords()
    # impermeable walls (u_D . n = 0): u_y vanishes on the y walls and u_z on
    # the z walls, and both traces are exact in the nodal space (degree <= 2
    # per reference direction on either mapping), while the tangential
    # components vary along the walls
    uD = lambda t: np.stack([np.sin(X[1] + t) * (1 + X[2]),
                             0.3 * X[1] * (1 - X[1]) * (1 + 0.5 * X[0]) * (1 + t),
                             0.1 * X[2] * (1 - X[2]) * (1 + X[1]) * (1 + t)])
    f = lambda t: (1 + t) * W.mms_forcing(*X)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((3, om.n_u)) * 0.1
    p0 = rng.standard_normal(om.n_p) * 0.1
    st = Stepper(om, 50.0, c=30.0, extrapolate=bool(extrapolate))
    s = b.dg_solver_create(gm.handle, 50.0, 30.0)
    dt = 0.02
    try:
        u, p = dev(u0.reshape(-1)), dev(p0)
        ou, op, ouh = u0, p0, u0
        for k in range(3):
            t = k * dt
            fld = dict(uD_stage1=dev(uD(t + GAMMA * dt).reshape(-1)),
                       uD_stage2=dev(uD(t + dt).reshape(-1)), f_n=dev(f(t).reshape(-1)),
                       f_ng=dev(f(t + GAMMA * dt).reshape(-1)), f_n1=dev(f(t + dt).reshape(-1)))
            b.trbdf2_step(s, step_params(b, dt, fld, extrapolate), u, p)
            ou, op, ouh = st.step(ou, op, ouh, t, dt, uD=uD, f=f)
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, k
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, k
    finally:
        b.dg_solver_destroy(s)


@pytest.mark.parametrize("precond", ["jacobi", "mg_fp32"])
def test_trilinear_forced_workload_reduced_matches_oracle(precond):
    """The manufactured-forcing workload on sine-perturbed trilinear Q3/Q2
    cells with no-slip walls, reduced to 4^3 cells: from rest, constant
    seeded forcing, 3 steps compared with the oracle.  The Helmholtz solves
    use Jacobi or the FP32 multigrid (mixed precision) at the same 1e-13
    tolerance: the preconditioner changes the path, not the solution."""
    from paper_2107_07776_gb300 import binding as b
    w = W.MMS64.scaled((4, 4, 4))
    gm = b.Mesh.from_workload(w)
    om = OMesh(3, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree, map=w.map,
               map_param=list(w.map_param))
    X = om.node_coords()
    fh = W.forcing(w, X)
    st = Stepper(om, w.Re, c=w.c)
    s = b.dg_solver_create(gm.handle, w.Re, w.c)
    try:
        u = torch.zeros(3 * om.n_u, dtype=torch.float64, device="cuda")
        p = torch.zeros(om.n_p, dtype=torch.float64, device="cuda")
        fd = dev(fh.reshape(-1))
        ou, op = np.zeros((3, om.n_u)), np.zeros(om.n_p)
        ouh = ou
        prm = step_params(b, w.dt, dict(f_n=fd, f_ng=fd, f_n1=fd))
        if precond == "mg_fp32":
            prm.helm = opts(b, b.DG_SYS_HELMHOLTZ, precond=b.DG_PC_MG_FP32, guess=b.DG_GUESS_EXTRAP)
        for k in range(3):
            info = b.trbdf2_step(s, prm, u, p)
            assert all(i.status == 0 for i in info)
            ou, op, ouh = st.step(ou, op, ouh, k * w.dt, w.dt, f=lambda t: fh)
            assert rel_l2(u.cpu().numpy(), ou.reshape(-1)) < 1e-8, k
            assert rel_l2(p.cpu().numpy(), op) < 1e-8, k
    finally:
        b.dg_solver_destroy(s)


def test_trilinear_workload_mixed_precision_error_vs_fp64():
    """The trilinear workload at 16^3 Q3/Q2 (1.6 M DoFs), 5 steps at the
    benchmark tolerance (1e-8 relative residual): FP32 multigrid + learned
    guess (trained on the first steps) against the plain FP64 solver (FP64
    multigrid, extrapolated guess).  Both stop at the same residual, so the
    difference is of the order of the tolerance times the conditioning."""
    from paper_2107_07776_gb300 import binding as b
    w = W.MMS64.scaled((16, 16, 16))
    gm = b.Mesh.from_workload(w)
    X = gm.node_coords(0).cpu().numpy()
    fd = dev(W.forcing(w, X).reshape(-1))
    res = {}
    for name, pc, guess in (("plain", b.DG_PC_MG_FP64, b.DG_GUESS_EXTRAP),
                            ("mixed", b.DG_PC_MG_FP32, b.DG_GUESS_LEARNED)):
        s = b.dg_solver_create(gm.handle, w.Re, w.c)
        try:
            if guess == b.DG_GUESS_LEARNED:
                b.dg_guess_configure(s, enable=1, train=1, systems=1)
            u = torch.zeros(gm.n_dofs_u, dtype=torch.float64, device="cuda")
            p = torch.zeros(gm.n_dofs_p, dtype=torch.float64, device="cuda")
            prm = step_params(b, w.dt, dict(f_n=fd, f_ng=fd, f_n1=fd), tol=1e-8)
            prm.helm = opts(b, b.DG_SYS_HELMHOLTZ, tol=1e-8, precond=pc, guess=guess)
            for _ in range(5):
                info = b.trbdf2_step(s, prm, u, p)
                assert all(i.status == 0 for i in info)
            res[name] = (u.cpu().numpy(), p.cpu().numpy())
        finally:
            b.dg_solver_destroy(s)
    eu = rel_l2(res["mixed"][0], res["plain"][0])
    ep = rel_l2(res["mixed"][1], res["plain"][1])
    assert eu < 1e-6 and ep < 1e-5, (eu, ep)


def test_failures_are_reported_from_the_host():
    """Failure injection without any GPU fault: max_iter = 1 (no
    convergence), a NaN planted in the right-hand side on the host, bad
    options, and an exhausted wall-clock limit."""
    from paper_2107_07776_gb300 import binding as b
    gm = b.Mesh(3, (4, 4, 4), (0, 0, 0), (1, 1, 1), (True,) * 3, 2)
    s = b.dg_solver_create(gm.handle, 100.0, 1e3)
    try:
        rp = torch.tensor(W.random_vector(gm.n_dofs_p, 1), device="cuda")
        xp = torch.zeros_like(rp)
        o = opts(b, b.DG_SYS_HELMHOLTZ, tol=1e-12, max_iter=1)
        info = b.dg_solve_stage(s, None, 2.9, None, rp, xp, o, raise_on_error=False)
        assert info.status == b.DG_ENOCONV and info.iterations == 1
        assert info.res_final < info.res0              # best iterate returned
        bad = rp.clone()
        bad[17] = float("nan")
        info = b.dg_solve_stage(s, None, 2.9, None, bad, xp, opts(b, b.DG_SYS_HELMHOLTZ),
                                raise_on_error=False)
        assert info.status == b.DG_EBREAKDOWN
        o = opts(b, b.DG_SYS_HELMHOLTZ)
        o.tol_rel = -1.0
        info = b.dg_solve_stage(s, None, 2.9, None, rp, xp, o, raise_on_error=False)
        assert info.status == b.DG_EINVAL
        o = opts(b, b.DG_SYS_HELMHOLTZ, tol=1e-14, precond=b.DG_PC_NONE)
        o.timeout_s = 1e-9
        info = b.dg_solve_stage(s, None, 2.9, None, rp, xp, o, raise_on_error=False)
        assert info.status == b.DG_ETIMEOUT
        ru = torch.tensor(W.random_vector(gm.n_dofs_u, 2), device="cuda")
        xu = torch.zeros_like(ru)
        ub = torch.zeros_like(ru)
        o = opts(b, b.DG_SYS_MOMENTUM, tol=1e-14, max_iter=1)
        info = b.dg_solve_stage(s, b.momentum_coeffs(1.0, 1.0, 0.5), 0.0, ub, ru, xu, o,
                                raise_on_error=False)
        assert info.status == b.DG_ENOCONV
        # the library still works after every failure
        info = b.dg_solve_stage(s, None, 2.9, None, rp, xp, opts(b, b.DG_SYS_HELMHOLTZ, tol=1e-10))
        assert info.status == 0
    finally:
        b.dg_solver_destroy(s)


def test_checkpoint_resume_is_bitwise(tmp_path):
    from paper_2107_07776_gb300 import binding as b
    w = W.TG2D
    gm = b.Mesh.from_workload(w)
    X = gm.node_coords(0).cpu().numpy()
    Xp = gm.node_coords(1).cpu().numpy()
    u0 = dev(W.tg2d_u(*X, 0.0, 0.01).reshape(-1))
    p0 = dev(W.tg2d_p(*Xp, 0.0, 0.01))
    prm = step_params(b, w.dt, tol=1e-10)

    def run(nsteps, u, p, s):
        for _ in range(nsteps):
            b.trbdf2_step(s, prm, u, p)

    s1 = b.dg_solver_create(gm.handle, w.Re, w.c)
    ua, pa = u0.clone(), p0.clone()
    run(4, ua, pa, s1)
    s2 = b.dg_solver_create(gm.handle, w.Re, w.c)
    ub_, pb = u0.clone(), p0.clone()
    run(2, ub_, pb, s2)
    path = str(tmp_path / "ck.bin")
    b.dg_solver_save(s2, path)
    b.dg_solver_destroy(s2)
    s3 = b.dg_solver_create(gm.handle, w.Re, w.c)
    b.dg_solver_load(s3, path)
    run(2, ub_, pb, s3)
    assert torch.equal(ua, ub_) and torch.equal(pa, pb)
    for s in (s1, s3):
        b.dg_solver_destroy(s)
