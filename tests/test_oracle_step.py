"""Pins of the oracle's TR-BDF2 projection step (Section 2 of the paper)
against closed forms and the paper's printed convergence table.

 * Taylor-Green exact solution (Section 4.1): second order in time with the
   space error made negligible (Q4), high order in space at small dt;
 * the paper's Table of relative L2 errors (Q2-Q1, C = 1.63) as a sanity band
   (factor 2: the paper leaves quadrature, penalty scale and solver
   tolerances unstated);
 * exact conservation of int p on periodic meshes (1^T K = 0 and F_p(1) = 0).
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh
from oracle.trbdf2 import GAMMA, Stepper, interpolate, l2_error

GOLD = os.path.join(os.path.dirname(__file__), "golden", "tg_q2q1_paper.txt")
GOLD_C3 = os.path.join(os.path.dirname(__file__), "golden", "tg_q2q1_c3_paper.txt")


def run_tg(N, k, dt, T, Re, extrapolate=True, fixed_point=0, its=None):
    m = Mesh(2, [N, N], [0, 0], [2 * math.pi] * 2, [True, True], k)
    st = Stepper(m, Re, extrapolate=extrapolate, fixed_point=fixed_point, fixed_point_tol=1e-6)
    u = interpolate(m, lambda x, y: W.paper_tg_u(x, y, 0.0, Re))
    p = interpolate(m, lambda x, y: W.paper_tg_p(x, y, 0.0, Re), p_space=True)
    uh = interpolate(m, lambda x, y: W.paper_tg_u(x, y, -(1 - GAMMA) * dt, Re))
    t = 0.0
    pint0 = (st.Mp @ p).sum()
    # the C = 3 table's time steps do not divide T: take ceil(T / dt) steps
    nsteps = int(round(T / dt)) if fixed_point == 0 else math.ceil(T / dt - 1e-9)
    for _ in range(nsteps):
        u, p, uh = st.step(u, p, uh, t, dt)
        if its is not None:
            its.append(tuple(st.fixed_point_iterations))
        t += dt
    e2 = n2 = 0.0
    for i in range(2):
        e2 += l2_error(m, u[i], lambda x, y, i=i: W.paper_tg_u(x, y, t, Re)[i], relative=False) ** 2
        n2 += l2_error(m, 0 * u[i], lambda x, y, i=i: W.paper_tg_u(x, y, t, Re)[i],
                       relative=False) ** 2
    ep = l2_error(m, p, lambda x, y: W.paper_tg_p(x, y, t, Re), p_space=True)
    return math.sqrt(e2 / n2), ep, (st.Mp @ p).sum() - pint0


def test_second_order_in_time():
    errs = [run_tg(10, 4, dt, 1.0, 10.0)[0] for dt in (0.25, 0.125)]
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_convergence_under_hyperbolic_scaling():
    """N = 8 -> 16 at the table's C = 1.63 (lagged field): rate above 2, as in
    the paper's table (2.01).  At fixed h and dt -> 0 the error instead grows
    with the number of steps, because the non-incremental pressure form
    (Eq. helmholtz2a in weak form) solves K p^{n+1} against D M^-1 P p^n and
    K differs from D M^-1 P by an O(h^r) term every step."""
    e8 = run_tg(8, 2, 0.64, 3.2, 100.0, extrapolate=False)[0]
    e16 = run_tg(16, 2, 0.32, 3.2, 100.0, extrapolate=False)[0]
    assert math.log2(e8 / e16) > 2.0, (e8, e16)


def _gold():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return [(float(a), int(b), float(c), float(d)) for a, b, c, d in rows]


@pytest.mark.parametrize("row", _gold()[:2])
def test_paper_table_band_lagged(row):
    """At the table's C = 1.63 the extrapolated advecting field diverges (see
    test_extrapolated_field_limit); the lagged one lands in the band."""
    dt, N, eu_paper, ep_paper = row
    eu, ep, dp = run_tg(N, 2, dt, 3.2, 100.0, extrapolate=False)
    assert eu_paper / 2 < eu < eu_paper * 2, eu
    assert ep_paper / 3 < ep < ep_paper * 3, ep
    assert abs(dp) < 1e-7   # roundoff of the RHS amplified by 1/alpha ~ 1e5


@pytest.mark.parametrize("row", _gold()[:2])
def test_paper_table_band_extrapolated_at_quarter_courant(row):
    """The table's errors are space-dominated (its text: the time step does
    not affect second-order accuracy), so at C = 0.41 the extrapolated
    scheme must land in the same band."""
    dt, N, eu_paper, _ = row
    eu, _, dp = run_tg(N, 2, dt / 4, 3.2, 100.0, extrapolate=True)
    assert eu_paper / 2 < eu < eu_paper * 2, eu
    assert abs(dp) < 1e-7   # roundoff of the RHS amplified by 1/alpha ~ 1e5


def test_extrapolated_field_limit():
    """Records the stability limit of the extrapolation readings: at C = 1.63
    on the 8x8 Taylor-Green test the extrapolated advecting field grows."""
    eu, _, _ = run_tg(8, 2, 0.64, 3.2, 100.0, extrapolate=True)
    assert eu > 1.0


def test_tg2d_workload_tracks_exact_decay():
    w = W.TG2D
    m = Mesh(2, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree)
    st = Stepper(m, w.Re, c=w.c)
    nu = 1.0 / w.Re
    u = interpolate(m, lambda x, y: W.tg2d_u(x, y, 0.0, nu))
    p = interpolate(m, lambda x, y: W.tg2d_p(x, y, 0.0, nu), p_space=True)
    uh = interpolate(m, lambda x, y: W.tg2d_u(x, y, -(1 - GAMMA) * w.dt, nu))
    t = 0.0
    for _ in range(w.steps):
        u, p, uh = st.step(u, p, uh, t, w.dt)
        t += w.dt
    err = max(l2_error(m, u[i], lambda x, y, i=i: W.tg2d_u(x, y, t, nu)[i]) for i in range(2))
    assert err < 0.05


# ---- fully nonlinear momentum stages (fixed point iterations, Section 2) ----
def _gold_c3():
    rows = [l.split() for l in open(GOLD_C3) if l.strip() and not l.startswith("#")]
    return [(float(a), int(b), float(c), float(d)) for a, b, c, d in rows]


@pytest.mark.parametrize("row", [_gold_c3()[0], pytest.param(_gold_c3()[1], marks=pytest.mark.slow)])
def test_fixed_point_stages_paper_table_c3(row):
    """At C = 3 the paper iterates the momentum predictors to a fixed point
    (the implicit advecting field is the unknown itself); the oracle's
    fully nonlinear stages land in the band of the paper's table."""
    dt, N, eu_paper, ep_paper = row
    its = []
    eu, ep, dp = run_tg(N, 2, dt, 3.2, 100.0, extrapolate=False, fixed_point=200, its=its)
    assert eu_paper / 2 < eu < eu_paper * 2, eu
    assert ep_paper / 3 < ep < ep_paper * 3, ep
    assert abs(dp) < 1e-7
    assert all(i < 200 for st in its for i in st), its   # converged before the cap


def test_fully_nonlinear_form_is_more_accurate_at_c3():
    """The paper's remark on larger Courant numbers: at C = 3 the fixed-point
    form is more accurate than both linearised advecting fields."""
    dt, N = 1.18, 8
    e_fp = run_tg(N, 2, dt, 3.2, 100.0, extrapolate=False, fixed_point=200)[0]
    e_lag = run_tg(N, 2, dt, 3.54, 100.0, extrapolate=False)[0]
    e_ext = run_tg(N, 2, dt, 3.54, 100.0, extrapolate=True)[0]
    assert e_fp < e_lag and e_fp < e_ext, (e_fp, e_lag, e_ext)


def test_fixed_point_of_a_steady_field_is_reached_at_once():
    """A field with no advection (u = 0, p = 0) is its own fixed point: the
    second iterate does not change, so the iteration stops after two solves."""
    m = Mesh(2, [4, 4], [0, 0], [2 * math.pi] * 2, [True, True], 2)
    st = Stepper(m, 100.0, extrapolate=False, fixed_point=50, fixed_point_tol=1e-12)
    u = np.zeros((2, m.n_u))
    p = np.zeros(m.n_p)
    u1, p1, _ = st.step(u, p, u.copy(), 0.0, 0.1)
    assert np.abs(u1).max() == 0.0 and np.abs(p1).max() == 0.0
    assert st.fixed_point_iterations == [2, 2]


# ------------------------------------------------------ impermeable walls
def test_wall_normal_trace_of_polynomial_data():
    """Traces of a nodal field at the walls: u_y = y + 2 and u_z = 3 z - 1 on
    [0,2]x[0,1]x[0,1.5] (x periodic) are exact in Q2, so the largest normal
    trace is max(|2|, |3|, |-1|, |3.5|) = 3.5 (u_y at y = 1 is 3, u_z at
    z = 1.5 is 3.5)."""
    from oracle.trbdf2 import wall_normal_trace
    m = Mesh(3, [2, 3, 2], [0, 0, 0], [2.0, 1.0, 1.5], [True, False, False], 2)
    x, y, z = m.node_coords()
    uD = np.stack([10.0 + 0 * x, y + 2.0, 3.0 * z - 1.0])
    assert abs(wall_normal_trace(m, uD) - 3.5) < 1e-12
    # the x component is tangential to every wall of this mesh
    uD[1] = y * (1 - y)
    uD[2] = z * (1.5 - z)
    assert wall_normal_trace(m, uD) < 1e-13


def test_stepper_refuses_data_with_a_normal_component():
    """The boundary Lax-Friedrichs speed is |ubar+ . n|, the mirror state's
    max(|ubar+ . n|, |(2 u_D - ubar+) . n|) when u_D . n = 0: data with a
    normal component is refused, tangential data is accepted."""
    m = Mesh(2, [2, 2], [0, 0], [1.0, 1.0], [True, False], 2)
    st = Stepper(m, 10.0, c=10.0)
    x, y = m.node_coords()
    u = np.zeros((2, m.n_u))
    p = np.zeros(m.n_p)
    with pytest.raises(ValueError):
        st.step(u, p, u, 0.0, 0.01, uD=lambda t: np.stack([0 * x, 0.1 + 0 * y]))
    un, _, _ = st.step(u, p, u, 0.0, 0.01, uD=lambda t: np.stack([0.1 + 0 * x, y * (1 - y)]))
    assert np.abs(un).max() > 0.0
