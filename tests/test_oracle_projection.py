"""Pins of the oracle's comparison projection schemes (Section 2: Bell,
Colella and Glaz; Guermond and Quartapelle's BDF2), against the paper's
Taylor-Green tables (Section 4.1, Q2-Q1, C = 1.63) as a factor-2 band on the
velocity, second order in time on the closed-form flow, and exact
conservation of int p on periodic meshes (the pressure systems keep it:
1^T K = 0 and F_p(1) = 0)."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh
from oracle.projection import ProjectionStepper
from oracle.trbdf2 import Stepper, interpolate, l2_error

HERE = os.path.dirname(__file__)


def gold(name):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", name))
            if l.strip() and not l.startswith("#")]
    return [(float(a), int(b), float(c), float(d)) for a, b, c, d in rows]


def run(scheme, N, dt, T, Re, k=2, fixed_point=0, fp_tol=1e-10):
    m = Mesh(2, [N, N], [0, 0], [2 * math.pi] * 2, [True, True], k)
    st = Stepper(m, Re)
    ps = ProjectionStepper(st, scheme, fixed_point=fixed_point, fixed_point_tol=fp_tol)
    u = interpolate(m, lambda x, y: W.paper_tg_u(x, y, 0.0, Re))
    p = interpolate(m, lambda x, y: W.paper_tg_p(x, y, 0.0, Re), p_space=True)
    up = interpolate(m, lambda x, y: W.paper_tg_u(x, y, -dt, Re))
    pint0 = (st.Mp @ p).sum()
    t = 0.0
    for _ in range(int(round(T / dt))):
        u, p, up = ps.step(u, p, up, t, dt)
        t += dt
    e2 = n2 = 0.0
    for i in range(2):
        ex = lambda x, y, i=i: W.paper_tg_u(x, y, t, Re)[i]
        e2 += l2_error(m, u[i], ex, relative=False) ** 2
        n2 += l2_error(m, 0 * u[i], ex, relative=False) ** 2
    ep = l2_error(m, p, lambda x, y: W.paper_tg_p(x, y, t, Re), p_space=True)
    return math.sqrt(e2 / n2), ep, (st.Mp @ p).sum() - pint0


def test_bcg_paper_table_first_row():
    """8x8, dt 0.64: the fully nonlinear BCG predictor (Picard on the
    midpoint advecting field) lands within a factor 2 of the table's 0.48
    (velocity) and 0.41 (pressure)."""
    dt, N, eu_p, ep_p = gold("tg_q2q1_bcg_paper.txt")[0]
    eu, ep, dp = run("bcg", N, dt, 3.2, 100.0, fixed_point=300)
    assert eu_p / 2 < eu < eu_p * 2, eu
    assert ep_p / 2 < ep < ep_p * 2, ep
    assert abs(dp) < 1e-7


@pytest.mark.parametrize("row", [0, 1])
def test_bdf2_paper_table(row):
    dt, N, eu_p, ep_p = gold("tg_q2q1_gq_paper.txt")[row]
    eu, ep, dp = run("bdf2", N, dt, 3.2, 100.0)
    assert eu_p / 2 < eu < eu_p * 2, eu
    assert ep_p / 3 < ep < ep_p * 3, ep
    assert abs(dp) < 1e-7


@pytest.mark.parametrize("scheme,T", [("bcg", 0.5), ("bdf2", 1.0)])
def test_second_order_in_time(scheme, T):
    """Q4 on 10x10 (space error negligible), Re 10, T = 0.5 or 1: halving dt cuts
    the velocity error about four times (from dt = 0.125: the BDF2 start-up
    step leaves a rate of 1.6 between 0.25 and 0.125)."""
    errs = [run(scheme, 10, dt, T, 10.0, k=4, fixed_point=50, fp_tol=1e-7)[0]
            for dt in (0.125, 0.0625)]
    assert math.log2(errs[0] / errs[1]) > 1.8, errs
