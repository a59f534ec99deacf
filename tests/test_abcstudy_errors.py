"""The ABC study's error measure (relative L2 of u and p, relative H1 of u
by a (k+3)-point Gauss rule on the uniform periodic mesh) equals the
oracle's on the same perturbed fields (no GPU needed: the measure works on
host arrays)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh
from oracle.trbdf2 import l2_error


@pytest.mark.parametrize("N,k", [(3, 3), (4, 2)])
def test_study_errors_equal_the_oracles(N, k):
    from paper_2107_07776_gb300.abcstudy import abc_gradient, nodal_errors
    w = W.ABC.scaled((N,) * 3, degree=k)
    om = Mesh(3, [N] * 3, list(w.lo), list(w.hi), [True] * 3, k)
    X, Xp = om.node_coords(), om.node_coords(True)
    u = W.abc_u(*X, 0.0) * 1.01 + 0.001 * np.cos(X[0])
    p = W.abc_p(*Xp, 0.0) * 0.97
    t = 0.3
    eu, ep, eh = nodal_errors(w, None, u.reshape(-1), p, t)
    e2 = n2 = g2 = d2 = 0.0
    for i in range(3):
        ex = lambda x, y, z, i=i: W.abc_u(x, y, z, t)[i]
        gr = lambda x, y, z, i=i: np.stack(abc_gradient(x, y, z, t, 1.0)[i])
        e2 += l2_error(om, u[i], ex, relative=False) ** 2
        n2 += l2_error(om, 0 * u[i], ex, relative=False) ** 2
        g2 += l2_error(om, u[i], gr, relative=False, h1=True) ** 2
        d2 += l2_error(om, 0 * u[i], gr, relative=False, h1=True) ** 2
    eo = l2_error(om, p, lambda x, y, z: W.abc_p(x, y, z, t), p_space=True)
    assert abs(eu / math.sqrt(e2 / n2) - 1) < 1e-10
    assert abs(eh / math.sqrt(g2 / d2) - 1) < 1e-10
    assert abs(ep / eo - 1) < 1e-10
