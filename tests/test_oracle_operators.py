"""Pins of the oracle's assembled operators (Section 3 of the paper).

Each check is fixed by mathematics independent of the oracle:
 * hand-computed integrals of the SIP form on one or two cells (penalty
   reading (k+1)^2 |Gamma|/|K|, boundary penalty 2 C_u, interior average);
 * consistency: for continuous polynomial fields the DG forms reduce to the
   strong operators (integration by parts), e.g. (A - B_D) u = M(-Lap u)
   when the Dirichlet data is u itself -- a dropped term, sign or wrong
   normal breaks these;
 * symmetry, definiteness and kernels of M, A, K;
 * geometric invariants of the mapped meshes.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.dg import Mesh

MESHES = {
    "cart2d": dict(dim=2, n=[3, 2], lo=[0, 0], hi=[1.5, 1.0], periodic=[False, False], map=0),
    "graded2d": dict(dim=2, n=[3, 4], lo=[0, 0], hi=[2.0, 1.0], periodic=[False, False], map=1,
                     map_param=[0.0, 1.5, 0.0]),
    "cart3d": dict(dim=3, n=[2, 2, 3], lo=[0, 0, 0], hi=[1.0, 1.0, 1.5],
                   periodic=[False, False, False], map=0),
    "graded3d": dict(dim=3, n=[2, 3, 2], lo=[0, 0, 0], hi=[4.0, 1.0, 1.0],
                     periodic=[True, False, False], map=1, map_param=[0.0, 1.5, 1.5]),
}


def mk(name, degree=2):
    return Mesh(degree=degree, **MESHES[name])


def close(a, b, tol=1e-12):
    scale = max(1.0, float(np.abs(b).max()))
    assert np.abs(a - b).max() <= tol * scale, np.abs(a - b).max()


# --------------------------------------------------------- closed forms
def test_sipg_one_cell_unit_square():
    """u = v = x on one unit square, k = 2: int grad u.grad v = 1, each boundary
    consistency/symmetry term -1, penalty 2 * 9 * int_dOmega x^2 = 18 * 5/3."""
    m = Mesh(2, [1, 1], [0, 0], [1, 1], [False, False], 2)
    x = m.node_coords()[0]
    assert abs(x @ (m.csr("sipg_u") @ x) - 29.0) < 1e-12


def test_sipg_one_cell_unit_cube():
    m = Mesh(3, [1, 1, 1], [0, 0, 0], [1, 1, 1], [False] * 3, 2)
    x = m.node_coords()[0]
    assert abs(x @ (m.csr("sipg_u") @ x) - 41.0) < 1e-12


def test_sipg_penalty_uses_face_over_volume():
    """[0,2]x[0,1], one cell: sigma = 9*1/2 on x faces, 9*2/2 on y faces;
    2 - 2 - 2 + 2*4.5*4 + 2*9*(8/3 + 8/3) = 130."""
    m = Mesh(2, [1, 1], [0, 0], [2, 1], [False, False], 2)
    x = m.node_coords()[0]
    assert abs(x @ (m.csr("sipg_u") @ x) - 130.0) < 1e-11


def test_sipg_interior_jump_penalty():
    """u = 1 on the left of two unit squares: interior penalty C = (9+9)/2 on
    the shared edge, boundary penalty 2*9 on the left cell's three walls."""
    m = Mesh(2, [2, 1], [0, 0], [2, 1], [False, False], 2)
    u = np.zeros(m.n_u)
    u[: m.nb_u] = 1.0
    assert abs(u @ (m.csr("sipg_u") @ u) - (9.0 + 54.0)) < 1e-12


def test_pressure_sipg_energy_is_h1_for_continuous():
    """For continuous p the SIP energy is int |grad p|^2; Neumann walls add
    nothing."""
    m = Mesh(2, [2, 3], [0, 0], [1, 1], [False, False], 2)
    xp, yp = m.node_coords(True)
    p = 2 * xp - yp
    assert abs(p @ (m.csr("sipg_p") @ p) - 5.0) < 1e-12


def test_mass_is_l2_product():
    m = Mesh(2, [2, 2], [0, 0], [1, 2], [False, False], 2)
    x, y = m.node_coords()
    M = m.csr("mass_u")
    assert abs(x @ (M @ y) - 1.0) < 1e-13           # int_0^1 int_0^2 x y = 1
    assert abs(np.ones(m.n_u) @ (M @ np.ones(m.n_u)) - 2.0) < 1e-13


# --------------------------------------------------------- consistency
@pytest.mark.parametrize("name", list(MESHES))
def test_consistency_identities(name):
    m = mk(name)
    d = m.dim
    X = m.node_coords()
    Xp = m.node_coords(True)
    M = m.csr("mass_u")
    Mp = m.csr("mass_p")
    x, y = X[0], X[1]
    xp, yp = Xp[0], Xp[1]
    z = X[2] if d == 3 else 0 * x
    zp = Xp[2] if d == 3 else 0 * xp
    periodic_x = bool(m.periodic[0])
    # polynomial fields: for a periodic axis use fields independent of x
    if periodic_x:
        u = y * y - 3 * y * z + z * z
        lap = 4.0 + 0 * y
        p = 2 * yp - 3 * zp + 0.5 * yp * zp
        dp = [0 * y, 2 + 0.5 * z, -3 + 0.5 * y]
        ub = np.concatenate([0 * y + 1.0, z, y])  # constant x, div-free
        ubgrad = (2 * y - 3 * z) * z + (-3 * y + 2 * z) * y
    else:
        u = x * x - 3 * x * y + y * y + (z * z if d == 3 else 0)
        lap = (6.0 if d == 3 else 4.0) + 0 * x
        p = 2 * xp - 3 * yp + 0.5 * xp * yp
        dp = [2 + 0.5 * y, -3 + 0.5 * x] + ([0 * x] if d == 3 else [])
        ub = np.concatenate([y, x] + ([0 * x] if d == 3 else []))
        ubgrad = y * (2 * x - 3 * y) + x * (-3 * x + 2 * y)
    A = m.csr("sipg_u")
    close((A - m.csr("dirvisc_u")) @ u, M @ (-lap))
    close(m.csr("explvisc_u") @ u, M @ lap)
    Ea = m.csr("expladv_u", ub)
    close(Ea @ u, -(M @ ubgrad))   # div(u ubar) = ubar.grad u (ubar div-free)
    C = m.csr("adv_u", ub)
    close((C - m.csr("diradv_u", ub)) @ u, M @ ubgrad)
    for c in range(d):
        close(m.csr("graddg", comp=c) @ p, -(M @ dp[c]))
        close(m.csr("proj", comp=c) @ p, M @ dp[c])
    # divergence: D u = -M^p div u for continuous u with div u in Q_{k-1}
    if periodic_x:
        uu = [0 * y, y * y, z * z]
        divp = 2 * yp + 2 * zp
    else:
        uu = [x * x, y * y] + ([0 * x] if d == 3 else [])
        divp = 2 * xp + 2 * yp
    Du = sum(m.csr("div", comp=c) @ uu[c] for c in range(d))
    close(Du, -(Mp @ divp))


# --------------------------------------------------------- structure
@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("dim", [2, 3])
def test_symmetry_definiteness_kernels(dim, periodic):
    n = [3, 2, 2][:dim]
    m = Mesh(dim, n, [0] * dim, [1.0, 1.5, 0.7][:dim], [periodic] * dim, 2)
    M, A = m.csr("mass_u").toarray(), m.csr("sipg_u").toarray()
    Mp, K = m.csr("mass_p").toarray(), m.csr("sipg_p").toarray()
    for X in (M, A, Mp, K):
        assert np.abs(X - X.T).max() < 1e-13 * max(1, np.abs(X).max())
    assert sla.eigvalsh(M).min() > 0
    assert sla.eigvalsh(Mp).min() > 0
    ek = sla.eigvalsh(K)
    assert abs(ek[0]) < 1e-10 and ek[1] > 1e-3      # kernel = constants only
    assert np.abs(K @ np.ones(len(K))).max() < 1e-12
    ea = sla.eigvalsh(A)
    if periodic:
        assert abs(ea[0]) < 1e-10 and ea[1] > 1e-3
        assert np.abs(A @ np.ones(len(A))).max() < 1e-12
    else:
        assert ea[0] > 1e-3                           # walls make A SPD
    assert sla.eigvalsh(2.9 * Mp + K).min() > 0
    assert sla.eigvalsh(1700.0 * M + A).min() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_advection_constant_field(dim):
    """Periodic, constant ubar: C 1 = 0 and C + C^T = LF dissipation >= 0."""
    m = Mesh(dim, [3, 2, 2][:dim], [0] * dim, [1.0] * dim, [True] * dim, 2)
    ub = np.concatenate([np.full(m.n_u, v) for v in [0.7, -0.4, 0.25][:dim]])
    C = m.csr("adv_u", ub).toarray()
    assert np.abs(C @ np.ones(len(C))).max() < 1e-12
    assert sla.eigvalsh(C + C.T).min() > -1e-12


def test_penalty_scales_like_inverse_h():
    """In 2D every term of the SIP form a_p is invariant under x -> L x when
    the penalty scales like |Gamma|/|K| = 1/h (the reading taken here); a
    dimensionless penalty (the printed diam(Gamma)/diam(K)) would make the
    penalty part change by a factor L and break this invariance."""
    K1 = Mesh(2, [6, 5], [0, 0], [1.0, 1.0], [True, True], 2).csr("sipg_p").toarray()
    K16 = Mesh(2, [6, 5], [0, 0], [16.0, 16.0], [True, True], 2).csr("sipg_p").toarray()
    assert np.abs(K1 - K16).max() < 1e-10
    assert sla.eigvalsh(K1).min() > -1e-10


# --------------------------------------------------------- mapped geometry
def test_perturbed_mesh_geometry():
    m = Mesh(3, [4, 3, 4], [0, 0, 0], [1, 1, 1], [False] * 3, 3, map=2,
             map_param=[0.05, 0, 0])
    assert abs(m.volume() - 1.0) < 1e-13          # boundary vertices are fixed
    M = m.csr("mass_u")
    assert abs(np.ones(m.n_u) @ (M @ np.ones(m.n_u)) - 1.0) < 1e-13
    A = m.csr("sipg_u")
    assert np.abs((A - A.T).toarray()).max() < 1e-11
    K = m.csr("sipg_p")
    assert np.abs(K @ np.ones(m.n_p)).max() < 1e-11
    # constant velocity has zero discrete divergence on any conforming mesh
    one = np.ones(m.n_u)
    for c in range(3):
        assert np.abs(m.csr("div", comp=c) @ one).max() < 1e-12
    # node coordinates stay inside the cube and differ from the Cartesian ones
    X = m.node_coords()
    assert X.min() > 0 and X.max() < 1
    Xc = Mesh(3, [4, 3, 4], [0, 0, 0], [1, 1, 1], [False] * 3, 3).node_coords()
    assert np.abs(X - Xc).max() > 1e-3


def test_graded_mesh_is_tanh_law():
    """Tensor-product tanh grading with beta = 1.5: node coordinates of the
    graded axis follow 1/2 (1 - tanh(beta (1 - 2 eta))/tanh(beta)) at the cell
    edges; checked through the mass of each cell row."""
    beta = 1.5
    n = 8
    m = Mesh(2, [2, n], [0, 0], [1, 1], [True, False], 2, map=1, map_param=[0, beta, 0])
    Mb = m.assemble("mass_u").blocks[:, 0]
    vol = Mb.sum(axis=(1, 2)).reshape(n, 2)[:, 0]
    eta = np.arange(n + 1) / n
    ycut = 0.5 * (1 - np.tanh(beta * (1 - 2 * eta)) / math.tanh(beta))
    np.testing.assert_allclose(vol, 0.5 * np.diff(ycut), rtol=1e-13)


# --------------------------------------------------------- LF dissipation (Eq. trilinear)
def _two_cells(dim, k=2, hx=1.0):
    n = [2, 1, 1][:dim]
    return Mesh(dim, n, [0] * dim, [2 * hx, 1.0, 1.0][:dim], [False] * dim, k)


def _piecewise_field(m, left, right):
    """Advecting field constant on each of the two cells (x-component only):
    left on cell 0, right on cell 1, zero y/z components."""
    ub = np.zeros((m.dim, m.n_u))
    ub[0, : m.nb_u] = left
    ub[0, m.nb_u:] = right
    return ub.reshape(-1)


@pytest.mark.parametrize("dim", [2, 3])
def test_lf_flux_self_term_two_cells(dim):
    """u = 1 on the left unit cell, 0 on the right, ubar = (a, 0) left and
    (b, 0) right (|a| != |b|).  With the test function on the left cell:
    the volume term vanishes (grad v = 0); the interior face at x = 1
    (outward normal +x) gives 1/2 u ubar.n + lambda/2 [[u]] with lambda =
    max(|a|, |b|); the wall x = 0 gives lambda_wall u v with lambda_wall =
    |ubar.n| = |a|; the other walls have ubar.n = 0.  Face measures are 1:
        u^T C u = a/2 + max(|a|, |b|)/2 + |a|.
    lambda instead of lambda/2 on interior faces, min for max, or another
    wall speed all change the value."""
    a, b = 0.3, -0.8
    m = _two_cells(dim)
    C = m.csr("adv_u", _piecewise_field(m, a, b))
    u = np.zeros(m.n_u)
    u[: m.nb_u] = 1.0
    assert abs(u @ (C @ u) - (a / 2 + max(abs(a), abs(b)) / 2 + abs(a))) < 1e-13
    # swap the speeds: the max now comes from the row cell's own side
    C2 = m.csr("adv_u", _piecewise_field(m, b, a))
    assert abs(u @ (C2 @ u) - (b / 2 + max(abs(a), abs(b)) / 2 + abs(b))) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_lf_flux_coupling_term_two_cells(dim):
    """Row of the right cell (test v = 1 there), trial u = 1 on the left cell:
    only the shared face couples them.  From the right cell the outward
    normal is -x, the neighbour's flux is 1/2 u_L (ubar_L.n) = -a/2 and the
    dissipation -lambda/2 u_L with lambda = max(|a|, |b|):
        v^T C u = -a/2 - max(|a|, |b|)/2."""
    a, b = 0.3, -0.8
    m = _two_cells(dim)
    C = m.csr("adv_u", _piecewise_field(m, a, b))
    u = np.zeros(m.n_u)
    u[: m.nb_u] = 1.0
    v = np.zeros(m.n_u)
    v[m.nb_u:] = 1.0
    assert abs(v @ (C @ u) - (-a / 2 - max(abs(a), abs(b)) / 2)) < 1e-13


def test_lf_wall_speed_uses_normal_component():
    """One unit square, ubar = (a, c) constant, u = v = 1: the volume term
    vanishes and each wall contributes |ubar.n| times its length:
    2|a| + 2|c|."""
    a, c = 0.45, -0.2
    m = Mesh(2, [1, 1], [0, 0], [1, 1], [False, False], 2)
    ub = np.concatenate([np.full(m.n_u, a), np.full(m.n_u, c)])
    u = np.ones(m.n_u)
    assert abs(u @ (m.csr("adv_u", ub) @ u) - (2 * abs(a) + 2 * abs(c))) < 1e-13


# --------------------------------------------------------- pressure penalty (Eq. weakform_p_1)
@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("hx", [1.0, 0.5])
def test_pressure_penalty_jump_two_cells(k, hx):
    """p = 1 on the left of two cells of width hx (height 1), 0 on the right:
    no gradients, so p^T K p is the penalty of the shared face alone,
    C_p |Gamma| with C_p = (sigma+ + sigma-)/2, sigma = k^2 |Gamma|/|K| and k
    the VELOCITY degree: k^2 / hx.  The pressure degree (k-1)^2 or the
    velocity penalty (k+1)^2 give other values.  The coupling entry is
    -k^2 / hx, and homogeneous Neumann walls add nothing."""
    m = Mesh(2, [2, 1], [0, 0], [2 * hx, 1.0], [False, False], k)
    p = np.zeros(m.n_p)
    p[: m.nb_p] = 1.0
    q = np.zeros(m.n_p)
    q[m.nb_p:] = 1.0
    K = m.csr("sipg_p")
    assert abs(p @ (K @ p) - k * k / hx) < 1e-12
    assert abs(q @ (K @ p) + k * k / hx) < 1e-12


def test_pressure_penalty_jump_3d():
    """The same in 3D with unit cubes: k^2 |Gamma|^2 / |K| = 4."""
    m = Mesh(3, [2, 1, 1], [0, 0, 0], [2, 1, 1], [False] * 3, 2)
    p = np.zeros(m.n_p)
    p[: m.nb_p] = 1.0
    assert abs(p @ (m.csr("sipg_p") @ p) - 4.0) < 1e-12


def _sipg_1d(vx, periodic, pen):
    """Textbook 1D SIP matrix on the cells [vx_c, vx_c+1] with the two-point
    Gauss nodal basis: sum_c int u'v' + sum over interior faces of
    (-{{u'}}[v] - [u]{{v'}} + sigma [u][v]), [w] = w_left - w_right,
    sigma = pen (1/h_left + 1/h_right)/2; no terms on boundary faces
    (natural boundary); a periodic axis adds the face between the last and
    the first cell.  Also the diagonal mass w_i h."""
    g = 1.0 / math.sqrt(3.0)
    xr = np.array([(1 - g) / 2, (1 + g) / 2])
    n = len(vx) - 1
    h = np.diff(vx)

    def val(i, t):  # nodal basis i on [0, 1] at t
        return (t - xr[1 - i]) / (xr[i] - xr[1 - i])

    def der(i):
        return 1.0 / (xr[i] - xr[1 - i])

    K = np.zeros((2 * n, 2 * n))
    M = np.zeros(2 * n)
    for c in range(n):
        for i in range(2):
            M[2 * c + i] = 0.5 * h[c]
            for j in range(2):
                K[2 * c + i, 2 * c + j] += h[c] * der(i) * der(j) / h[c] ** 2  # two-point rule is exact
    faces = [(c, c + 1) for c in range(n - 1)] + ([(n - 1, 0)] if periodic else [])
    for L, R in faces:
        sig = pen * (1 / h[L] + 1 / h[R]) / 2
        # traces and derivatives of the basis functions of both cells at the face
        tr = {(L, i): (val(i, 1.0), der(i) / h[L]) for i in range(2)}
        tr.update({(R, i): (-val(i, 0.0), der(i) / h[R]) for i in range(2)})  # jump sign: minus on the right
        funcs = [(L, 0), (L, 1), (R, 0), (R, 1)]
        for cu, iu in funcs:
            ju, du = tr[(cu, iu)]
            for cv, iv in funcs:
                jv, dv = tr[(cv, iv)]
                K[2 * cv + iv, 2 * cu + iu] += -0.5 * du * jv - 0.5 * ju * dv + sig * ju * jv
    return K, M


@pytest.mark.parametrize("name,per", [("cart3d", [True, True, True]), ("graded3d", [True, False, False]),
                                      ("cart3d", [True, True, False])])
def test_q1_pressure_operator_is_a_kronecker_sum(name, per):
    """On Cartesian (and tanh-graded) cells with the collocated two-point
    Gauss rule the pressure SIP operator of degree-2 velocity meshes (Q1
    pressure, penalty k^2 = 4) is the sum over the axes of the 1D SIP matrix
    along that axis times the diagonal masses of the others: the oracle's
    3D face-by-face assembly against textbook 1D matrices."""
    spec = dict(MESHES[name])
    spec["periodic"] = per
    m = Mesh(spec["dim"], spec["n"], spec["lo"], spec["hi"], spec["periodic"], 2, map=spec["map"],
             map_param=spec.get("map_param", [0, 0, 0]))
    n = spec["n"]
    Xp = m.node_coords(True).reshape(3, n[2], n[1], n[0], 2, 2, 2)
    g = 1.0 / math.sqrt(3.0)
    vx = []
    for a in range(3):  # the vertex lattice from the nodes of one line of cells
        line = [Xp[0][0, 0, :, 0, 0, :], Xp[1][0, :, 0, 0, :, 0], Xp[2][:, 0, 0, :, 0, 0]][a]
        hh = (line[:, 1] - line[:, 0]) / g
        lo = line[:, 0] - hh * (1 - g) / 2
        vx.append(np.append(lo, lo[-1] + hh[-1]))
    Ks, Ms = zip(*[_sipg_1d(vx[a], per[a], 4.0) for a in range(3)])
    Dm = [np.diag(x) for x in Ms]
    # (c2 i2, c1 i1, c0 i0) ordering, x fastest
    K = (np.kron(np.kron(Dm[2], Dm[1]), Ks[0]) + np.kron(np.kron(Dm[2], Ks[1]), Dm[0])
         + np.kron(np.kron(Ks[2], Dm[1]), Dm[0]))
    # to the oracle's (cell, node) ordering: cell = c0 + n0 (c1 + n1 c2), node = i0 + 2 i1 + 4 i2
    perm = np.empty(K.shape[0], dtype=int)
    for c2 in range(n[2]):
        for c1 in range(n[1]):
            for c0 in range(n[0]):
                for i2 in range(2):
                    for i1 in range(2):
                        for i0 in range(2):
                            kron = (((c2 * 2 + i2) * n[1] + c1) * 2 + i1) * 2 * n[0] + 2 * c0 + i0
                            perm[(c0 + n[0] * (c1 + n[1] * c2)) * 8 + i0 + 2 * i1 + 4 * i2] = kron
    K = K[np.ix_(perm, perm)]
    A = m.assemble("sipg_p")
    Ad = np.array([A.apply(e) for e in np.eye(K.shape[0])]).T
    assert np.abs(Ad - K).max() < 1e-11 * np.abs(K).max()
    Mp = m.assemble("mass_p")
    mass = np.kron(np.kron(Ms[2], Ms[1]), Ms[0])[perm]
    assert np.abs(Mp.apply(np.ones(K.shape[0])) - mass).max() < 1e-13 * mass.max()
