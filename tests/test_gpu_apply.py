"""Parity of the CUDA operator applies with the oracle's assembled operators
(Section 3): element by element on seeded inputs, FP64 to 1e-12 relative
(the tolerance the work states for applies), FP32 to 2e-5 relative (about
100 ulp of the float path, accumulated over the O(10^2) terms per output).
Meshes span several CTAs with ragged tails, 2D and 3D, periodic (including a
one-cell period, where a cell is its own neighbour) and walled, Cartesian and
tanh-graded and sine-perturbed trilinear, degrees 2 to 4; the benchmark-size
workloads (32^3 Taylor-Green, 64^3 Q3 trilinear, 256x64x64 graded channel)
are checked on sampled cells at full size."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh as OMesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    # dim, n, lo, hi, periodic, degree, map, map_param
    (2, (5, 3), (0, 0), (1.0, 0.7), (True, True), 2, 0, (0, 0, 0)),
    (2, (4, 6), (0, 0), (2.0, 1.0), (False, False), 3, 1, (0.0, 1.5, 0)),
    (2, (1, 2), (0, 0), (1.0, 1.0), (True, False), 4, 0, (0, 0, 0)),
    (3, (5, 3, 7), (0, 0, 0), (1.0, 0.8, 1.3), (True, True, True), 2, 0, (0, 0, 0)),
    (3, (4, 5, 3), (0, 0, 0), (4.0, 1.0, 1.0), (True, False, False), 2, 1, (0.0, 1.5, 1.5)),
    (3, (3, 2, 3), (0, 0, 0), (1.0, 1.0, 1.0), (False, False, False), 3, 0, (0, 0, 0)),
    (3, (1, 1, 2), (0, 0, 0), (1.0, 1.0, 1.0), (True, True, False), 2, 0, (0, 0, 0)),
    (3, (2, 3, 2), (0, 0, 0), (1.0, 1.0, 1.0), (True, False, True), 4, 1, (0.0, 1.2, 0.0)),
    # trilinear (sine-perturbed vertices): general-geometry kernels
    (2, (4, 3), (0, 0), (1.0, 0.8), (False, False), 2, 2, (0.04, 0, 0)),
    (2, (5, 4), (0, 0), (1.0, 1.0), (True, True), 3, 2, (0.05, 0, 0)),
    (3, (3, 4, 2), (0, 0, 0), (1.0, 1.0, 1.0), (False, False, False), 3, 2, (0.03, 0, 0)),
    (3, (4, 3, 3), (0, 0, 0), (1.0, 1.2, 0.9), (True, True, True), 2, 2, (0.05, 0, 0)),
    (3, (1, 2, 3), (0, 0, 0), (1.0, 1.0, 1.0), (True, False, False), 2, 2, (0.04, 0, 0)),
    (3, (2, 2, 3), (0, 0, 0), (1.0, 1.0, 1.0), (True, False, True), 4, 2, (0.03, 0, 0)),
]


def meshes(case):
    from paper_2107_07776_gb300.binding import Mesh
    dim, n, lo, hi, per, k, mp, prm = case
    return (Mesh(dim, n, lo, hi, per, k, mp, prm),
            OMesh(dim, list(n), list(lo), list(hi), list(per), k, map=mp, map_param=list(prm)))


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("fp64_arith", [0, 1])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_poisson_apply_matches_oracle(ci, fp64_arith):
    """fp64_arith 0: float-float arithmetic (48-bit significands, error a few
    2^-48 per operation, far inside 1e-12); 1: native FP64."""
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    b.dg_mesh_set_fp64_arith(gm.handle, fp64_arith)
    x = W.random_vector(om.n_p, 100 + ci)
    alpha = 2.9
    ref = alpha * om.assemble("mass_p").apply(x) + om.assemble("sipg_p").apply(x)
    y = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
    b.dg_apply_poisson(gm.handle, alpha, dev(x), y)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), ref) < 1e-12
    y32 = torch.empty(om.n_p, dtype=torch.float32, device="cuda")
    b.dg_apply_poisson_f32(gm.handle, alpha, dev(x, torch.float32), y32)
    torch.cuda.synchronize()
    assert rel_err(y32.double().cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("fp64_arith", [0, 1])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_momentum_apply_matches_oracle(ci, fp64_arith):
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    b.dg_mesh_set_fp64_arith(gm.handle, fp64_arith)
    d = om.dim
    x = W.random_vector(d * om.n_u, 200 + ci)
    ub = W.random_vector(d * om.n_u, 300 + ci)
    mass, visc, adv = 1.0 / (b.GAMMA * 0.01), 1.0 / 200.0, 0.5
    M = om.assemble("mass_u")
    A = om.assemble("sipg_u")
    C = om.assemble("adv_u", ub)
    ref = np.concatenate([mass * M.apply(x[i * om.n_u:(i + 1) * om.n_u])
                          + visc * A.apply(x[i * om.n_u:(i + 1) * om.n_u])
                          + adv * C.apply(x[i * om.n_u:(i + 1) * om.n_u]) for i in range(d)])
    co = b.momentum_coeffs(mass, visc, adv)
    y = torch.empty(d * om.n_u, dtype=torch.float64, device="cuda")
    b.dg_apply_momentum(gm.handle, co, dev(ub), dev(x), y)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), ref) < 1e-12
    y32 = torch.empty(d * om.n_u, dtype=torch.float32, device="cuda")
    b.dg_apply_momentum_f32(gm.handle, co, dev(ub, torch.float32), dev(x, torch.float32), y32)
    torch.cuda.synchronize()
    assert rel_err(y32.double().cpu().numpy(), ref) < 2e-5


@pytest.mark.parametrize("variant", [5, 6])
@pytest.mark.parametrize("ci", [i for i, c in enumerate(CASES) if c[6] != 2])
def test_face_once_variants_match_oracle(ci, variant):
    """The face-once form (every face's flux once into a scratch, then the
    cells) in float-float, native FP64 and FP32, against the oracle."""
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    b.dg_mesh_set_variant(gm.handle, variant)
    d = om.dim
    x = W.random_vector(d * om.n_u, 200 + ci)
    ub = W.random_vector(d * om.n_u, 300 + ci)
    mass, visc, adv = 1.0 / (b.GAMMA * 0.01), 1.0 / 200.0, 0.5
    M, A, C = om.assemble("mass_u"), om.assemble("sipg_u"), om.assemble("adv_u", ub)
    ref_u = np.concatenate([mass * M.apply(x[i * om.n_u:(i + 1) * om.n_u])
                            + visc * A.apply(x[i * om.n_u:(i + 1) * om.n_u])
                            + adv * C.apply(x[i * om.n_u:(i + 1) * om.n_u]) for i in range(d)])
    xp = W.random_vector(om.n_p, 100 + ci)
    ref_p = 2.9 * om.assemble("mass_p").apply(xp) + om.assemble("sipg_p").apply(xp)
    co = b.momentum_coeffs(mass, visc, adv)
    for arith in (0, 1):
        b.dg_mesh_set_fp64_arith(gm.handle, arith)
        y = torch.empty(d * om.n_u, dtype=torch.float64, device="cuda")
        b.dg_apply_momentum(gm.handle, co, dev(ub), dev(x), y)
        yp = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
        b.dg_apply_poisson(gm.handle, 2.9, dev(xp), yp)
        torch.cuda.synchronize()
        assert rel_err(y.cpu().numpy(), ref_u) < 1e-12, arith
        assert rel_err(yp.cpu().numpy(), ref_p) < 1e-12, arith
    y32 = torch.empty(d * om.n_u, dtype=torch.float32, device="cuda")
    b.dg_apply_momentum_f32(gm.handle, co, dev(ub, torch.float32), dev(x, torch.float32), y32)
    yp32 = torch.empty(om.n_p, dtype=torch.float32, device="cuda")
    b.dg_apply_poisson_f32(gm.handle, 2.9, dev(xp, torch.float32), yp32)
    torch.cuda.synchronize()
    assert rel_err(y32.double().cpu().numpy(), ref_u) < 2e-5
    assert rel_err(yp32.double().cpu().numpy(), ref_p) < 2e-5


@pytest.mark.parametrize("ci", [i for i, c in enumerate(CASES) if c[0] == 3 and c[5] == 2 and c[6] != 2])
def test_q1_thread_per_cell_variant_matches_oracle(ci):
    """Variant 7 for the pressure operator against the oracle: the
    tensor-product kernel in float-float and FP32, the two-threads-per-cell
    kernel in native FP64; the momentum
    operator (not Q1 scalar) runs its fallback and stays exact."""
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    b.dg_mesh_set_variant(gm.handle, 7)
    xp = W.random_vector(om.n_p, 700 + ci)
    ref_p = 2.9 * om.assemble("mass_p").apply(xp) + om.assemble("sipg_p").apply(xp)
    for arith in (0, 1):
        b.dg_mesh_set_fp64_arith(gm.handle, arith)
        yp = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
        b.dg_apply_poisson(gm.handle, 2.9, dev(xp), yp)
        torch.cuda.synchronize()
        assert rel_err(yp.cpu().numpy(), ref_p) < 1e-12, arith
    yp32 = torch.empty(om.n_p, dtype=torch.float32, device="cuda")
    b.dg_apply_poisson_f32(gm.handle, 2.9, dev(xp, torch.float32), yp32)
    torch.cuda.synchronize()
    assert rel_err(yp32.double().cpu().numpy(), ref_p) < 2e-5
    d = om.dim
    x = W.random_vector(d * om.n_u, 800 + ci)
    ref_u = np.concatenate([3.0 * om.assemble("mass_u").apply(x[i * om.n_u:(i + 1) * om.n_u])
                            + 0.01 * om.assemble("sipg_u").apply(x[i * om.n_u:(i + 1) * om.n_u])
                            for i in range(d)])
    y = torch.empty(d * om.n_u, dtype=torch.float64, device="cuda")
    b.dg_apply_momentum(gm.handle, b.momentum_coeffs(3.0, 0.01, 0.0), None, dev(x), y)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), ref_u) < 1e-12


def test_q1_thread_per_cell_variant_in_multigrid():
    """The Chebyshev-fused epilogues of variants 5, 6 (face-once, per
    component and components interleaved) and 7 (the Q1 tensor-product form):
    an FP32-multigrid Helmholtz solve on a Q2/Q1 mesh whose operators all run
    one variant converges to the same solution as with the default
    variant."""
    from paper_2107_07776_gb300 import binding as b
    sols = []
    for variant in (1, 5, 6, 7):
        gm = b.Mesh(3, (8, 6, 8), (0, 0, 0), (1.0, 0.8, 1.0), (True, False, True), 2)
        b.dg_mesh_set_variant(gm.handle, variant)
        s = b.dg_solver_create(gm.handle, 100.0, 1e3)
        try:
            rhs = torch.tensor(W.random_vector(gm.n_dofs_p, 5), device="cuda")
            x = torch.zeros_like(rhs)
            o = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-11, max_iter=100, precond=b.DG_PC_MG_FP32)
            info = b.dg_solve_stage(s, None, 2.9, None, rhs, x, o)
            assert info.status == 0 and info.iterations < 30
            sols.append(x.cpu().numpy())
        finally:
            b.dg_solver_destroy(s)
    for x in sols[1:]:
        assert rel_err(x, sols[0]) < 1e-9


def test_node_coords_match_oracle():
    for case in CASES:
        gm, om = meshes(case)
        for field in (0, 1):
            g = gm.node_coords(field).cpu().numpy()
            o = om.node_coords(p_space=bool(field))
            assert np.abs(g - o).max() < 1e-13


@pytest.mark.parametrize("fp64_arith", [0, 1])
@pytest.mark.parametrize("wname", ["tgv32", "mms64", "channel"])
def test_full_size_workload_sampled_cells(wname, fp64_arith):
    """The benchmark-size meshes as the library launches them: 32^3 Q2/Q1
    Taylor-Green (periodic), 64^3 Q3/Q2 on sine-perturbed trilinear cells
    (walls), 256x64x64 Q2/Q1 tanh-graded channel (walls in y, z): every
    output of 64 sampled cells (first/last cells, a wall row, random) against
    the oracle's rows for those cells."""
    from paper_2107_07776_gb300 import binding as b
    w = W.WORKLOADS[wname]
    gm = b.Mesh.from_workload(w)
    b.dg_mesh_set_fp64_arith(gm.handle, fp64_arith)
    om = OMesh(w.dim, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree,
               map=w.map, map_param=list(w.map_param))
    rng = np.random.default_rng(7)
    N = om.n_cells
    n0, n1 = w.n[0], w.n[1]
    cells = np.unique(np.concatenate([[0, N - 1, n0 - 1, n0 * (n1 - 1), N - n0],
                                      rng.integers(0, N, 59)]))
    # pressure
    xp = W.random_vector(om.n_p, 11)
    y = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
    alpha = 1.0 / (w.c ** 2 * (b.GAMMA * w.dt) ** 2)
    b.dg_apply_poisson(gm.handle, alpha, dev(xp), y)
    yc = y.cpu().numpy().reshape(N, -1)[cells].reshape(-1)
    ref = alpha * om.assemble("mass_p", cells=cells).apply(xp) + \
        om.assemble("sipg_p", cells=cells).apply(xp)
    assert rel_err(yc, ref) < 1e-12
    # momentum; advecting field: the workload's initial velocity (its forcing
    # for the manufactured case, which starts from rest)
    X = gm.node_coords(0).cpu().numpy()
    Xp = gm.node_coords(1).cpu().numpy()
    ub = W.initial_state(w, X, Xp)[0]
    if not np.any(ub):
        ub = W.forcing(w, X)
    ub = ub.reshape(-1)
    xu = W.random_vector(3 * om.n_u, 12)
    mass, visc, adv = 1.0 / (b.GAMMA * w.dt), 1.0 / (2 * w.Re), 0.5
    yu = torch.empty(3 * om.n_u, dtype=torch.float64, device="cuda")
    b.dg_apply_momentum(gm.handle, b.momentum_coeffs(mass, visc, adv), dev(ub), dev(xu), yu)
    yu = yu.cpu().numpy().reshape(3, N, -1)
    Mb = om.assemble("mass_u", cells=cells)
    Ab = om.assemble("sipg_u", cells=cells)
    Cb = om.assemble("adv_u", ub, cells=cells)
    for i in range(3):
        xi = xu[i * om.n_u:(i + 1) * om.n_u]
        ref = mass * Mb.apply(xi) + visc * Ab.apply(xi) + adv * Cb.apply(xi)
        assert rel_err(yu[i][cells].reshape(-1), ref) < 1e-12


@pytest.mark.parametrize("tuning", ["autotune", 5, 6, 7])
@pytest.mark.parametrize("wname", ["tgv32", "channel"])
def test_full_size_benchmark_variants_sampled_cells(wname, tuning):
    """The kernels the benchmark times, at full size: after dg_autotune (the
    benchmark's own call) or with the face-once variants (5, 6: every face's
    flux once into the mesh's scratch, then the cells) and the
    Q1 tensor-product variant (7) forced.  64 sampled cells of the
    float-float FP64 applies at 1e-12, and of the FP32 Poisson apply (the
    multigrid's finest operator) at 2e-5, against the oracle's rows."""
    from paper_2107_07776_gb300 import binding as b
    w = W.WORKLOADS[wname]
    gm = b.Mesh.from_workload(w)
    if tuning == "autotune":
        b.dg_autotune(gm.handle)
        assert b.dg_autotune_report(gm.handle) != "[]"
    else:
        b.dg_mesh_set_variant(gm.handle, tuning)
    om = OMesh(w.dim, list(w.n), list(w.lo), list(w.hi), list(w.periodic), w.degree,
               map=w.map, map_param=list(w.map_param))
    rng = np.random.default_rng(17)
    N = om.n_cells
    n0, n1 = w.n[0], w.n[1]
    cells = np.unique(np.concatenate([[0, N - 1, n0 - 1, n0 * (n1 - 1), N - n0],
                                      rng.integers(0, N, 59)]))
    alpha = 1.0 / (w.c ** 2 * (b.GAMMA * w.dt) ** 2)
    xp = W.random_vector(om.n_p, 21)
    refp = alpha * om.assemble("mass_p", cells=cells).apply(xp) + \
        om.assemble("sipg_p", cells=cells).apply(xp)
    y = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
    b.dg_apply_poisson(gm.handle, alpha, dev(xp), y)
    assert rel_err(y.cpu().numpy().reshape(N, -1)[cells].reshape(-1), refp) < 1e-12
    y32 = torch.empty(om.n_p, dtype=torch.float32, device="cuda")
    b.dg_apply_poisson_f32(gm.handle, alpha, torch.tensor(xp, dtype=torch.float32,
                                                          device="cuda"), y32)
    assert rel_err(y32.double().cpu().numpy().reshape(N, -1)[cells].reshape(-1), refp) < 2e-5
    X = gm.node_coords(0).cpu().numpy()
    ub = W.initial_state(w, X, gm.node_coords(1).cpu().numpy())[0].reshape(-1)
    xu = W.random_vector(3 * om.n_u, 22)
    mass, visc, adv = 1.0 / (b.GAMMA * w.dt), 1.0 / (2 * w.Re), 0.5
    yu = torch.empty(3 * om.n_u, dtype=torch.float64, device="cuda")
    b.dg_apply_momentum(gm.handle, b.momentum_coeffs(mass, visc, adv), dev(ub), dev(xu), yu)
    yu = yu.cpu().numpy().reshape(3, N, -1)
    Mb = om.assemble("mass_u", cells=cells)
    Ab = om.assemble("sipg_u", cells=cells)
    Cb = om.assemble("adv_u", ub, cells=cells)
    for i in range(3):
        xi = xu[i * om.n_u:(i + 1) * om.n_u]
        ref = mass * Mb.apply(xi) + visc * Ab.apply(xi) + adv * Cb.apply(xi)
        assert rel_err(yu[i][cells].reshape(-1), ref) < 1e-12


def test_bad_arguments_are_rejected():
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[0])
    x = torch.zeros(om.n_p, dtype=torch.float64, device="cuda")
    with pytest.raises(b.DGError):
        b.dg_apply_poisson(gm.handle, 1.0, x, x)          # aliasing
    with pytest.raises(b.DGError):
        b.dg_apply_momentum(gm.handle, b.momentum_coeffs(1, 1, 1), None, x, x)


@pytest.mark.parametrize("scale", [1e-25, 1e-12, 1e12, 1e25])
def test_float_float_apply_keeps_relative_accuracy_over_magnitudes(scale):
    """The FP64-accurate applies split doubles into float pairs with integer
    operations; the operators are linear, so inputs scaled over 50 orders of
    magnitude keep the 1e-12 relative parity."""
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[4])
    x = W.random_vector(om.n_p, 500) * scale
    ref = 2.9 * om.assemble("mass_p").apply(x) + om.assemble("sipg_p").apply(x)
    y = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
    b.dg_apply_poisson(gm.handle, 2.9, dev(x), y)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), ref) < 1e-12
    d = om.dim
    xu = W.random_vector(d * om.n_u, 501) * scale
    ub = W.random_vector(d * om.n_u, 502)
    M, A, C = om.assemble("mass_u"), om.assemble("sipg_u"), om.assemble("adv_u", ub)
    ref = np.concatenate([300.0 * M.apply(xu[i * om.n_u:(i + 1) * om.n_u])
                          + 0.01 * A.apply(xu[i * om.n_u:(i + 1) * om.n_u])
                          + 0.5 * C.apply(xu[i * om.n_u:(i + 1) * om.n_u]) for i in range(d)])
    yu = torch.empty(d * om.n_u, dtype=torch.float64, device="cuda")
    b.dg_apply_momentum(gm.handle, b.momentum_coeffs(300.0, 0.01, 0.5), dev(ub), dev(xu), yu)
    torch.cuda.synchronize()
    assert rel_err(yu.cpu().numpy(), ref) < 1e-12
