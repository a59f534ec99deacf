"""Parity of the stage right-hand sides, gradient projection and Jacobi
diagonals (Sections 2-3) with the oracle's assembled forms, FP64 to 1e-12
relative, on meshes with walls (Dirichlet data terms active) and periodic
ones, 2D and 3D, several CTAs with ragged tails."""
import numpy as np
import pytest

import workloads as W
from oracle.dg import Mesh as OMesh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    (2, (5, 3), (0, 0), (1.0, 0.7), (True, True), 2, 0, (0, 0, 0)),
    (2, (4, 6), (0, 0), (2.0, 1.0), (False, False), 3, 1, (0.0, 1.5, 0)),
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


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("ci,variant", [(i, None) for i in range(len(CASES))] +
                         [(i, 5) for i, c in enumerate(CASES) if c[6] != 2])
def test_momentum_rhs(ci, variant):
    """variant 5: the mesh runs the face-once form, which the explicit terms
    follow (every face's central flux once, then the cells)."""
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    if variant is not None:
        b.dg_mesh_set_variant(gm.handle, variant)
    d, nu = om.dim, om.n_u
    rs = lambda s, n: W.random_vector(n, 1000 * ci + s)
    um, w0, w1, wb0, wb1, uD, ub, f = (rs(i, d * nu) for i in range(8))
    p = rs(9, om.n_p)
    mass, vis, adv, dv, da = 3.0, [0.01, 0.02], [0.5, 0.3], 0.07, 0.4
    M = om.assemble("mass_u")
    Ev = om.assemble("explvisc_u")
    Ea = [om.assemble("expladv_u", wb0), om.assemble("expladv_u", wb1)]
    Bv = om.assemble("dirvisc_u")
    Ba = om.assemble("diradv_u", ub)
    walls = not all(om.periodic[a] for a in range(d))
    ref = []
    for i in range(d):
        sl = slice(i * nu, (i + 1) * nu)
        r = mass * M.apply(um[sl]) + M.apply(f[sl])
        for t, (w, E) in enumerate([(w0, Ea[0]), (w1, Ea[1])]):
            r += vis[t] * Ev.apply(w[sl]) + adv[t] * E.apply(w[sl])
        r += om.assemble("graddg", comp=i).apply(p)
        if walls:
            r += dv * Bv.apply(uD[sl]) + da * Ba.apply(uD[sl])
        ref.append(r)
    ref = np.concatenate(ref)
    T = {k: dev(v) for k, v in dict(um=um, w0=w0, w1=w1, wb0=wb0, wb1=wb1, uD=uD, ub=ub, f=f, p=p).items()}
    desc = b.dg_momentum_rhs()
    desc.mass, desc.u_mass, desc.n_terms = mass, T["um"].data_ptr(), 2
    desc.visc[0], desc.visc[1], desc.adv[0], desc.adv[1] = vis[0], vis[1], adv[0], adv[1]
    desc.w[0], desc.w[1] = T["w0"].data_ptr(), T["w1"].data_ptr()
    desc.wbar[0], desc.wbar[1] = T["wb0"].data_ptr(), T["wb1"].data_ptr()
    desc.p, desc.uD, desc.dir_visc, desc.dir_adv = T["p"].data_ptr(), T["uD"].data_ptr(), dv, da
    desc.ubar, desc.f = T["ub"].data_ptr(), T["f"].data_ptr()
    out = torch.empty(d * nu, dtype=torch.float64, device="cuda")
    b.dg_rhs_momentum(gm.handle, desc, out)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_projection_and_pressure_rhs(ci):
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    d, nu = om.dim, om.n_u
    p = W.random_vector(om.n_p, 50 + ci)
    uss = W.random_vector(d * nu, 60 + ci)
    pold = W.random_vector(om.n_p, 70 + ci)
    M = om.assemble("mass_u")
    Minv = np.linalg.inv(M.blocks[:, 0])
    ref = np.concatenate([
        np.einsum("cij,cj->ci", Minv, om.assemble("proj", comp=i).apply(p).reshape(-1, om.nb_u)).reshape(-1)
        for i in range(d)])
    ut = torch.empty(d * nu, dtype=torch.float64, device="cuda")
    b.dg_project_gradient(gm.handle, dev(p), ut)
    torch.cuda.synchronize()
    assert rel_err(ut.cpu().numpy(), ref) < 1e-12
    alpha, tau = 2.9, 0.37
    refp = alpha * om.assemble("mass_p").apply(pold) + sum(
        om.assemble("div", comp=i).apply(uss[i * nu:(i + 1) * nu]) for i in range(d)) / tau
    rp = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
    b.dg_rhs_pressure(gm.handle, alpha, tau, dev(uss), dev(pold), rp)
    torch.cuda.synchronize()
    assert rel_err(rp.cpu().numpy(), refp) < 1e-12


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_diagonals(ci):
    from paper_2107_07776_gb300 import binding as b
    gm, om = meshes(CASES[ci])
    d, nu = om.dim, om.n_u
    ub = W.random_vector(d * nu, 80 + ci)
    mass, visc, adv = 170.0, 0.003, 0.5
    A = (mass * om.csr("mass_u") + visc * om.csr("sipg_u") + adv * om.csr("adv_u", ub))
    dg = torch.empty(nu, dtype=torch.float64, device="cuda")
    b.dg_momentum_diagonal(gm.handle, b.momentum_coeffs(mass, visc, adv), dev(ub), dg)
    torch.cuda.synchronize()
    assert rel_err(dg.cpu().numpy(), A.diagonal()) < 1e-12
    H = 2.9 * om.csr("mass_p") + om.csr("sipg_p")
    dp = torch.empty(om.n_p, dtype=torch.float64, device="cuda")
    b.dg_poisson_diagonal(gm.handle, 2.9, dp)
    torch.cuda.synchronize()
    assert rel_err(dp.cpu().numpy(), H.diagonal()) < 1e-12
