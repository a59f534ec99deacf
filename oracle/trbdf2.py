"""Oracle TR-BDF2 projection step (test infrastructure only).

Follows Section 2 (Eqs. trbdf2, first_stage, helmholtz2a, second_stage,
helmholtz3a) and the algebraic systems at the end of Section 3, in the
paper's order:

  stage 1: extrapolate ubar_1; solve (M/(gamma dt) + A + C(ubar_1)) u* = M u^n/(gamma dt)
           + F_u^(1); project u~** = M^-1 P p^n; u** = u* + gamma dt u~**;
           solve (alpha_1 M^p + K) p^{n+gamma} = alpha_1 M^p p^n + F_p^(1)(u**);
           u~ = M^-1 P p^{n+gamma}; u^{n+gamma} = u* - gamma dt (u~ - u~**)
  stage 2: the same with (1-gamma) dt, a31, a32, a33 and ubar_2.

Readings (where the paper is silent or inconsistent):
  * ubar_1 = (1 + g/(2(1-g))) u^n - g/(2(1-g)) u^{n-1+g}: the printed
    coefficients are exactly the linear extrapolation to t^{n+g/2} from
    t^{n-1+g}, the level the scheme stores (the printed u^{n-1} would target
    the wrong time);
  * ubar_2 = (1/g) u^{n+g} - ((1-g)/g) u^n: the printed first coefficient
    1 + (1+g)/g makes the pair sum to 3; with (1-g) it is the linear
    extrapolation to t^{n+1} and sums to one;
  * the stage-1 final update uses u~^{n+g} = M^-1 P p^{n+g} (the printed
    superscript n+1,** is a typo);
  * forcing f (zero in the paper) enters as int f.v with the TR-BDF2 stage
    weights: (f^n + f^{n+g})/2 in stage 1 and a31 f^n + a32 f^{n+g} + a33
    f^{n+1} in stage 2;
  * Dirichlet data u_D is a velocity-layout nodal field whose boundary
    traces are the data;
  * walls are impermeable: u_D . n = 0 on every wall (no-slip walls and
    moving lids).  There the boundary Lax-Friedrichs speed of the mirror
    state, max(|ubar+ . n|, |(2 u_D - ubar+) . n|) (Section 3, the flux
    "taking boundary conditions into account"), equals |ubar+ . n|, the
    speed the assembled forms use; data with a normal component (inflow
    or outflow boundaries) is refused rather than given another reading.
Systems are solved by sparse LU (small) or scipy CG/GMRES to a relative
residual of 1e-13 (large); mass solves are per-cell dense solves.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dg import Mesh, gauss_legendre, lagrange

GAMMA = 2.0 - math.sqrt(2.0)


def tr_bdf2_coeffs(g: float = GAMMA):
    """a31, a32, a33 of Eq. second_stage."""
    a31 = (1.0 - g) / (2.0 * (2.0 - g))
    return a31, a31, 1.0 / (2.0 - g)


def extrapolate_stage1(u, u_hist, g: float = GAMMA):
    """u^{n+g/2} from u^n and u^{n-1+g} (reading of the first-stage
    extrapolation)."""
    c = g / (2.0 * (1.0 - g))
    return (1.0 + c) * u - c * u_hist


def extrapolate_stage2(u_g, u_n, g: float = GAMMA):
    """second-stage advecting field from u^{n+g} and u^n, linear to t^{n+1}."""
    return (1.0 / g) * u_g - ((1.0 - g) / g) * u_n


@dataclass
class MomentumCoeffs:
    mass: float   # 1/(g dt) or 1/((1-g) dt)
    visc: float   # 1/(2 Re) or a33/Re
    adv: float    # 1/2 or a33


def solve(A: sp.spmatrix, b: np.ndarray, spd: bool, tol: float = 1e-13, x0=None,
          direct_max: int = 60000) -> np.ndarray:
    n = A.shape[0]
    if n <= direct_max:
        return spla.spsolve(A.tocsc(), b)
    d = A.diagonal()
    Pinv = spla.LinearOperator(A.shape, matvec=lambda v: v / d)
    if spd:
        x, info = spla.cg(A, b, x0=x0, rtol=tol, atol=0.0, maxiter=20000, M=Pinv)
    else:
        x, info = spla.gmres(A, b, x0=x0, rtol=tol, atol=0.0, restart=50, maxiter=2000, M=Pinv)
    if info != 0:
        raise RuntimeError(f"oracle solve did not converge ({info})")
    return x


def wall_normal_trace(mesh: Mesh, uD: np.ndarray) -> float:
    """Largest |u_D . n| over the wall faces of the structured box, from the
    traces of the nodal field u_D (shape (dim, n_u)).  The walls are the
    planes x_a = lo_a, hi_a for every mapping built here (the tanh grading
    keeps them and the sine perturbation vanishes on the boundary), so n =
    -e_a or +e_a and the normal component is the trace of component a."""
    d, k = mesh.dim, mesh.degree
    nodes = gauss_legendre(k + 1)[0]
    ends = [lagrange(nodes, 0.0)[0], lagrange(nodes, 1.0)[0]]
    shape = [mesh.n[a] for a in reversed(range(d))] + [k + 1] * d
    worst = 0.0
    for a in range(d):
        if mesh.periodic[a]:
            continue
        comp = np.asarray(uD[a]).reshape(shape)  # (cells z,y,x, nodes z,y,x)
        cax, nax = d - 1 - a, 2 * d - 1 - a
        for s, l in ((0, ends[0]), (1, ends[1])):
            layer = np.take(comp, 0 if s == 0 else mesh.n[a] - 1, axis=cax)
            tr = np.tensordot(layer, l, axes=([nax - 1], [0]))
            worst = max(worst, float(np.abs(tr).max()))
    return worst


class Stepper:
    """Holds the constant operators of one mesh and takes TR-BDF2 steps.

    Vectors: velocity u has shape (dim, n_u) (component-major, each component
    [cell][node]); pressure p has shape (n_p,).
    """

    def __init__(self, mesh: Mesh, Re: float, c: float = 1e3, g: float = GAMMA,
                 tol: float = 1e-13, extrapolate: bool = True, fixed_point: int = 0,
                 fixed_point_tol: float = 1e-10, direct_max: int = 60000):
        self.mesh, self.Re, self.c, self.g, self.tol = mesh, Re, c, g, tol
        # systems up to direct_max unknowns are solved by sparse LU, larger
        # ones by Jacobi-preconditioned CG / GMRES to the relative residual tol
        self.direct_max = direct_max
        # extrapolate=False lags the advecting field (ubar_1 = u^n, ubar_2 =
        # u^{n+g}); the extrapolated fields lose stability near C = 1 on the
        # Taylor-Green test, where the paper's table uses C = 1.63.
        self.extrapolate = extrapolate
        # fixed_point > 0: the fully nonlinear momentum stages of Section 2
        # (the advecting field of the implicit advection term is the unknown
        # itself, found by at most fixed_point Picard iterations that start
        # from the field above and stop when the relative change of the
        # iterate drops below fixed_point_tol); the explicit advection term of
        # stage 1 is then advected by u^n
        self.fixed_point, self.fixed_point_tol = fixed_point, fixed_point_tol
        self.fixed_point_iterations = [0, 0]  # of the last step, per stage
        d = mesh.dim
        self.M = mesh.csr("mass_u")
        self.A = mesh.csr("sipg_u")
        self.Ev = mesh.csr("explvisc_u")
        self.Mp = mesh.csr("mass_p")
        self.K = mesh.csr("sipg_p")
        self.G = [mesh.csr("graddg", comp=i) for i in range(d)]
        self.P = [mesh.csr("proj", comp=i) for i in range(d)]
        self.D = [mesh.csr("div", comp=i) for i in range(d)]
        self.walls = not all(bool(mesh.periodic[a]) for a in range(d))
        self.Bv = mesh.csr("dirvisc_u") if self.walls else None
        mb = mesh.assemble("mass_u").blocks[:, 0]          # (cells, nb, nb)
        self._Minv = np.linalg.inv(mb)

    # building blocks (each one is also compared with the library) -------
    def mass_solve(self, b: np.ndarray) -> np.ndarray:
        """M^{-1} b for one scalar velocity field (M is block diagonal)."""
        nb = self.mesh.nb_u
        B = b.reshape(-1, nb)
        return np.einsum("cij,cj->ci", self._Minv, B).reshape(-1)

    def projection(self, p: np.ndarray) -> np.ndarray:
        """u~ with M u~ = P p (Section 3, projection matrix P)."""
        return np.stack([self.mass_solve(self.P[i] @ p) for i in range(self.mesh.dim)])

    def momentum_matrix(self, co: MomentumCoeffs, ubar: np.ndarray) -> sp.csr_matrix:
        C = self.mesh.csr("adv_u", ubar.reshape(-1))
        return (co.mass * self.M + co.visc * self.A + co.adv * C).tocsr()

    def dirichlet_rhs(self, co: MomentumCoeffs, ubar, uD) -> np.ndarray:
        """Boundary data terms of F_u (Eq. rhs1, last four terms)."""
        d = self.mesh.dim
        if uD is None or not self.walls:
            return np.zeros((d, self.mesh.n_u))
        Ba = self.mesh.csr("diradv_u", ubar.reshape(-1))
        return np.stack([co.visc * (self.Bv @ uD[i]) + co.adv * (Ba @ uD[i]) for i in range(d)])

    def explicit_rhs(self, terms, p) -> np.ndarray:
        """sum over (visc, adv, w, wbar) of the unpenalised viscous and central
        advective terms of Eq. rhs1, plus the DG pressure gradient of p."""
        d = self.mesh.dim
        out = np.zeros((d, self.mesh.n_u))
        for visc, adv, w, wbar in terms:
            Ea = self.mesh.csr("expladv_u", wbar.reshape(-1)) if adv != 0.0 else None
            for i in range(d):
                out[i] += visc * (self.Ev @ w[i])
                if Ea is not None:
                    out[i] += adv * (Ea @ w[i])
        for i in range(d):
            out[i] += self.G[i] @ p
        return out

    def pressure_rhs(self, uss: np.ndarray, p_old: np.ndarray, alpha: float, tau: float):
        """alpha M^p p_old + F_p(u**) (Eqs. weakform_p_1, helmholtz_1)."""
        r = alpha * (self.Mp @ p_old)
        for i in range(self.mesh.dim):
            r += (self.D[i] @ uss[i]) / tau
        return r

    def helmholtz_matrix(self, alpha: float) -> sp.csr_matrix:
        return (alpha * self.Mp + self.K).tocsr()

    def solve_momentum(self, Amat, rhs, x0=None):
        return np.stack([solve(Amat, rhs[i], spd=False, tol=self.tol,
                               x0=None if x0 is None else x0[i], direct_max=self.direct_max)
                         for i in range(self.mesh.dim)])

    def solve_stage(self, co: MomentumCoeffs, ubar0, rhs_of, stage: int):
        """The momentum predictor of one stage: linear with the advecting
        field ubar0, or (fixed_point > 0) Picard iterations on the field.
        rhs_of(ubar) gives the stage's right-hand side for the current field
        (only the Dirichlet data terms depend on it)."""
        ubar = ubar0
        u_new = self.solve_momentum(self.momentum_matrix(co, ubar), rhs_of(ubar))
        it = 1
        while it < max(1, self.fixed_point):
            ubar = u_new
            u_next = self.solve_momentum(self.momentum_matrix(co, ubar), rhs_of(ubar))
            change = np.linalg.norm(u_next - u_new) / max(np.linalg.norm(u_next), 1e-300)
            u_new = u_next
            it += 1
            if change < self.fixed_point_tol:
                break
        self.fixed_point_iterations[stage] = it
        return u_new

    def pressure_stage(self, ustar, p_old, alpha, tau, x0=None):
        ut_old = self.projection(p_old)
        uss = ustar + tau * ut_old
        rhs = self.pressure_rhs(uss, p_old, alpha, tau)
        p_new = solve(self.helmholtz_matrix(alpha), rhs, spd=True, tol=self.tol, x0=x0,
                      direct_max=self.direct_max)
        ut_new = self.projection(p_new)
        return ustar - tau * (ut_new - ut_old), p_new

    def _wall_data(self, uD: np.ndarray) -> np.ndarray:
        """The Dirichlet data of a stage, after checking that it is
        tangential on every wall (the impermeable-wall reading above)."""
        uD = np.asarray(uD)
        tol = 1e-10 * max(1.0, float(np.abs(uD).max()))
        if self.walls and wall_normal_trace(self.mesh, uD) > tol:
            raise ValueError("Dirichlet data must satisfy u_D . n = 0 on the walls")
        return uD

    # the step ----------------------------------------------------------
    def step(self, u: np.ndarray, p: np.ndarray, u_hist: np.ndarray, t: float, dt: float,
             uD: Optional[Callable[[float], np.ndarray]] = None,
             f: Optional[Callable[[float], np.ndarray]] = None):
        """One TR-BDF2 step from t to t+dt.  Returns (u^{n+1}, p^{n+1},
        u^{n+g}); u^{n+g} is the history level of the next step."""
        g, Re, c = self.g, self.Re, self.c
        a31, a32, a33 = tr_bdf2_coeffs(g)
        d = self.mesh.dim
        # ---- stage 1 (Eqs. first_stage, weakform_u_1) ----
        ub1 = extrapolate_stage1(u, u_hist, g) if self.extrapolate else u
        co1 = MomentumCoeffs(1.0 / (g * dt), 1.0 / (2.0 * Re), 0.5)
        rhs = np.stack([co1.mass * (self.M @ u[i]) for i in range(d)])
        # the explicit advection term is advected by ubar_1, or by u^n in the
        # fully nonlinear form
        rhs += self.explicit_rhs([(co1.visc, co1.adv, u, u if self.fixed_point else ub1)], p)
        if f is not None:
            fc = 0.5 * (f(t) + f(t + g * dt))
            rhs += np.stack([self.M @ fc[i] for i in range(d)])
        uD1 = None if uD is None else self._wall_data(uD(t + g * dt))
        ustar = self.solve_stage(co1, ub1, lambda ub: rhs + self.dirichlet_rhs(co1, ub, uD1), 0)
        # ---- stage 1 pressure (Eqs. helmholtz2a, helmholtz_1) ----
        alpha1 = 1.0 / (c * c * g * g * dt * dt)
        u_g, p_g = self.pressure_stage(ustar, p, alpha1, g * dt)
        # ---- stage 2 (Eqs. second_stage, weakform_u_2) ----
        ub2 = extrapolate_stage2(u_g, u, g) if self.extrapolate else u_g
        co2 = MomentumCoeffs(1.0 / ((1.0 - g) * dt), a33 / Re, a33)
        rhs = np.stack([co2.mass * (self.M @ u_g[i]) for i in range(d)])
        rhs += self.explicit_rhs([(a32 / Re, a32, u_g, u_g), (a31 / Re, a31, u, u)], p_g)
        if f is not None:
            fc = a31 * f(t) + a32 * f(t + g * dt) + a33 * f(t + dt)
            rhs += np.stack([self.M @ fc[i] for i in range(d)])
        uD2 = None if uD is None else self._wall_data(uD(t + dt))
        ustar2 = self.solve_stage(co2, ub2, lambda ub: rhs + self.dirichlet_rhs(co2, ub, uD2), 1)
        # ---- stage 2 pressure (Eqs. helmholtz3a, helmholtz_2) ----
        alpha2 = 1.0 / (c * c * (1.0 - g) ** 2 * dt * dt)
        u_new, p_new = self.pressure_stage(ustar2, p_g, alpha2, (1.0 - g) * dt)
        return u_new, p_new, u_g


def interpolate(mesh: Mesh, fn: Callable, p_space: bool = False) -> np.ndarray:
    """Nodal interpolant of fn(*xyz) -> array (components first)."""
    X = mesh.node_coords(p_space)
    return np.asarray(fn(*X), dtype=np.float64)


def l2_error(mesh: Mesh, vec: np.ndarray, fn: Callable, p_space: bool = False,
             relative: bool = True, h1: bool = False):
    """L2 (or H1-seminorm if h1) error of a scalar nodal field against fn,
    by a (k+3)-point Gauss rule per direction."""
    xyz, w, val, grad = mesh.eval_qp(vec, p_space)
    if h1:
        ex = np.asarray(fn(*xyz))  # gradient components
        e2 = sum(((grad[a] - ex[a]) ** 2 * w).sum() for a in range(mesh.dim))
        n2 = sum((ex[a] ** 2 * w).sum() for a in range(mesh.dim))
    else:
        ex = np.asarray(fn(*xyz))
        e2 = ((val - ex) ** 2 * w).sum()
        n2 = (ex ** 2 * w).sum()
    return math.sqrt(e2 / n2) if relative else math.sqrt(e2)
