"""Oracle steps of the two comparison projection schemes of Section 2
(test infrastructure only): Bell-Colella-Glaz (Crank-Nicolson based, Eqs.
momentum_BCG, helmholtz_BCG) and Guermond-Quartapelle (BDF2 based, Eqs.
momentum_HI, helmholtz_HI), both in artificial compressibility form and on
the same assembled DG operators as the TR-BDF2 oracle (Section 3).

Bell-Colella-Glaz, one step from t^n to t^{n+1}:
  (u* - u^n)/dt + A (u* + u^n)/(2 Re) + c(w; (u* + u^n)/2) = -grad p^n,
  w = (u* + u^n)/2 (fully nonlinear: Picard iterations on w, starting from
  u^n; or, with fixed_point <= 1, one solve with w = 3/2 u^n - 1/2 u^{n-1});
  (alpha M^p + K) dp = (1/dt) D u*, alpha = 1/(c dt)^2;
  u^{n+1} = u* - dt M^-1 P dp, p^{n+1} = p^n + dp.
Guermond-Quartapelle BDF2:
  (3 u* - 4 u^n + u^{n-1})/(2 dt) + A u*/Re + c(w; u*) = -grad p^n,
  w = u^{n,*}, the previous step's predicted (unprojected) velocity (u^n on
  the first step);
  u** = u* + tau M^-1 P p^n, tau = 2 dt / 3;
  (alpha M^p + K) p^{n+1} = alpha M^p p^n + (1/tau) D u**, alpha = 1/(c tau)^2;
  u^{n+1} = u** - tau M^-1 P p^{n+1}.

Readings (the paper is silent or inconsistent here):
  * the implicit half of the BCG advection is the Lax-Friedrichs form C(w)
    and the explicit half the central form E_a(w), as TR-BDF2's stages
    treat their implicit and explicit advection; the explicit viscous half is
    the unpenalised form E_v;
  * the BDF2 momentum predictor divides by 2 dt (the printed "/dt" would not
    be BDF2, and the update's 2 dt / 3 assumes 2 dt);
  * the BDF2 Helmholtz equation uses tau = 2 dt / 3 in alpha and in the
    divergence term, consistent with its update (the printed dt there is
    inconsistent with it), the same pattern as the TR-BDF2 stages;
  * u^{n,*} in the BDF2 advection is read as the previous step's
    intermediate velocity, as the starred superscripts denote the stages'
    predicted velocities throughout Section 2 (the second-order
    extrapolation 2 u^n - u^{n-1} diverges at the table's C = 1.63);
  * its advection is the same DG form c(w; .) as the other schemes (the
    skew-symmetric divergence term of the continuous equation vanishes for
    divergence-free w, and the paper compares the schemes on one
    discretisation);
  * Dirichlet data at t^{n+1}; forcing (f^n + f^{n+1})/2 for BCG and f^{n+1}
    for BDF2, as int f.v.
"""
from __future__ import annotations

from typing import Callable, Optional

import numpy as np

from .trbdf2 import MomentumCoeffs, Stepper


class ProjectionStepper:
    """scheme "bcg" or "bdf2"; vectors as in Stepper: u (dim, n_u), p (n_p),
    u_prev = u^{n-1} (the caller's first-step history, u^n if unknown)."""

    def __init__(self, stepper: Stepper, scheme: str, fixed_point: int = 0,
                 fixed_point_tol: float = 1e-10):
        if scheme not in ("bcg", "bdf2"):
            raise ValueError(scheme)
        self.st, self.scheme = stepper, scheme
        self.fixed_point, self.fixed_point_tol = fixed_point, fixed_point_tol
        self.fixed_point_iterations = 0
        self.u_pred = None  # BDF2: the last step's predicted velocity u^{n,*}

    def step(self, u: np.ndarray, p: np.ndarray, u_prev: np.ndarray, t: float, dt: float,
             uD: Optional[Callable[[float], np.ndarray]] = None,
             f: Optional[Callable[[float], np.ndarray]] = None):
        """Returns (u^{n+1}, p^{n+1}, u^n); u^n is the next step's u_prev."""
        st, d = self.st, self.st.mesh.dim
        Re, c = st.Re, st.c
        uDn = None if uD is None else st._wall_data(uD(t + dt))
        if self.scheme == "bcg":
            co = MomentumCoeffs(1.0 / dt, 1.0 / (2.0 * Re), 0.5)
            fc = None if f is None else 0.5 * (f(t) + f(t + dt))

            def rhs_of(w):
                r = np.stack([co.mass * (st.M @ u[i]) for i in range(d)])
                r += st.explicit_rhs([(co.visc, co.adv, u, w)], p)
                if fc is not None:
                    r += np.stack([st.M @ fc[i] for i in range(d)])
                return r + st.dirichlet_rhs(co, w, uDn)

            if self.fixed_point > 1:
                w = u
                ustar = st.solve_momentum(st.momentum_matrix(co, w), rhs_of(w))
                it = 1
                while it < self.fixed_point:
                    w = 0.5 * (ustar + u)
                    nxt = st.solve_momentum(st.momentum_matrix(co, w), rhs_of(w))
                    change = np.linalg.norm(nxt - ustar) / max(np.linalg.norm(nxt), 1e-300)
                    ustar = nxt
                    it += 1
                    if change < self.fixed_point_tol:
                        break
                self.fixed_point_iterations = it
            else:
                w = 1.5 * u - 0.5 * u_prev
                ustar = st.solve_momentum(st.momentum_matrix(co, w), rhs_of(w))
                self.fixed_point_iterations = 1
            alpha = 1.0 / (c * c * dt * dt)
            u_new, dp = st.pressure_stage(ustar, np.zeros_like(p), alpha, dt)
            return u_new, p + dp, u
        # BDF2
        co = MomentumCoeffs(1.5 / dt, 1.0 / Re, 1.0)
        w = u if self.u_pred is None else self.u_pred
        r = np.stack([(st.M @ (4.0 * u[i] - u_prev[i])) / (2.0 * dt) for i in range(d)])
        r += st.explicit_rhs([], p)
        if f is not None:
            f1 = f(t + dt)
            r += np.stack([st.M @ f1[i] for i in range(d)])
        r += st.dirichlet_rhs(co, w, uDn)
        ustar = st.solve_momentum(st.momentum_matrix(co, w), r)
        self.u_pred = ustar
        tau = 2.0 * dt / 3.0
        u_new, p_new = st.pressure_stage(ustar, p, 1.0 / (c * c * tau * tau), tau)
        return u_new, p_new, u
