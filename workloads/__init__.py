"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

Holds none of the method's arithmetic: workload descriptions (mesh sizes,
degrees, Reynolds numbers, time steps), closed-form initial/exact fields as
functions of physical coordinates, and seeded random vectors.  Each side
evaluates these fields at node coordinates it computes itself.

Workloads (the paper's hot-path problems, all synthetic, no dataset):
  tg2d      2D periodic square [0,2pi]^2, 8x8 quads, Q2/Q1, nu = 0.01 (Re 100),
            Taylor-Green u = (sin x cos y, -cos x sin y) e^{-2 nu t},
            p = (cos 2x + cos 2y) e^{-4 nu t} / 4, dt = 0.01, 10 steps.
  tgv32     3D periodic cube [0,2pi]^3, 32^3 hexes, Q2/Q1, Re 1600, Taylor-Green
            vortex u = (sin x cos y cos z, -cos x sin y cos z, 0),
            p = (cos 2x + cos 2y)(cos 2z + 2)/16, dt = 1e-3, 20 steps.
  mms64     3D unit cube 64^3, vertices perturbed by 0.05 sin(2pi x)sin(2pi y)sin(2pi z),
            Q3/Q2, walls, seeded Fourier forcing (8 modes, N(0,1)/|kappa|^2).
  tgv48     tgv32 at 48^3 over 400 steps (learned initial guess).
  channel   [0,4]x[0,1]x[0,1], 256x64x64, tanh wall grading (beta 1.5) in y, z,
            Q2/Q1, Re 5000, parabolic profile + seeded 1% perturbation.
  abc       3D periodic cube [0,2pi]^3, 8^3 hexes, Q2/Q1, Re 1, the
            Arnold-Beltrami-Childress flow u = (sin z + cos y, sin x + cos z,
            sin y + cos x) e^{-t/Re} with p = -(sin x cos z + sin y cos x +
            sin z cos y) e^{-2t/Re}, dt 0.32 (C = 1.63), T = 3.2 (10 steps);
            refined by doubling the cells and halving dt (hyperbolic scaling)
            or quartering it (parabolic scaling, mu = 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Tuple

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    periodic: Tuple[bool, ...]
    degree: int
    Re: float
    dt: float
    steps: int
    map: int = 0
    map_param: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    c: float = 1e3

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_dofs_u(self) -> int:
        return self.dim * self.n_cells * (self.degree + 1) ** self.dim

    @property
    def n_dofs_p(self) -> int:
        return self.n_cells * self.degree ** self.dim

    def scaled(self, n: Tuple[int, ...], **kw) -> "Workload":
        d = dict(self.__dict__)
        d["n"] = tuple(n)
        d.update(kw)
        return Workload(**d)


TG2D = Workload("tg2d", 2, (8, 8), (0.0, 0.0), (TWO_PI, TWO_PI), (True, True), 2,
                Re=100.0, dt=0.01, steps=10)
TGV32 = Workload("tgv32", 3, (32, 32, 32), (0.0,) * 3, (TWO_PI,) * 3, (True,) * 3, 2,
                 Re=1600.0, dt=1e-3, steps=20)
MMS64 = Workload("mms64", 3, (64, 64, 64), (0.0,) * 3, (1.0,) * 3, (False,) * 3, 3,
                 Re=100.0, dt=1e-3, steps=10, map=2, map_param=(0.05, 0.0, 0.0))
TGV48 = Workload("tgv48", 3, (48, 48, 48), (0.0,) * 3, (TWO_PI,) * 3, (True,) * 3, 2,
                 Re=1600.0, dt=1e-3, steps=400)
CHANNEL = Workload("channel", 3, (256, 64, 64), (0.0,) * 3, (4.0, 1.0, 1.0),
                   (True, False, False), 2, Re=5000.0, dt=5e-4, steps=50, map=1,
                   map_param=(0.0, 1.5, 1.5))

ABC = Workload("abc", 3, (8, 8, 8), (0.0,) * 3, (TWO_PI,) * 3, (True,) * 3, 2,
               Re=1.0, dt=0.32, steps=10)

WORKLOADS = {w.name: w for w in (TG2D, TGV32, MMS64, TGV48, CHANNEL, ABC)}


# ---------------------------------------------------------------- fields
def tg2d_u(x, y, t=0.0, nu=0.01):
    e = math.exp(-2.0 * nu * t)
    return np.stack([np.sin(x) * np.cos(y) * e, -np.cos(x) * np.sin(y) * e])


def tg2d_p(x, y, t=0.0, nu=0.01):
    return 0.25 * (np.cos(2 * x) + np.cos(2 * y)) * math.exp(-4.0 * nu * t)


def tg2d_grad_u(x, y, t=0.0, nu=0.01):
    """gradients of the two components: [[du/dx, du/dy], [dv/dx, dv/dy]]"""
    e = math.exp(-2.0 * nu * t)
    return [np.stack([np.cos(x) * np.cos(y) * e, -np.sin(x) * np.sin(y) * e]),
            np.stack([np.sin(x) * np.sin(y) * e, -np.cos(x) * np.cos(y) * e])]


def paper_tg_u(x, y, t=0.0, Re=100.0):
    """Taylor-Green field exactly as printed in Section 4.1 (cos/sin order)."""
    e = math.exp(-2.0 * t / Re)
    return np.stack([np.cos(x) * np.sin(y) * e, -np.sin(x) * np.cos(y) * e])


def paper_tg_p(x, y, t=0.0, Re=100.0):
    return -0.25 * (np.cos(2 * x) + np.cos(2 * y)) * math.exp(-4.0 * t / Re)


def tgv3d_u(x, y, z):
    return np.stack([np.sin(x) * np.cos(y) * np.cos(z), -np.cos(x) * np.sin(y) * np.cos(z),
                     np.zeros_like(x)])


def tgv3d_p(x, y, z):
    return (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0


def abc_u(x, y, z, t=0.0, Re=1.0):
    """Arnold-Beltrami-Childress flow (A = B = C = 1) of Section 4.1: a
    Beltrami field (curl u = u), so u.grad u = grad |u|^2/2 and the viscous
    term decays it like e^{-t/Re}."""
    e = math.exp(-t / Re)
    return np.stack([(np.sin(z) + np.cos(y)) * e, (np.sin(x) + np.cos(z)) * e,
                     (np.sin(y) + np.cos(x)) * e])


def abc_p(x, y, z, t=0.0, Re=1.0):
    """Its pressure, -|u|^2/2 up to a constant.  Section 4.1 prints the
    spatial part without a time factor; the exact solution of the equations
    decays like |u|^2, e^{-2t/Re} (the reading taken here)."""
    return -(np.sin(x) * np.cos(z) + np.sin(y) * np.cos(x) + np.sin(z) * np.cos(y)) * \
        math.exp(-2.0 * t / Re)


def channel_u0(x, y, z, seed: int = 1, amp: float = 0.01):
    """Parabolic streamwise profile 16 y(1-y) z(1-z) plus a divergence-free
    perturbation: the analytic curl of the vector potential
    A_c = env(y, z) sum_m a_mc sin(2 pi (k_m0 x/4 + k_m1 y + k_m2 z) + ph_mc),
    env = y^2 (1-y)^2 z^2 (1-z)^2 (8 seeded modes, k in {1..4}^3,
    a ~ N(0,1), ph ~ U[0, 2pi)), scaled so that max|u'| = amp."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 5, size=(8, 3))
    a = rng.standard_normal((8, 3))
    ph = rng.uniform(0.0, TWO_PI, size=(8, 3))
    env = (y * (1 - y) * z * (1 - z)) ** 2
    denv = [np.zeros_like(x),
            2 * y * (1 - y) * (1 - 2 * y) * (z * (1 - z)) ** 2,
            2 * z * (1 - z) * (1 - 2 * z) * (y * (1 - y)) ** 2]
    # dA[c][j] = d A_c / d x_j
    dA = [[np.zeros_like(x) for _ in range(3)] for _ in range(3)]
    for m in range(8):
        kk = (TWO_PI * k[m, 0] / 4.0, TWO_PI * k[m, 1], TWO_PI * k[m, 2])
        arg = kk[0] * x + kk[1] * y + kk[2] * z
        for c in range(3):
            s = np.sin(arg + ph[m, c])
            co = np.cos(arg + ph[m, c])
            for j in range(3):
                dA[c][j] += a[m, c] * (denv[j] * s + env * co * kk[j])
    pert = np.stack([dA[2][1] - dA[1][2], dA[0][2] - dA[2][0], dA[1][0] - dA[0][1]])
    scale = np.abs(pert).max()
    if scale > 0:
        pert *= amp / scale
    base = np.stack([16.0 * y * (1 - y) * z * (1 - z), np.zeros_like(x), np.zeros_like(x)])
    return base + pert


def mms_forcing_modes(seed: int = 0, n_modes: int = 8):
    """Seeded Fourier modes of the manufactured forcing: integer wave vectors
    in {1..4}^3, amplitudes N(0,1)/|kappa|^2 per component, phases U[0,2pi)."""
    rng = np.random.default_rng(seed)
    kap = rng.integers(1, 5, size=(n_modes, 3))
    amp = rng.standard_normal((n_modes, 3)) / (kap ** 2).sum(axis=1, keepdims=True)
    ph = rng.uniform(0.0, TWO_PI, size=(n_modes, 3))
    return kap, amp, ph


def mms_forcing(x, y, z, t=0.0, seed: int = 0):
    kap, amp, ph = mms_forcing_modes(seed)
    out = np.zeros((3,) + np.shape(x))
    for m in range(kap.shape[0]):
        arg = TWO_PI * (kap[m, 0] * x + kap[m, 1] * y + kap[m, 2] * z)
        for c in range(3):
            out[c] += amp[m, c] * np.sin(arg + ph[m, c])
    return out


# ---------------------------------------------------------------- vectors
def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) FP64 vector."""
    return np.random.default_rng(seed).standard_normal(n)


def initial_state(w: Workload, X, Xp):
    """Initial velocity [dim, n] and pressure [n_p] of a workload at the
    velocity node coordinates X and pressure node coordinates Xp."""
    if w.name.startswith("tgv"):
        return tgv3d_u(*X), tgv3d_p(*Xp)
    if w.name == "tg2d":
        return tg2d_u(*X, 0.0, 1.0 / w.Re), tg2d_p(*Xp, 0.0, 1.0 / w.Re)
    if w.name == "channel":
        return channel_u0(*X), np.zeros(Xp.shape[1])
    if w.name == "abc":
        return abc_u(*X, 0.0, w.Re), abc_p(*Xp, 0.0, w.Re)
    return np.zeros((w.dim, X.shape[1])), np.zeros(Xp.shape[1])


def forcing(w: Workload, X):
    """Body force [dim, n] at the velocity nodes X, or None: the manufactured
    forcing of the trilinear workload (constant in time); the other workloads
    are unforced."""
    if w.name.startswith("mms"):
        return mms_forcing(*X)
    return None
