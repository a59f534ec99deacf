"""Oracle mesh and operators (test infrastructure only).

Python face of ``dg_oracle.c``: a structured hexahedral/quadrilateral mesh
(Section 3 of the paper), the assembled block operators of Section 3's weak
forms, and conversion to scipy CSR matrices (Section 3, "algebraic systems":
M, A, C(ubar), M^p, K, P).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp

from .build import build

KIND = {
    "mass_u": 0,      # int phi_j phi_i
    "sipg_u": 1,      # a_u with unit viscosity (Eq. bilin_diff)
    "adv_u": 2,       # c(ubar, ., .) with unit factor (Eq. trilinear)
    "mass_p": 3,      # int psi_j psi_i
    "sipg_p": 4,      # a_p (Eq. weakform_p_1)
    "explvisc_u": 5,  # -int grad w : grad v + sum_E {{grad w}} : <<v>>  (Eq. rhs1)
    "expladv_u": 6,   # +int (w x wbar) : grad v - sum_E {{w x wbar}} : <<v>> (Eq. rhs1)
    "graddg": 7,      # int p div v - sum_E {{p}} [[v]]  (Eq. rhs1), one component
    "proj": 8,        # P_ij = int grad psi_j . phi_i, one component
    "div": 9,         # int u . grad q - sum_E {{u}} . [[q]]  (Eq. weakform_p_1)
    "dirvisc_u": 10,  # boundary: -int (u_D x n) : grad v + int 2 C_u u_D . v
    "diradv_u": 11,   # boundary: -int (u_D x ubar) n . v + int lambda u_D . v
}
_P_TEST = {"mass_p", "sipg_p", "div"}
_P_TRIAL = {"mass_p", "sipg_p", "graddg", "proj"}

_lib = None


class _OraMesh(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("periodic", ctypes.c_int32 * 3),
        ("degree", ctypes.c_int32),
        ("map", ctypes.c_int32),
        ("map_param", ctypes.c_double * 3),
        ("nq_u", ctypes.c_int32),
        ("nq_p", ctypes.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(str(path))
        P = ctypes.POINTER
        L.ora_gauss_legendre.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
        L.ora_lagrange.argtypes = [ctypes.c_int, P(ctypes.c_double), ctypes.c_double,
                                   P(ctypes.c_double), P(ctypes.c_double)]
        L.ora_assemble.argtypes = [P(_OraMesh), ctypes.c_int, P(ctypes.c_double), ctypes.c_int,
                                   ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_double),
                                   P(ctypes.c_int64)]
        L.ora_block_apply.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_double),
                                      P(ctypes.c_double)]
        L.ora_node_coords.argtypes = [P(_OraMesh), ctypes.c_int, P(ctypes.c_double)]
        L.ora_eval_qp.argtypes = [P(_OraMesh), ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                                  P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                  P(ctypes.c_double)]
        L.ora_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def gauss_legendre(n: int):
    """Gauss-Legendre points and weights on [0, 1] (Newton on the Legendre
    three-term recurrence)."""
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().ora_gauss_legendre(n, _dp(x), _dp(w)) != 0:
        raise ValueError(n)
    return x, w


def lagrange(nodes: np.ndarray, x: float):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    v = np.zeros(len(nodes))
    d = np.zeros(len(nodes))
    lib().ora_lagrange(len(nodes), _dp(nodes), float(x), _dp(v), _dp(d))
    return v, d


@dataclass
class BlockOp:
    """Rows of an operator: blocks[r, slot, i, j] couples test node i of row
    cell r with trial node j of cell cols[r, slot]."""
    blocks: np.ndarray
    cols: np.ndarray
    nt: int
    ns: int
    ncol_cells: int

    @property
    def nslot(self):
        return self.blocks.shape[1]

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.size == self.ncol_cells * self.ns
        y = np.empty(self.blocks.shape[0] * self.nt)
        lib().ora_block_apply(self.blocks.shape[0], self.nslot, self.nt, self.ns,
                              _dp(self.blocks), _ip(self.cols), _dp(x), _dp(y))
        return y

    def to_csr(self) -> sp.csr_matrix:
        R, S, nt, ns = self.blocks.shape
        rows = (np.arange(R)[:, None, None, None] * nt + np.arange(nt)[None, None, :, None])
        rows = np.broadcast_to(rows, self.blocks.shape)
        cols = self.cols[:, :, None, None] * ns + np.arange(ns)[None, None, None, :]
        cols = np.broadcast_to(cols, self.blocks.shape)
        valid = np.broadcast_to((self.cols >= 0)[:, :, None, None], self.blocks.shape)
        A = sp.coo_matrix((self.blocks[valid], (rows[valid], cols[valid])),
                          shape=(R * nt, self.ncol_cells * ns))
        return A.tocsr()


@dataclass
class Mesh:
    """Structured box mesh of Section 3 (quadrilaterals in 2D, hexahedra in
    3D) with a Q_k velocity / Q_{k-1} pressure DG pair.

    map: 0 Cartesian, 1 tanh-graded per axis (map_param = beta per axis,
    x = lo + (hi-lo) (1 - tanh(beta (1 - 2 eta)) / tanh(beta)) / 2), 2
    sine-perturbed vertices (x += A (hi-lo) prod_a sin(2 pi eta_a)).
    """
    dim: int
    n: Sequence[int]
    lo: Sequence[float]
    hi: Sequence[float]
    periodic: Sequence[bool]
    degree: int
    map: int = 0
    map_param: Sequence[float] = (0.0, 0.0, 0.0)
    nq_u: int = 0
    nq_p: int = 0
    _c: Optional[_OraMesh] = field(default=None, repr=False)

    def __post_init__(self):
        c = _OraMesh()
        c.dim = self.dim
        n = list(self.n) + [1] * (3 - len(self.n))
        lo = list(self.lo) + [0.0] * (3 - len(self.lo))
        hi = list(self.hi) + [1.0] * (3 - len(self.hi))
        per = list(self.periodic) + [False] * (3 - len(self.periodic))
        for a in range(3):
            c.n[a] = int(n[a]) if a < self.dim else 1
            c.lo[a] = lo[a]
            c.hi[a] = hi[a]
            c.periodic[a] = int(bool(per[a]))
            c.map_param[a] = float(list(self.map_param)[a]) if a < len(self.map_param) else 0.0
        c.degree = self.degree
        c.map = self.map
        c.nq_u = self.nq_u
        c.nq_p = self.nq_p
        self._c = c

    # sizes -------------------------------------------------------------
    @property
    def n_cells(self) -> int:
        return int(np.prod([self.n[a] for a in range(self.dim)]))

    @property
    def nb_u(self) -> int:
        return (self.degree + 1) ** self.dim

    @property
    def nb_p(self) -> int:
        return self.degree ** self.dim

    @property
    def n_u(self) -> int:
        """scalar velocity DoFs (one component)"""
        return self.n_cells * self.nb_u

    @property
    def n_p(self) -> int:
        return self.n_cells * self.nb_p

    # operators ---------------------------------------------------------
    def assemble(self, kind: str, fld: Optional[np.ndarray] = None, comp: int = 0,
                 cells: Optional[np.ndarray] = None) -> BlockOp:
        kid = KIND[kind]
        nt = self.nb_p if kind in _P_TEST else self.nb_u
        ns = self.nb_p if kind in _P_TRIAL else self.nb_u
        nslot = 2 * self.dim + 1
        if cells is None:
            R = self.n_cells
            cptr = None
        else:
            cells = np.ascontiguousarray(cells, dtype=np.int64)
            R = len(cells)
            cptr = _ip(cells)
        blocks = np.empty((R, nslot, nt, ns))
        cols = np.empty((R, nslot), dtype=np.int64)
        if fld is not None:
            fld = np.ascontiguousarray(fld, dtype=np.float64)
            assert fld.size == self.dim * self.n_u
            fptr = _dp(fld)
        else:
            if kind in ("adv_u", "expladv_u", "diradv_u"):
                raise ValueError(f"{kind} needs an advecting field")
            fptr = None
        if not 0 <= comp < self.dim:
            raise ValueError(comp)
        rc = lib().ora_assemble(ctypes.byref(self._c), kid, fptr, comp, R, cptr, _dp(blocks),
                                _ip(cols))
        if rc != 0:
            raise RuntimeError(f"ora_assemble({kind}) failed: {rc}")
        return BlockOp(blocks, cols, nt, ns, self.n_cells)

    def csr(self, kind: str, fld=None, comp: int = 0) -> sp.csr_matrix:
        return self.assemble(kind, fld, comp).to_csr()

    # geometry helpers --------------------------------------------------
    def node_coords(self, p_space: bool = False) -> np.ndarray:
        """[dim, cells * nodes] physical coordinates of the nodes."""
        nb = self.nb_p if p_space else self.nb_u
        out = np.empty((self.dim, self.n_cells * nb))
        lib().ora_node_coords(ctypes.byref(self._c), int(p_space), _dp(out))
        return out

    def eval_qp(self, vec: np.ndarray, p_space: bool = False, nq: Optional[int] = None):
        """Values and gradients of a scalar nodal field at a Gauss rule with
        nq points per direction (default k+3); returns xyz, w*detJ, val, grad."""
        nq = nq or self.degree + 3
        vec = np.ascontiguousarray(vec, dtype=np.float64)
        nqd = nq ** self.dim
        M = self.n_cells * nqd
        xyz = np.empty((self.dim, M))
        w = np.empty(M)
        val = np.empty(M)
        grad = np.empty((self.dim, M))
        rc = lib().ora_eval_qp(ctypes.byref(self._c), int(p_space), nq, _dp(vec), _dp(xyz),
                               _dp(w), _dp(val), _dp(grad))
        if rc != 0:
            raise RuntimeError(rc)
        return xyz, w, val, grad

    def volume(self) -> float:
        xyz, w, _, _ = self.eval_qp(np.zeros(self.n_u))
        return float(w.sum())
