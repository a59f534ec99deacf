"""Thin ctypes binding of the C ABI in include/dg.h.

Argument marshalling only: every function forwards to the CUDA library
``libdgns.so`` with the same name; tensors are passed by ``data_ptr()``.
There is no CPU fallback: importing this module on a machine without the
built library raises.
"""
from __future__ import annotations

import ctypes
import math
from pathlib import Path
from typing import Optional, Sequence

HERE = Path(__file__).resolve().parent
LIB_PATH = HERE / "libdgns.so"

DG_OK, DG_EINVAL, DG_ECUDA, DG_ENOMEM, DG_ENOCONV, DG_EBREAKDOWN, DG_ETIMEOUT, DG_EUNSUPPORTED = range(8)
DG_MAP_CARTESIAN, DG_MAP_GRADED_TANH, DG_MAP_PERTURBED_SIN = 0, 1, 2
DG_SYS_MOMENTUM, DG_SYS_HELMHOLTZ = 0, 1
DG_PC_NONE, DG_PC_JACOBI, DG_PC_MG_FP64, DG_PC_MG_FP32 = 0, 1, 2, 3
DG_GUESS_ZERO, DG_GUESS_EXTRAP, DG_GUESS_LEARNED, DG_GUESS_GIVEN = 0, 1, 2, 3
DG_SCHEME_BCG, DG_SCHEME_BDF2 = 1, 2
GAMMA = 2.0 - math.sqrt(2.0)

c_double_p = ctypes.c_void_p
c_void_p = ctypes.c_void_p


class dg_mesh_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_cells", ctypes.c_int32 * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int32 * 3), ("degree_u", ctypes.c_int32),
                ("map", ctypes.c_int32), ("map_param", ctypes.c_double * 3)]


class dg_momentum_coeffs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("visc", ctypes.c_double), ("adv", ctypes.c_double)]


class dg_momentum_rhs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("u_mass", c_void_p), ("n_terms", ctypes.c_int32),
                ("visc", ctypes.c_double * 2), ("adv", ctypes.c_double * 2),
                ("w", c_void_p * 2), ("wbar", c_void_p * 2), ("p", c_void_p), ("uD", c_void_p),
                ("dir_visc", ctypes.c_double), ("dir_adv", ctypes.c_double),
                ("ubar", c_void_p), ("f", c_void_p)]


class dg_solve_opts(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int32), ("tol_rel", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("guess", ctypes.c_int32),
                ("timeout_s", ctypes.c_double), ("mg_degree", ctypes.c_int32)]


class dg_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("res0", ctypes.c_double),
                ("res_final", ctypes.c_double), ("status", ctypes.c_int32)]


class dg_guess_opts(ctypes.Structure):
    _fields_ = [("enable", ctypes.c_int32), ("train", ctypes.c_int32),
                ("systems", ctypes.c_int32), ("hidden", ctypes.c_int32),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint64)]


class dg_guess_stats(ctypes.Structure):
    _fields_ = [("train_steps", ctypes.c_int64), ("last_loss", ctypes.c_double),
                ("history", ctypes.c_int32 * 4)]


class dg_projection_params(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("dt", ctypes.c_double), ("uD", c_void_p),
                ("f_n", c_void_p), ("f_n1", c_void_p), ("mom", dg_solve_opts),
                ("helm", dg_solve_opts), ("fixed_point", ctypes.c_int32),
                ("fixed_point_tol", ctypes.c_double)]


class dg_step_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gamma", ctypes.c_double),
                ("extrapolate", ctypes.c_int32), ("uD_stage1", c_void_p),
                ("uD_stage2", c_void_p), ("f_n", c_void_p), ("f_ng", c_void_p),
                ("f_n1", c_void_p), ("mom", dg_solve_opts), ("helm", dg_solve_opts),
                ("fixed_point", ctypes.c_int32), ("fixed_point_tol", ctypes.c_double)]


# name -> (restype, argtypes); the list mirrors include/dg.h
P = ctypes.POINTER
SIGNATURES = {
    "dg_mesh_create": (ctypes.c_int, [P(dg_mesh_desc), c_void_p, P(c_void_p)]),
    "dg_mesh_destroy": (None, [c_void_p]),
    "dg_mesh_info": (ctypes.c_int, [c_void_p, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)]),
    "dg_mesh_node_coords": (ctypes.c_int, [c_void_p, ctypes.c_int32, c_void_p, c_void_p]),
    "dg_mesh_set_fp64_arith": (ctypes.c_int, [c_void_p, ctypes.c_int32]),
    "dg_apply_momentum": (ctypes.c_int, [c_void_p, P(dg_momentum_coeffs), c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_apply_momentum_f32": (ctypes.c_int, [c_void_p, P(dg_momentum_coeffs), c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_apply_poisson": (ctypes.c_int, [c_void_p, ctypes.c_double, c_void_p, c_void_p, c_void_p]),
    "dg_apply_poisson_f32": (ctypes.c_int, [c_void_p, ctypes.c_double, c_void_p, c_void_p, c_void_p]),
    "dg_autotune": (ctypes.c_int, [c_void_p, c_void_p]),
    "dg_autotune_report": (ctypes.c_int, [c_void_p, ctypes.c_char_p, ctypes.c_int64]),
    "dg_rhs_momentum": (ctypes.c_int, [c_void_p, P(dg_momentum_rhs), c_void_p, c_void_p]),
    "dg_project_gradient": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_rhs_pressure": (ctypes.c_int, [c_void_p, ctypes.c_double, ctypes.c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_momentum_diagonal": (ctypes.c_int, [c_void_p, P(dg_momentum_coeffs), c_void_p, c_void_p, c_void_p]),
    "dg_poisson_diagonal": (ctypes.c_int, [c_void_p, ctypes.c_double, c_void_p, c_void_p]),
    "dg_solver_create": (ctypes.c_int, [c_void_p, ctypes.c_double, ctypes.c_double, P(c_void_p)]),
    "dg_solver_destroy": (None, [c_void_p]),
    "dg_solve_stage": (ctypes.c_int, [c_void_p, P(dg_momentum_coeffs), ctypes.c_double, c_void_p, c_void_p, c_void_p, P(dg_solve_opts), P(dg_solve_info)]),
    "trbdf2_step": (ctypes.c_int, [c_void_p, P(dg_step_params), c_void_p, c_void_p, P(dg_solve_info)]),
    "dg_solver_set_history": (ctypes.c_int, [c_void_p, c_void_p]),
    "dg_solver_set_stream": (ctypes.c_int, [c_void_p, c_void_p]),
    "dg_solver_get_fixed_point": (ctypes.c_int, [c_void_p, P(ctypes.c_int32)]),
    "dg_projection_step": (ctypes.c_int, [c_void_p, P(dg_projection_params), c_void_p, c_void_p, P(dg_solve_info)]),
    "dg_solver_set_tracing": (ctypes.c_int, [c_void_p, ctypes.c_int32]),
    "dg_solver_get_trace": (ctypes.c_int, [c_void_p, P(ctypes.c_double), P(ctypes.c_int64)]),
    "dg_guess_configure": (ctypes.c_int, [c_void_p, P(dg_guess_opts)]),
    "dg_guess_get_stats": (ctypes.c_int, [c_void_p, P(dg_guess_stats)]),
    "dg_mlp_forward_backward": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, c_void_p, c_void_p, c_void_p, c_void_p, P(ctypes.c_float), c_void_p, c_void_p]),
    "dg_mesh_set_variant": (ctypes.c_int, [c_void_p, ctypes.c_int32]),
    "dg_mlp_infer": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_solver_save": (ctypes.c_int, [c_void_p, ctypes.c_char_p]),
    "dg_solver_load": (ctypes.c_int, [c_void_p, ctypes.c_char_p]),
    "dg_solve_helmholtz_noalloc": (ctypes.c_int, [c_void_p, ctypes.c_double, c_void_p, c_void_p, P(dg_solve_opts), P(dg_solve_info), c_void_p]),
    "dg_kernel_launches": (ctypes.c_int64, []),
    "dg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libdgns.so (built by paper_2107_07776_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class DGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().dg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib().dg_status_string(status).decode()} ({msg})")


def check(status: int, where: str) -> None:
    if status != DG_OK:
        raise DGError(status, where)


def ptr(t) -> Optional[int]:
    """Device (or host) address of a tensor, an int, or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def stream_ptr(stream=None) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ------------------------------------------------------------------ calls
def dg_mesh_create(desc: dg_mesh_desc, stream=None) -> int:
    out = c_void_p()
    check(lib().dg_mesh_create(ctypes.byref(desc), stream_ptr(stream), ctypes.byref(out)),
          "dg_mesh_create")
    return out.value


def dg_mesh_destroy(mesh: int) -> None:
    lib().dg_mesh_destroy(mesh)


def dg_mesh_info(mesh: int):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().dg_mesh_info(mesh, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "dg_mesh_info")
    return a.value, b.value, c.value


def dg_mesh_node_coords(mesh: int, field: int, xyz, stream=None) -> None:
    check(lib().dg_mesh_node_coords(mesh, field, ptr(xyz), stream_ptr(stream)),
          "dg_mesh_node_coords")


def dg_mesh_set_fp64_arith(mesh: int, mode: int) -> None:
    check(lib().dg_mesh_set_fp64_arith(mesh, mode), "dg_mesh_set_fp64_arith")


def dg_mesh_set_variant(mesh: int, variant: int) -> None:
    check(lib().dg_mesh_set_variant(mesh, variant), "dg_mesh_set_variant")


def dg_apply_momentum(mesh: int, co: dg_momentum_coeffs, ubar, src, dst, stream=None) -> None:
    check(lib().dg_apply_momentum(mesh, ctypes.byref(co), ptr(ubar), ptr(src), ptr(dst),
                                  stream_ptr(stream)), "dg_apply_momentum")


def dg_apply_momentum_f32(mesh: int, co: dg_momentum_coeffs, ubar, src, dst, stream=None) -> None:
    check(lib().dg_apply_momentum_f32(mesh, ctypes.byref(co), ptr(ubar), ptr(src), ptr(dst),
                                      stream_ptr(stream)), "dg_apply_momentum_f32")


def dg_apply_poisson(mesh: int, alpha: float, src, dst, stream=None) -> None:
    check(lib().dg_apply_poisson(mesh, alpha, ptr(src), ptr(dst), stream_ptr(stream)),
          "dg_apply_poisson")


def dg_apply_poisson_f32(mesh: int, alpha: float, src, dst, stream=None) -> None:
    check(lib().dg_apply_poisson_f32(mesh, alpha, ptr(src), ptr(dst), stream_ptr(stream)),
          "dg_apply_poisson_f32")


def dg_autotune(mesh: int, stream=None) -> None:
    check(lib().dg_autotune(mesh, stream_ptr(stream)), "dg_autotune")


def dg_autotune_report(mesh: int) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib().dg_autotune_report(mesh, buf, len(buf)), "dg_autotune_report")
    return buf.value.decode()


def dg_rhs_momentum(mesh: int, desc: dg_momentum_rhs, rhs, stream=None) -> None:
    check(lib().dg_rhs_momentum(mesh, ctypes.byref(desc), ptr(rhs), stream_ptr(stream)),
          "dg_rhs_momentum")


def dg_project_gradient(mesh: int, p, u_tilde, stream=None) -> None:
    check(lib().dg_project_gradient(mesh, ptr(p), ptr(u_tilde), stream_ptr(stream)),
          "dg_project_gradient")


def dg_rhs_pressure(mesh: int, alpha: float, tau: float, uss, p_old, rhs, stream=None) -> None:
    check(lib().dg_rhs_pressure(mesh, alpha, tau, ptr(uss), ptr(p_old), ptr(rhs),
                                stream_ptr(stream)), "dg_rhs_pressure")


def dg_momentum_diagonal(mesh: int, co: dg_momentum_coeffs, ubar, diag, stream=None) -> None:
    check(lib().dg_momentum_diagonal(mesh, ctypes.byref(co), ptr(ubar), ptr(diag),
                                     stream_ptr(stream)), "dg_momentum_diagonal")


def dg_poisson_diagonal(mesh: int, alpha: float, diag, stream=None) -> None:
    check(lib().dg_poisson_diagonal(mesh, alpha, ptr(diag), stream_ptr(stream)),
          "dg_poisson_diagonal")


def dg_solver_create(mesh: int, Re: float, c: float) -> int:
    out = c_void_p()
    check(lib().dg_solver_create(mesh, Re, c, ctypes.byref(out)), "dg_solver_create")
    return out.value


def dg_solver_destroy(solver: int) -> None:
    lib().dg_solver_destroy(solver)


def dg_solve_stage(solver: int, co: Optional[dg_momentum_coeffs], alpha: float, ubar, rhs, x,
                   opts: dg_solve_opts, raise_on_error: bool = True) -> dg_solve_info:
    info = dg_solve_info()
    st = lib().dg_solve_stage(solver, ctypes.byref(co) if co is not None else None, alpha,
                              ptr(ubar), ptr(rhs), ptr(x), ctypes.byref(opts), ctypes.byref(info))
    if raise_on_error:
        check(st, "dg_solve_stage")
    info.status = st
    return info


def trbdf2_step(solver: int, params: dg_step_params, u, p):
    info = (dg_solve_info * 4)()
    check(lib().trbdf2_step(solver, ctypes.byref(params), ptr(u), ptr(p), info), "trbdf2_step")
    return list(info)


def dg_solver_set_history(solver: int, u_hist) -> None:
    check(lib().dg_solver_set_history(solver, ptr(u_hist)), "dg_solver_set_history")


def dg_solver_set_stream(solver: int, stream=None) -> None:
    check(lib().dg_solver_set_stream(solver, stream_ptr(stream)), "dg_solver_set_stream")


def dg_projection_step(solver: int, params: dg_projection_params, u, p):
    info = (dg_solve_info * 2)()
    check(lib().dg_projection_step(solver, ctypes.byref(params), ptr(u), ptr(p), info),
          "dg_projection_step")
    return list(info)


def dg_solver_get_fixed_point(solver: int):
    it = (ctypes.c_int32 * 2)()
    check(lib().dg_solver_get_fixed_point(solver, it), "dg_solver_get_fixed_point")
    return [it[0], it[1]]


def dg_solver_set_tracing(solver: int, on: int) -> None:
    check(lib().dg_solver_set_tracing(solver, on), "dg_solver_set_tracing")


TRACE_PHASES = ("momentum_rhs", "guess", "momentum_solve", "projection_pressure_rhs",
                "helmholtz_solve", "unused")


def dg_solver_get_trace(solver: int):
    arr = (ctypes.c_double * 6)()
    steps = ctypes.c_int64()
    check(lib().dg_solver_get_trace(solver, arr, ctypes.byref(steps)), "dg_solver_get_trace")
    return dict(zip(TRACE_PHASES, list(arr))), steps.value


def dg_guess_configure(solver: int, enable: int = 1, train: int = 1, systems: int = 1,
                       hidden: int = 128, lr: float = 1e-3, seed: int = 1) -> None:
    o = dg_guess_opts()
    o.enable, o.train, o.systems, o.hidden, o.lr, o.seed = enable, train, systems, hidden, lr, seed
    check(lib().dg_guess_configure(solver, ctypes.byref(o)), "dg_guess_configure")


def dg_guess_get_stats(solver: int) -> dg_guess_stats:
    st = dg_guess_stats()
    check(lib().dg_guess_get_stats(solver, ctypes.byref(st)), "dg_guess_get_stats")
    return st


def dg_mlp_forward_backward(M: int, n_in: int, hidden: int, n_out: int, weights, X, T, Y, grad,
                            stream=None) -> float:
    loss = ctypes.c_float(0.0)
    check(lib().dg_mlp_forward_backward(M, n_in, hidden, n_out, ptr(weights), ptr(X), ptr(T),
                                        ptr(Y), ctypes.byref(loss), ptr(grad), stream_ptr(stream)),
          "dg_mlp_forward_backward")
    return loss.value


def dg_mlp_infer(M: int, n_in: int, hidden: int, n_out: int, weights, X, Y, stream=None) -> None:
    check(lib().dg_mlp_infer(M, n_in, hidden, n_out, ptr(weights), ptr(X), ptr(Y),
                             stream_ptr(stream)), "dg_mlp_infer")


def dg_solver_save(solver: int, path: str) -> None:
    check(lib().dg_solver_save(solver, path.encode()), "dg_solver_save")


def dg_solver_load(solver: int, path: str) -> None:
    check(lib().dg_solver_load(solver, path.encode()), "dg_solver_load")


# ------------------------------------------------------------------ helpers
def mesh_desc(dim: int, n: Sequence[int], lo: Sequence[float], hi: Sequence[float],
              periodic: Sequence[bool], degree: int, map: int = 0,
              map_param: Sequence[float] = (0.0, 0.0, 0.0)) -> dg_mesh_desc:
    d = dg_mesh_desc()
    d.dim = dim
    for a in range(3):
        d.n_cells[a] = int(n[a]) if a < len(n) else 1
        d.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        d.hi[a] = float(hi[a]) if a < len(hi) else 1.0
        d.periodic[a] = int(bool(periodic[a])) if a < len(periodic) else 1
        d.map_param[a] = float(map_param[a]) if a < len(map_param) else 0.0
    d.degree_u = degree
    d.map = map
    return d


def momentum_coeffs(mass: float, visc: float, adv: float) -> dg_momentum_coeffs:
    co = dg_momentum_coeffs()
    co.mass, co.visc, co.adv = mass, visc, adv
    return co


def solve_opts(system: int, tol: float = 1e-8, max_iter: int = 500, restart: int = 30,
               precond: int = DG_PC_JACOBI, guess: int = DG_GUESS_ZERO,
               timeout_s: float = 0.0, mg_degree: int = 0) -> dg_solve_opts:
    o = dg_solve_opts()
    o.system, o.tol_rel, o.max_iter, o.restart = system, tol, max_iter, restart
    o.precond, o.guess, o.timeout_s, o.mg_degree = precond, guess, timeout_s, mg_degree
    return o


class Mesh:
    """Owner of a dg_mesh handle with its sizes (convenience for callers)."""

    def __init__(self, dim, n, lo, hi, periodic, degree, map=0, map_param=(0.0, 0.0, 0.0),
                 stream=None):
        self.desc = mesh_desc(dim, n, lo, hi, periodic, degree, map, map_param)
        self.handle = dg_mesh_create(self.desc, stream)
        self.dim, self.degree = dim, degree
        self.n_cells, self.n_dofs_u, self.n_dofs_p = dg_mesh_info(self.handle)
        self.nb_u = (degree + 1) ** dim
        self.nb_p = degree ** dim

    @classmethod
    def from_workload(cls, w, stream=None):
        return cls(w.dim, w.n, w.lo, w.hi, w.periodic, w.degree, w.map, w.map_param, stream)

    def node_coords(self, field: int = 0):
        import torch
        nb = self.nb_u if field == 0 else self.nb_p
        xyz = torch.empty((self.dim, self.n_cells * nb), dtype=torch.float64, device="cuda")
        dg_mesh_node_coords(self.handle, field, xyz)
        return xyz

    def close(self):
        if self.handle:
            dg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_solve_helmholtz_noalloc(mesh: int, alpha: float, rhs, x, opts: dg_solve_opts,
                               stream=None, raise_on_error: bool = True) -> dg_solve_info:
    info = dg_solve_info()
    st = lib().dg_solve_helmholtz_noalloc(mesh, alpha, ptr(rhs), ptr(x), ctypes.byref(opts),
                                          ctypes.byref(info), stream_ptr(stream))
    if raise_on_error:
        check(st, "dg_solve_helmholtz_noalloc")
    info.status = st
    return info


def dg_kernel_launches() -> int:
    return int(lib().dg_kernel_launches())


def dg_status_string(status: int) -> str:
    return lib().dg_status_string(status).decode()


def dg_last_error() -> str:
    return lib().dg_last_error().decode(errors="replace")
