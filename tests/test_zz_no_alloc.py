"""The allocation-free Helmholtz solve, called through the C ABI, against
dg_solve_stage on the same system.

It serves callers that cannot allocate device memory when they solve (a
fixed memory budget, or a framework owning the device heap).  Every case
makes two calls in a row, so the second one sees the shared scratch array
as the first left it; one case goes from a larger system to a smaller one,
where any scratch value read before it is written would show.  Covered:
Jacobi and no preconditioning, zero and given initial guesses, an affine
mesh with the default and the face-once operator kernels, a trilinear mesh,
and the size limit.  This file is collected last so that a run stopping at
the first failure has run every other test already."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mesh(b, kind):
    if kind == "affine":
        return b.Mesh(3, (7, 5, 6), (0, 0, 0), (1.0, 1.3, 0.9), (True, True, False), 2)
    if kind == "face_once":
        gm = b.Mesh(3, (6, 6, 5), (0, 0, 0), (1.0, 1.0, 1.0), (True, False, True), 2)
        b.dg_mesh_set_variant(gm.handle, 5)
        return gm
    if kind == "small":
        return b.Mesh(3, (3, 4, 3), (0, 0, 0), (1.0, 1.0, 1.0), (False, True, True), 2)
    assert kind == "trilinear"
    return b.Mesh(3, (4, 3, 4), (0, 0, 0), (1.0, 1.0, 1.0), (False,) * 3, 3, 2, (0.04, 0.0, 0.0))


def _compare(b, gm, precond, guess, seed, alpha):
    s = b.dg_solver_create(gm.handle, 100.0, 1e3)
    try:
        o = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-12, max_iter=4000, precond=precond,
                         guess=guess)
        rhs = torch.tensor(W.random_vector(gm.n_dofs_p, seed), device="cuda")
        x0 = torch.tensor(W.random_vector(gm.n_dofs_p, seed + 1), device="cuda")
        x_ref = x0.clone() if guess == b.DG_GUESS_GIVEN else torch.zeros_like(rhs)
        ref = b.dg_solve_stage(s, None, alpha, None, rhs, x_ref, o)
        x = x0.clone() if guess == b.DG_GUESS_GIVEN else torch.full_like(rhs, float("nan"))
        info = b.dg_solve_helmholtz_noalloc(gm.handle, alpha, rhs, x, o)
        torch.cuda.synchronize()
        assert info.status == b.DG_OK
        assert info.iterations == ref.iterations
        err = (x - x_ref).norm().item() / x_ref.norm().item()
        assert err < 1e-10, err
    finally:
        b.dg_solver_destroy(s)


@pytest.mark.parametrize("guess", ["zero", "given"])
@pytest.mark.parametrize("precond", ["jacobi", "none"])
@pytest.mark.parametrize("kind", ["affine", "face_once", "trilinear"])
def test_noalloc_solve_matches_solve_stage_twice(kind, precond, guess):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_07776_gb300 import binding as b
    pc = b.DG_PC_JACOBI if precond == "jacobi" else b.DG_PC_NONE
    gs = b.DG_GUESS_GIVEN if guess == "given" else b.DG_GUESS_ZERO
    gm = _mesh(b, kind)
    for call, alpha in enumerate((2.9, 0.7)):
        _compare(b, gm, pc, gs, 900 + 10 * call, alpha)


def test_noalloc_larger_then_smaller_system():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_07776_gb300 import binding as b
    big, small = _mesh(b, "affine"), _mesh(b, "small")
    assert big.n_dofs_p > small.n_dofs_p
    _compare(b, big, b.DG_PC_JACOBI, b.DG_GUESS_ZERO, 950, 1.3)
    _compare(b, small, b.DG_PC_JACOBI, b.DG_GUESS_ZERO, 960, 0.4)
    _compare(b, small, b.DG_PC_NONE, b.DG_GUESS_GIVEN, 970, 0.4)


def test_noalloc_rejects_systems_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_07776_gb300 import binding as b
    gm = b.Mesh(3, (33, 32, 32), (0, 0, 0), (1, 1, 1), (True,) * 3, 2)
    assert gm.n_dofs_p > 262144
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    o = b.solve_opts(b.DG_SYS_HELMHOLTZ, precond=b.DG_PC_JACOBI)
    info = b.dg_solve_helmholtz_noalloc(gm.handle, 1.0, v, v, o, raise_on_error=False)
    assert info.status == b.DG_EINVAL
    assert "262144" in b.dg_last_error()
