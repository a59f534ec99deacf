"""The allocation-free Helmholtz solve, called through the C ABI, against
dg_solve_stage on the same system: two calls in a row (the second one sees
the scratch array as the first left it), and the size limit.

It serves callers that cannot allocate device memory when they solve (a
fixed memory budget, or a framework owning the device heap); this file is
collected last so that a run stopping at the first failure has run every
other test already."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_solve_matches_solve_stage_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_07776_gb300 import binding as b
    gm = b.Mesh(3, (7, 5, 6), (0, 0, 0), (1.0, 1.3, 0.9), (True, True, False), 2)
    s = b.dg_solver_create(gm.handle, 100.0, 1e3)
    try:
        o = b.solve_opts(b.DG_SYS_HELMHOLTZ, tol=1e-12, max_iter=3000,
                         precond=b.DG_PC_JACOBI, guess=b.DG_GUESS_ZERO)
        for call, alpha in enumerate((2.9, 0.7)):
            rhs = torch.tensor(W.random_vector(gm.n_dofs_p, 900 + call), device="cuda")
            x_ref = torch.zeros_like(rhs)
            ref = b.dg_solve_stage(s, None, alpha, None, rhs, x_ref, o)
            x = torch.full_like(rhs, float("nan"))
            info = b.dg_solve_helmholtz_noalloc(gm.handle, alpha, rhs, x, o)
            torch.cuda.synchronize()
            assert info.status == b.DG_OK
            assert info.iterations == ref.iterations
            err = (x - x_ref).norm().item() / x_ref.norm().item()
            assert err < 1e-10, (call, err)
    finally:
        b.dg_solver_destroy(s)


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
