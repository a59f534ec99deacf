"""Plain FP64 CPU oracle for the DG TR-BDF2 projection solver of Orlando et al.,
"An efficient and accurate implicit DG solver for the incompressible
Navier-Stokes equations" (arXiv 2107.07776).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package.  It shares no code with the
CUDA library: operators are assembled by naive quadrature over basis-function
pairs (``dg_oracle.c``) and systems are solved by library sparse solvers.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute-force integrals and the paper's
printed convergence tables.
"""
from .dg import Mesh, BlockOp, KIND  # noqa: F401
from .trbdf2 import Stepper, extrapolate_stage1, extrapolate_stage2  # noqa: F401
