"""GB300-native matrix-free DG TR-BDF2 solver (after Orlando et al.,
arXiv 2107.07776): CUDA kernels for sm_103a behind the C ABI of
include/dg.h, with a ctypes binding of the same names."""
from .build import build, LIB  # noqa: F401
