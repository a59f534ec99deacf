"""The C-ABI library loads and exports every entry point include/dg.h
declares; the binding mirrors the header.  No GPU needed (no compute calls)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def header_functions():
    src = (ROOT / "include" / "dg.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_2107_07776_gb300.build import build
    return build()


def test_header_declares_the_call_set():
    names = header_functions()
    for required in ("dg_mesh_create", "dg_apply_momentum", "dg_apply_poisson",
                     "dg_solve_stage", "trbdf2_step"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(str(built))
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_header(built):
    from paper_2107_07776_gb300 import binding
    assert sorted(binding.SIGNATURES) == header_functions()
    for n in binding.SIGNATURES:
        assert hasattr(binding, n), n      # same-named Python wrapper


def test_host_side_argument_errors(built):
    from paper_2107_07776_gb300 import binding as b
    L = b.lib()
    assert L.dg_status_string(b.DG_EINVAL) == b"invalid argument"
    d = b.mesh_desc(4, [2, 2, 2], [0] * 3, [1] * 3, [True] * 3, 2)
    out = ctypes.c_void_p()
    assert L.dg_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == b.DG_EINVAL
    assert b"dim" in L.dg_last_error()
    d = b.mesh_desc(3, [2, 2, 2], [0] * 3, [1] * 3, [True] * 3, 7)
    assert L.dg_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == b.DG_EUNSUPPORTED
    d = b.mesh_desc(3, [0, 2, 2], [0] * 3, [1] * 3, [True] * 3, 2)
    assert L.dg_mesh_create(ctypes.byref(d), None, ctypes.byref(out)) == b.DG_EINVAL
    assert L.dg_apply_poisson(None, 1.0, None, None, None) == b.DG_EINVAL
