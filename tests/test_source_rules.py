"""Source-level rules of the CUDA library that the compiler does not check.

Every kernel may be launched with programmatic dependent launch (the
`launch` helper sets the attribute on non-default streams), so every kernel
must wait for its predecessor (`pdl_entry()`, griddepcontrol.wait) before it
touches global memory: the first statement of every `__global__` body.
"""
import pathlib
import re

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2107_07776_gb300" / "csrc"


def kernel_bodies():
    for f in sorted(list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh"))):
        src = f.read_text()
        for m in re.finditer(r"__global__", src):
            brace = src.find("{", m.end())
            semi = src.find(";", m.end())
            if semi != -1 and semi < brace:  # a declaration
                continue
            head = src[m.end():brace]
            name = re.findall(r"(\w+)\s*\(", head)
            yield f.name, (name[-1] if name else "?"), src[brace + 1:brace + 200]


def test_every_kernel_waits_for_its_predecessor_first():
    bodies = list(kernel_bodies())
    assert len(bodies) > 50
    bad = [f"{f}:{k}" for f, k, body in bodies if not body.lstrip().startswith("pdl_entry();")]
    assert not bad, bad


def test_kernels_are_launched_through_the_launch_helper():
    # raw <<<...>>> launches would bypass the launch helper's error handling
    # and stream policy
    raw = []
    for f in sorted(list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh"))):
        for i, line in enumerate(f.read_text().splitlines(), 1):
            if "<<<" in line and not line.lstrip().startswith("//"):
                raw.append(f"{f.name}:{i}")
    assert not raw, raw
