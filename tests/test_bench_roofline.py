"""The bench line's roofline record, checked on the host (no GPU): the
algorithmic work of the momentum apply, and the rule that a recorded ncu
DRAM figure is reported only for the kernel sources it was captured on."""
from types import SimpleNamespace

import pytest

import bench
import workloads as W


def _channel_mesh():
    w = W.WORKLOADS["channel"]
    cells = 1
    for n in w.n:
        cells *= n
    nb = (w.degree + 1) ** w.dim
    return w, SimpleNamespace(n_cells=cells, n_dofs_u=w.dim * nb * cells)


def test_flop_model_of_the_momentum_apply_is_140_per_dof():
    # Q2 in 3D with advection: 140 flop per velocity DoF (27 nodes a cell)
    assert bench.apply_flops_per_cell(3, 3, True) / 27 == pytest.approx(3780 / 27)
    assert bench.apply_flops_per_cell(3, 3, True) == 2 * (2 * 3 * 81 + 27 + 3 * 9 * 34 + 2 * 3 * 27 + 3 * 9 * 11)


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    w, mesh = _channel_mesh()
    tune = [{"op": "momentum+advection", "precision": "f64", "chosen_variant": 6,
             "face_once": [0, 0, 0, 0, 0, 1, 1, 0]}]
    rec = bench.NCU_TRAFFIC["channel"][6]
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: rec["sha"])
    r = bench.roofline(w, mesh, tune, {"momentum_fp64": 4.1})
    assert r["traffic"] == rec["bytes"]
    # the face-once apply moves more than its algorithmic bytes, never less
    assert r["traffic"] >= r["traffic_algorithmic"] == 24 * mesh.n_dofs_u
    assert 0 < r["frac"] < 1 and r["bound"] == "alu"
    assert "cell_split_nc_kernel" in r["kernel"]
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: "0" * 16)
    assert bench.roofline(w, mesh, tune, {"momentum_fp64": 4.1})["traffic"] is None
    # another variant than the one captured: no figure either
    tune[0]["chosen_variant"] = 5
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: rec["sha"])
    assert bench.roofline(w, mesh, tune, {"momentum_fp64": 4.1})["traffic"] is None

