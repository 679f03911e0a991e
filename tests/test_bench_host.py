"""Host logic of bench.py's roofline object (no GPU): which stage it describes,
its arithmetic, and that the ncu-recorded traffic and instruction count are only
reported while the kernel's sources hash to the captured ones."""
import json
import os

import pytest

import bench


def _split(**ms):
    base = dict(setup=0.0, project=0.0, emit=0.0, tile_sort=0.0, composite_fwd=0.0, loss=0.0, composite_bwd=0.0,
                project_bwd=0.0, composite_step=0.0)
    base.update(ms)
    return base


COUNTERS = (1000, 5000, 36_000_000, 36_000_000, 1_000_000, 900_000, 800_000, 10)


def test_fused_step_roofline_arithmetic():
    peaks = {"sm_max_mhz": 2070.0, "hbm_gbs": 6689.5}
    line = bench.roofline(_split(composite_step=0.3, project_bwd=0.05), COUNTERS, peaks, "measured", {}, 300_000, 16)
    assert line["kernel"] == "composite_step" and line["bound"] == "alu" and line["unit"] == "TFLOP/s"
    flops = 36e6 * bench.FLOPS_PER_EVAL_FWD + 36e6 * bench.FLOPS_PER_EVAL_BWD
    ach = flops / 0.3e-3 / 1e12
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert line["achieved"] == pytest.approx(ach, abs=1e-3)
    assert line["peak"] == pytest.approx(peak, abs=1e-2)
    assert line["frac"] == pytest.approx(ach / peak, abs=1e-4)
    assert line["blended_per_s"] == pytest.approx(72e6 / 0.3e-3 / 1e9, abs=1e-3)
    assert line["time_ms"] == pytest.approx(0.3)


def test_separate_backward_roofline_counts_the_backward_only():
    line = bench.roofline(_split(composite_fwd=0.1, composite_bwd=0.2), COUNTERS, {"sm_max_mhz": 2070.0}, "m", {}, 300_000, 16)
    assert line["kernel"] == "composite_bwd"
    assert line["achieved"] == pytest.approx(36e6 * bench.FLOPS_PER_EVAL_BWD / 0.2e-3 / 1e12, abs=1e-3)


def test_memory_stage_on_top_reports_the_hbm_peak():
    line = bench.roofline(_split(project_bwd=0.5, composite_step=0.1), COUNTERS, {"hbm_gbs": 6689.5}, "measured", {}, 300_000, 16)
    assert line["kernel"] == "project_bwd" and line["bound"] == "hbm" and line["peak"] == 6689.5


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    """The traffic and instruction count of the committed capture are returned while
    the sources hash to the recorded value, and dropped (None) once they differ."""
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    import hashlib
    rec = {"k": {"stage": "composite_step", "dram_bytes_per_launch": 123, "sources": ["k.cu"],
                 "sources_sha256": hashlib.sha256(b"kernel v1\n").hexdigest(),
                 "warp_instructions_per_launch": 456}}
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._dram_traffic("composite_step") == 123
    assert bench._capture("composite_step", "warp_instructions_per_launch") == 456
    assert bench._dram_traffic("composite_bwd") is None  # no record for that stage
    line = bench.roofline(_split(composite_step=0.3), COUNTERS, {"sm_max_mhz": 2070.0}, "m", {}, 300_000, 16)
    assert line["traffic"] == 123
    assert line["issue"]["achieved"] == pytest.approx(456 / 0.3e-3 / 1e12, abs=1e-4)
    src.write_text("kernel v2\n")  # the kernel changed since the capture
    assert bench._dram_traffic("composite_step") is None
    line = bench.roofline(_split(composite_step=0.3), COUNTERS, {"sm_max_mhz": 2070.0}, "m", {}, 300_000, 16)
    assert line["traffic"] is None and "issue" not in line



def test_every_stage_has_a_roofline_entry():
    """Each stage of the split gets its own entry: the memory-bound ones with the
    survey's algorithmic bytes over the stage time against the measured HBM peak."""
    peaks = {"sm_max_mhz": 2070.0, "hbm_gbs": 6791.0}
    split = _split(setup=0.008, project=0.04, emit=0.02, tile_sort=0.04, composite_step=0.3, project_bwd=0.05)
    line = bench.roofline(split, COUNTERS, peaks, "measured", {}, 300_000, 16)
    st = line["stages"]
    assert set(st) == {"project", "emit", "tile_sort", "composite_step", "project_bwd"}
    N, V, P, K = 300_000, COUNTERS[0], COUNTERS[1], 16
    want = {"project": 12 * N + 224 * V + 48 * V, "emit": 24 * V + 12 * P, "tile_sort": 24 * P,
            "project_bwd": 276 * V + 236 * V}
    for k, b in want.items():
        assert st[k]["algorithmic_bytes"] == b and st[k]["bound"] == "hbm" and st[k]["unit"] == "GB/s"
        ach = b / (split[k] * 1e-3) / 1e9
        assert st[k]["achieved"] == pytest.approx(ach, abs=0.05)
        assert st[k]["frac"] == pytest.approx(ach / 6791.0, abs=1e-4)
    assert line["kernel"] == "composite_step" and st["composite_step"]["bound"] == "alu"
