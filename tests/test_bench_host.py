"""Host logic of bench.py that decides what a JSON line may claim (no GPU): a committed ncu
traffic figure is reported only for the kernel sources, temporal depth and sweep count it was
taken on, and every kernel family the solver can name has its source list."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _entries():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        return json.load(fh)


def test_source_lists_name_existing_files():
    csrc = os.path.join(ROOT, "paper_2505_17057_gb300", "csrc")
    for kernel, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(csrc, f)), (kernel, f)


def _split(key):
    parts = key.split(":")
    return parts[0], parts[1], parts[2] if len(parts) > 2 else "fp32"


def test_traffic_matches_only_its_capture_conditions():
    for key, e in _entries().items():
        workload, kernel, storage = _split(key)
        depth, sweeps = e.get("temporal_depth", 1), e.get("sweeps", 0)
        if e["source_sha"] != bench.kernel_source_sha(kernel):
            continue   # a stale entry is reported as null, which the next check also covers
        assert bench.traffic_from_profile(kernel, workload, depth, sweeps, storage) == e["dram_bytes_per_launch"]
        assert bench.traffic_from_profile(kernel, workload, depth + 1, sweeps, storage) is None
        assert bench.traffic_from_profile(kernel, workload, depth, sweeps + 1, storage) is None
        assert bench.traffic_from_profile(kernel, "other_workload", depth, sweeps, storage) is None
        other = "bf16" if storage == "fp32" else "fp32"
        if f"{workload}:{kernel}" + ("" if other == "fp32" else f":{other}") not in _entries():
            assert bench.traffic_from_profile(kernel, workload, depth, sweeps, other) is None


def test_traffic_is_null_once_a_source_changes(monkeypatch):
    key, e = next(iter(_entries().items()))
    workload, kernel, _ = _split(key)
    monkeypatch.setattr(bench, "kernel_source_sha", lambda k: "0" * 16)
    assert bench.traffic_from_profile(kernel, workload, e.get("temporal_depth", 1), e.get("sweeps", 0)) is None


@pytest.mark.parametrize("ranks,nodes,steps,seconds,want", [(1, 100, 10, 1.0, 1e-3), (4, 100, 10, 2.0, 2e-3)])
def test_job_mlups_counts_every_rank(ranks, nodes, steps, seconds, want):
    assert bench.job_mlups(ranks, nodes, steps, seconds) == pytest.approx(want)


def test_l2_note_and_clock_window():
    import bench
    note, bound = bench.l2_note(2 * 201_326_592, 2)      # tgv2d_4096 FP32: two 201 MB levels
    assert bound == "hbm" and "larger than L2" in note and "201 MB per level" in note
    note, bound = bench.l2_note(3 * 4_300_000, 3)        # ncde2d_1024: three 4 MB levels
    assert bound == "l2-resident" and note.startswith("L2-resident")
    assert bench.clock_window_calls(0.1364) == 7331      # about one second of 0.136 ms launches
    assert bench.clock_window_calls(5000.0) == 1         # at least one call
    assert bench.clock_window_calls(0.0) == 1_000_000    # no division by zero
