"""Host logic of bench.py and of the accuracy report, on the CPU: the stream
schedule of the batch step and the closed-form distances the report
compares against."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_stream_schedule_is_largest_first_and_balanced():
    import bench

    sizes = [int(x) for x in np.random.default_rng(0).integers(10_000, 2_000_000, size=32)]
    order, lane_of = bench.stream_schedule(sizes, 8)
    assert sorted(order) == list(range(32)) and len(lane_of) == 32
    assert [sizes[i] for i in order] == sorted(sizes, reverse=True)
    load = [0.0] * 8
    for i in order:
        load[lane_of[i]] += math.sqrt(sizes[i])
    # greedy largest-first: no lane exceeds the mean by more than the largest job
    assert max(load) <= sum(load) / 8 + math.sqrt(max(sizes)) + 1e-9
    # and on this input it is better balanced than round-robin
    rr = [0.0] * 8
    for i in range(32):
        rr[i % 8] += math.sqrt(sizes[i])
    assert max(load) <= max(rr) + 1e-9
    # fewer jobs than lanes: one per lane
    order, lane_of = bench.stream_schedule([5, 9, 7], 8)
    assert sorted(lane_of.values()) == [0, 1, 2] and order == [1, 2, 0]


def test_accuracy_reference_distances():
    from paper_1810_08218_gb300 import accuracy, meshes

    V, F, S = meshes.flat65()
    e = accuracy._exact("flat65", V.astype(np.float64), S)
    assert e[S[0]] == 0.0
    j = (S[0] + 7) % V.shape[0]
    assert abs(e[j] - np.linalg.norm(V[j] - V[S[0]])) < 1e-15
    # on the unit sphere: 0 at the source, pi at the antipode, pi/2 on the equator
    V = np.array([[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, 1.0, 0]])
    e = accuracy._exact("sphere_l7", V, np.array([0]))
    assert np.allclose(e, [0.0, math.pi, math.pi / 2, math.pi / 2], atol=1e-12)
    assert accuracy._exact("torus_1m", V, np.array([0])) is None


def test_recorded_traffic_is_dropped_when_the_kernel_code_changes(tmp_path, monkeypatch):
    """The bench line's roofline.traffic comes from a committed ncu figure
    keyed by a hash of the window kernel's sources without comments and
    whitespace: kept across a comment edit, dropped (None) once the code
    differs from the code the capture was taken on."""
    import json
    import shutil

    import bench

    csrc = tmp_path / "paper_1810_08218_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("ptp_distance.cu", "ptp_update.cuh", "ptp_internal.cuh", "ptp_schedule.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_1810_08218_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    record = {"torus_1m": {"kernel_source_sha256": bench._kernel_source_hash(), "dram_bytes_per_launch": 123.0}}
    (tmp_path / "profiles" / "ptp_window_traffic.json").write_text(json.dumps(record))
    assert bench._traffic("torus_1m") == 123.0
    assert bench._traffic("sphere_l7") is None  # no capture recorded for it
    src = csrc / "ptp_distance.cu"
    text = src.read_text()
    src.write_text(text + "\n// a comment only\n/* and a block\n   comment */\n\n")
    assert bench._traffic("torus_1m") == 123.0
    src.write_text(text + "\nstatic int one_more_line_of_code = 1;\n")
    assert bench._traffic("torus_1m") is None
