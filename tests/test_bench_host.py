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
