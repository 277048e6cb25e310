"""Pins for the oracle's toplesets (Sec. 4.1, Definition of V_r and its
partition properties): a library breadth-first search, the partition
properties, and the 6r ring sizes of a valence-6 lattice."""
import networkx as nx
import numpy as np
import pytest

import oracle
from paper_1810_08218_gb300 import meshes


def _graph(n, F):
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for a, b, c in F:
        G.add_edge(int(a), int(b))
        G.add_edge(int(b), int(c))
        G.add_edge(int(c), int(a))
    return G


@pytest.mark.parametrize("mesh", ["grid", "random", "sphere"])
def test_levels_match_library_bfs(mesh):
    if mesh == "grid":
        V, F = meshes.grid(23, 17, jitter=0.2, seed=4)
    elif mesh == "random":
        V, F = meshes.random_planar(600, seed=5)
    else:
        V, F = meshes.icosphere(3)
    n = V.shape[0]
    rng = np.random.default_rng(6)
    for m in (1, 3, 7):
        S = rng.integers(0, n, size=m)
        level, rho = oracle.toplesets(n, F, S)
        ref = nx.multi_source_dijkstra_path_length(_graph(n, F), set(int(s) for s in S), weight=lambda u, v, d: 1)
        expect = np.array([ref[v] for v in range(n)])
        assert np.array_equal(level, expect)
        assert rho == expect.max() + 1


def test_partition_properties():
    V, F = meshes.random_planar(800, seed=7)
    n = V.shape[0]
    level, rho = oracle.toplesets(n, F, [3, 3, 10])
    counts = np.bincount(level, minlength=rho)
    assert counts.sum() == n                      # sum |V_r| = |V|
    assert np.all(counts > 0)                     # every level 0..rho-1 is non-empty
    assert counts[0] == 2                         # V_0 = S, duplicates removed
    # every vertex of V_r (r > 0) has a neighbour in V_{r-1} and none below
    G = _graph(n, F)
    for v in range(n):
        nb = [level[w] for w in G.neighbors(v)]
        if level[v] > 0:
            assert min(nb) == level[v] - 1


def test_ring_sizes_on_valence6_lattice():
    """On the lattice with one diagonal per quad every interior vertex has
    valence 6 and the r-th ring around an interior source has 6r vertices
    until it meets the boundary."""
    N = 41
    V, F = meshes.grid(N, N)
    c = (N // 2) * N + N // 2
    level, rho = oracle.toplesets(N * N, F, [c])
    counts = np.bincount(level)
    for r in range(1, N // 2 + 1):
        assert counts[r] == 6 * r


def test_unreachable_and_errors():
    V1, F1 = meshes.grid(5, 5)
    F = np.concatenate([F1, F1 + 25]).astype(np.int32)
    level, rho = oracle.toplesets(50, F, [0])
    assert np.all(level[25:] == -1) and np.all(level[:25] >= 0)
    with pytest.raises(ValueError):
        oracle.toplesets(50, F, [50])
    with pytest.raises(ValueError):
        oracle.incident(25, np.array([[0, 1, 25]], dtype=np.int32))
    with pytest.raises(ValueError):
        oracle.incident(25, np.array([[0, 1, 1]], dtype=np.int32))
