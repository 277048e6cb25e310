"""Pins for the oracle's PTP iteration (Sec. 4.2) against what geometry and
the paper fix: exact planar fronts, Euclidean distance on flat meshes,
great-circle distance on spheres, the Dijkstra edge-path upper bound, the
order-independent fixpoint of the update operator, Jacobi invariance under
relabelling, the band bounds of Eq. upper_band / lower_band, and the
regular-grid error the paper prints (Sec. 5.2.2)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from paper_1810_08218_gb300 import meshes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dijkstra(V, F, S):
    E = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    w = np.linalg.norm(V[E[:, 0]] - V[E[:, 1]], axis=1)
    G = sp.coo_matrix((w, (E[:, 0], E[:, 1])), shape=(len(V), len(V))).tocsr()
    G = G.maximum(G.T)
    return csg.dijkstra(G, indices=np.atleast_1d(S), min_only=True)


def _mape(d, exact):
    m = exact > 0
    return 100.0 * np.mean(np.abs(d[m] - exact[m]) / exact[m])


def test_sources_zero_and_dijkstra_bound():
    for V, F in [meshes.grid(33, 29, jitter=0.2, seed=1), meshes.random_planar(700, seed=2), meshes.icosphere(3)]:
        S = [5, 17]
        r = oracle.ptp(V, F, S, eps=1e-3)
        assert r.status == oracle.OK
        assert np.all(r.d[S] == 0.0)
        dj = _dijkstra(V, F, S)
        assert np.all(r.d <= dj + 1e-12)
        assert np.all(np.isfinite(r.d))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_planar_front_is_exact(seed):
    """Sources = the whole column x = 0 of a jittered flat grid: the exact
    distance is the linear field d = x, which the planar update reproduces, so
    at a tight threshold every vertex must reach x to rounding."""
    V, F = meshes.grid(65, 65, jitter=0.2, seed=seed)
    S = np.arange(0, 65 * 65, 65)
    r = oracle.ptp(V, F, S, eps=1e-12)
    assert np.max(np.abs(r.d - V[:, 0])) < 1e-11
    # the paper's threshold stops within about eps relative of the limit
    r3 = oracle.ptp(V, F, S, eps=1e-3)
    assert np.max(np.abs(r3.d - V[:, 0])) < 3e-3


def test_flat_grid_euclidean():
    """65x65 jittered plane, centre source: the exact distance is Euclidean.
    PTP (first-order, no unfolding of obtuse triangles) must be far closer
    than the edge-path distance."""
    V, F, S = meshes.flat65()
    r = oracle.ptp(V, F, S, eps=1e-3)
    ex = np.linalg.norm(V - V[S[0]], axis=1)
    mape = _mape(r.d, ex)
    dij = _mape(_dijkstra(V, F, S), ex)
    assert mape < 2.5
    assert dij > 4 * mape
    assert r.K <= 2 * r.rho      # K about rho to 1.5 rho (Sec. 5.2)


def test_regular_grid_error_decreases_and_matches_paper_scale():
    """Refining a regular grid lowers the error (a consistent scheme), and at
    the paper's 1,002,001-vertex size the error is of the order the paper
    prints (Sec. 5.2.2); the paper's grid layout and source are not stated, so
    a factor-of-three band around its value is accepted."""
    mapes = []
    for N in (65, 129, 257):
        V, F = meshes.grid(N, N)
        S = [(N // 2) * N + N // 2]
        r = oracle.ptp(V, F, S, eps=1e-3)
        mapes.append(_mape(r.d, np.linalg.norm(V - V[S[0]], axis=1)))
    assert mapes[0] > 1.3 * mapes[1] > 1.3 * 1.3 * mapes[2]
    golden = {}
    for line in open(os.path.join(GOLDEN, "paper_regular_grid_mape.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            golden[k] = float(v)
    N = int(round(math.sqrt(golden["vertices"])))
    assert N * N == golden["vertices"]
    V, F = meshes.grid(N, N)
    S = [(N // 2) * N + N // 2]
    r = oracle.ptp(V, F, S, eps=1e-3)
    mape = _mape(r.d, np.linalg.norm(V - V[S[0]], axis=1))
    assert golden["mape_percent"] / 3 < mape < golden["mape_percent"] * 3


def test_sphere_great_circle():
    V, F = meshes.icosphere(5)
    s = meshes.random_source(V.shape[0], 0)
    r = oracle.ptp(V, F, [s], eps=1e-3)
    ex = np.arccos(np.clip(V @ V[s], -1.0, 1.0))
    assert _mape(r.d, ex) < 1.0
    assert np.max(np.abs(r.d - ex)) < 0.02
    assert r.K <= 2 * r.rho


@pytest.mark.parametrize("mesh", ["grid", "random"])
def test_fixpoint_is_order_independent(mesh):
    """Jacobi, Gauss-Seidel and random-order sweeps of the update operator
    reach one fixpoint, and PTP at a tight threshold reaches it too."""
    if mesh == "grid":
        V, F = meshes.grid(15, 13, jitter=0.2, seed=3)
    else:
        V, F = meshes.random_planar(200, seed=4)
    S = [7]
    dj, _ = oracle.relax(V, F, S, mode=0)
    dg, _ = oracle.relax(V, F, S, mode=1)
    dr1, _ = oracle.relax(V, F, S, mode=2, seed=11)
    dr2, _ = oracle.relax(V, F, S, mode=2, seed=12)
    for d in (dg, dr1, dr2):
        assert np.max(np.abs(d - dj)) < 1e-12
    r = oracle.ptp(V, F, S, eps=1e-14)
    assert np.max(np.abs(r.d - dj)) < 1e-12


def test_jacobi_iterates_do_not_depend_on_labels():
    """Each iterate d_k is a function of d_{k-1} alone (Sec. 4.2), so
    renumbering the vertices and reordering the faces must give the same
    iterates, band trace and result, bit for bit.  An in-place
    (Gauss-Seidel) sweep would depend on the numbering."""
    V, F = meshes.random_planar(400, seed=8)
    n = V.shape[0]
    S = [13]
    rng = np.random.default_rng(9)
    p = rng.permutation(n)           # new label of old vertex v is p[v]
    Vp = np.empty_like(V)
    Vp[p] = V
    Fp = p[F][rng.permutation(F.shape[0])]
    Fp = np.roll(Fp, 1, axis=1).astype(np.int32)   # same triangles, rotated corners
    a = oracle.ptp(V, F, S, eps=1e-3, trace=True, history=8)
    b = oracle.ptp(Vp, Fp, [p[S[0]]], eps=1e-3, trace=True, history=8)
    assert a.K == b.K and a.rho == b.rho and a.updates == b.updates
    assert np.array_equal(a.trace_i, b.trace_i) and np.array_equal(a.trace_j, b.trace_j)
    assert np.array_equal(a.hist[:, :], b.hist[:, p])
    assert np.array_equal(a.d, b.d[p])


def test_band_bounds_follow_the_equations():
    """Check the recorded band against Eq. upper_band (j_k = min(k, rho-1)) and
    Eq. lower_band (i advances by one exactly when every vertex of
    V_{i_{k-1}} changed by less than eps relative), from the stored iterates;
    and check that iterates never increase."""
    V, F = meshes.grid(21, 19, jitter=0.2, seed=5)
    S = [200]
    eps = 1e-3
    first = oracle.ptp(V, F, S, eps=eps)
    r = oracle.ptp(V, F, S, eps=eps, trace=True, history=first.K + 1)
    level, rho = oracle.toplesets(V.shape[0], F, S)
    assert rho == r.rho
    H = r.hist
    for k in range(1, r.K + 1):
        i_prev, j = r.trace_i[k - 1], r.trace_j[k - 1]
        assert j == min(k, rho - 1)
        assert np.all(H[k] <= H[k - 1])
        outside = ~((level >= i_prev) & (level <= j))
        assert np.array_equal(H[k][outside], H[k - 1][outside])
        Vi = np.where((level == i_prev) & ~np.isin(np.arange(V.shape[0]), S))[0]
        old, new = H[k - 1][Vi], H[k][Vi]
        ok = np.isfinite(old) & ((new == old) | (np.abs(new - old) < eps * old))
        advanced = (r.trace_i[k] if k < r.K else rho) == i_prev + 1
        assert advanced == bool(np.all(ok))
    assert r.trace_i[0] == 0


def test_not_converged_cap():
    V, F, S = meshes.flat65()
    r = oracle.ptp(V, F, S, eps=1e-3, max_iter=10)
    assert r.status == oracle.NOT_CONVERGED and r.K == 10
    level, _ = oracle.toplesets(V.shape[0], F, S)
    # after 10 iterations exactly the toplesets V_0 .. V_10 carry finite values
    assert np.array_equal(np.isfinite(r.d), level <= 10)


def test_fixed_band_variant_follows_its_rule():
    """band_mode 1 (the fixed band of the complexity analysis, Sec. 6.1): the
    lower bound after iteration k is ceil(k/2) regardless of convergence, so
    the run takes 2*rho - 1 iterations and still reaches the Dijkstra-bounded
    distances."""
    V, F, S = meshes.flat65()
    r = oracle.ptp(V, F, S, band_mode=1, trace=True)
    assert r.K == 2 * r.rho - 1
    assert np.array_equal(r.trace_i, [(k - 1 + 1) // 2 for k in range(1, r.K + 1)])
    ex = np.linalg.norm(V - V[S[0]], axis=1)
    assert _mape(r.d, ex) < 2.5
