"""Multi-source maps in the original vertex order (the path the paper uses for
multi-source problems, Sec. 5.1 and 6.1.5): geodesic Voronoi regions and farthest-point
sampling (Sec. 5.3, App. A), and the fixed-band variant (Sec. 6.1), against the
FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1810_08218_gb300 import meshes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_08218_gb300 import build, capi as c

    build.build()
    c.load()
    return c


def f32(V):
    return np.ascontiguousarray(V, dtype=np.float32)


def mesh_of(capi, V, F):
    return capi.ptp_mesh_create(torch.from_numpy(f32(V)).cuda(), torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda())


def test_fixed_band_matches_oracle(capi):
    for V, F, S in [meshes.flat65(), meshes.sphere_l7()]:
        mesh = mesh_of(capi, V, F)
        tops = capi.ptp_toplesets(mesh, S)
        d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
        st = capi.ptp_distance(tops, capi.ptp_params_default(band_mode=1), d)
        o = oracle.ptp(f32(V).astype(np.float64), F, S, band_mode=1)
        assert st["iterations"] == o.K == 2 * o.rho - 1
        assert st["band_updates"] == o.updates
        err = np.max(np.abs(d.cpu().numpy() - o.d))
        assert err <= TOL * meshes.bbox_diagonal(f32(V))


@pytest.mark.parametrize("name", ["sphere", "plane"])
def test_voronoi_distances_and_labels(capi, name):
    if name == "sphere":
        V, F = meshes.bumpy_icosphere(5, 64, 0.05, 0.1, seed=2)
    else:
        V, F = meshes.grid(120, 100, jitter=0.2, seed=3)
    n = V.shape[0]
    rng = np.random.default_rng(4)
    seeds = rng.choice(n, size=16, replace=False).astype(np.int32)
    mesh = mesh_of(capi, V, F)
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    st = capi.ptp_voronoi(mesh, seeds, capi.ptp_params_default(), d, lab)
    assert st["status"] == 0
    d = d.cpu().numpy()
    lab = lab.cpu().numpy()
    V64 = f32(V).astype(np.float64)
    diam = meshes.bbox_diagonal(f32(V))
    # the distance is the oracle's multi-source PTP map
    om = oracle.ptp(V64, F, seeds)
    assert np.max(np.abs(d - om.d)) <= TOL * diam
    assert np.array_equal(lab[seeds], np.arange(16))
    # labels: the nearest seed by the per-seed maps wherever that is clear
    per = np.stack([oracle.ptp(V64, F, [s]).d for s in seeds])
    order = np.sort(per, axis=0)
    clear = (order[1] - order[0]) > 5e-3 * diam
    best = np.argmin(per, axis=0)
    agree = lab[clear] == best[clear]
    assert agree.mean() > 0.995, agree.mean()
    assert clear.mean() > 0.8


@pytest.mark.parametrize("graph", [False, True])
def test_fps_samples_are_farthest(capi, graph):
    V, F = meshes.bumpy_icosphere(4, 64, 0.05, 0.1, seed=5)
    n = V.shape[0]
    ns = 24
    mesh = mesh_of(capi, V, F)
    samples = torch.empty(ns, dtype=torch.int32, device="cuda")
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    st = capi.ptp_fps(mesh, 7, ns, capi.ptp_params_default(), samples, d, use_graph=graph)
    assert st["status"] == 0
    s = samples.cpu().numpy()
    assert s[0] == 7 and len(set(s.tolist())) == ns
    V64 = f32(V).astype(np.float64)
    diam = meshes.bbox_diagonal(f32(V))
    for i in range(1, ns):
        o = oracle.ptp(V64, F, s[:i]).d
        # the chosen vertex is a farthest one under the oracle's map
        assert o[s[i]] >= o.max() - TOL * diam, (i, o[s[i]], o.max())
    final = oracle.ptp(V64, F, s).d
    assert np.max(np.abs(d.cpu().numpy() - final)) <= TOL * diam


def test_fps_graph_and_stream_paths_agree(capi):
    V, F = meshes.icosphere(5)
    mesh = mesh_of(capi, V, F)
    a = torch.empty(40, dtype=torch.int32, device="cuda")
    b = torch.empty(40, dtype=torch.int32, device="cuda")
    sa = capi.ptp_fps(mesh, 3, 40, capi.ptp_params_default(), a, use_graph=False)
    sb = capi.ptp_fps(mesh, 3, 40, capi.ptp_params_default(), b, use_graph=True)
    assert torch.equal(a, b)
    assert sa["iterations"] == sb["iterations"] and sa["band_updates"] == sb["band_updates"]


@pytest.mark.parametrize("name,band_mode", [("bumpy", 0), ("delaunay", 0), ("bumpy", 1)])
def test_fused_and_two_step_multi_source_agree(capi, name, band_mode):
    """Voronoi and FPS maps as one fused launch (the default) and, on a grid
    too small to split (3 CTAs), as the BFS followed by the window: the same
    iterates, so identical distances, labels and samples, with the adaptive
    and the fixed band.  The Delaunay mesh has vertices updated from their
    corner lists (no ring slot)."""
    if name == "bumpy":
        V, F = meshes.bumpy_icosphere(5, 64, 0.05, 0.1, seed=6)
    else:
        V, F = meshes.random_planar(20000, seed=8)
    n = V.shape[0]
    mesh = mesh_of(capi, V, F)
    seeds = np.random.default_rng(7).choice(n, size=12, replace=False).astype(np.int32)
    runs = []
    for grid in (0, 3):
        p = capi.ptp_params_default(grid=grid, band_mode=band_mode)
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        sv = capi.ptp_voronoi(mesh, seeds, p, d, lab)
        smp = torch.empty(20, dtype=torch.int32, device="cuda")
        df = torch.empty(n, dtype=torch.float32, device="cuda")
        sf = capi.ptp_fps(mesh, 11, 20, p, smp, df, use_graph=True)
        assert sv["status"] == 0 and sf["status"] == 0
        runs.append((d, lab, sv, smp, df, sf))
    (d0, l0, v0, s0, f0, p0), (d1, l1, v1, s1, f1, p1) = runs
    assert torch.equal(d0, d1) and torch.equal(l0, l1)
    assert v0["iterations"] == v1["iterations"] and v0["band_updates"] == v1["band_updates"]
    assert torch.equal(s0, s1) and torch.equal(f0, f1)
    assert p0["iterations"] == p1["iterations"] and p0["band_updates"] == p1["band_updates"]
