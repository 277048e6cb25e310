"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (default parameters: 512-thread CTAs, every
co-resident CTA).

* noisy torus 1024^2 (1,048,576 vertices): the fused launch against the FP64
  oracle element by element (max |dd| <= 1e-5 * diameter), with the oracle's
  K, rho and band updates;
* bumpy level-8 icosphere (655,362 vertices): 1,000-sample farthest-point
  sampling (captured CUDA graph), each checked sample a farthest vertex of
  the oracle's map from the samples before it, and the final map; the
  64-seed Voronoi map against the oracle's multi-source map;
* the uneven batch of 32 meshes (9,007,687 vertices): every map bit-identical
  to its single-map run, the smallest also against the oracle;
* the learned schedule on the torus: the plain map, K and band updates.
"""
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
    return capi.ptp_mesh_create(torch.from_numpy(f32(V)).cuda(), torch.from_numpy(np.ascontiguousarray(F)).cuda())


def test_torus_1m_fused_against_oracle(capi):
    V, F, S = meshes.torus_1m()
    V32 = f32(V)
    mesh = mesh_of(capi, V32, F)
    d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
    st = capi.ptp_distance_from_sources(mesh, S, capi.ptp_params_default(), d)
    o = oracle.ptp(V32.astype(np.float64), F, S, eps=1e-3)
    assert st["iterations"] == o.K and st["rho"] == o.rho and st["band_updates"] == o.updates
    err = np.max(np.abs(d.cpu().numpy().astype(np.float64) - o.d))
    assert err <= TOL * meshes.bbox_diagonal(V32), err


def test_bumpy_l8_fps_1000_and_voronoi_64(capi):
    V, F, S = meshes.bumpy_l8()
    V32 = f32(V)
    V64 = V32.astype(np.float64)
    n = V.shape[0]
    diam = meshes.bbox_diagonal(V32)
    mesh = mesh_of(capi, V32, F)
    ns = 1000
    samples = torch.empty(ns, dtype=torch.int32, device="cuda")
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    st = capi.ptp_fps(mesh, int(S[0]), ns, capi.ptp_params_default(), samples, d, use_graph=True)
    assert st["status"] == 0
    s = samples.cpu().numpy()
    assert s[0] == S[0] and len(set(s.tolist())) == ns
    for i in (1, 10, 100, 999):
        o = oracle.ptp(V64, F, s[:i]).d
        assert o[s[i]] >= o.max() - TOL * diam, (i, o[s[i]], o.max())
    final = oracle.ptp(V64, F, s).d
    assert np.max(np.abs(d.cpu().numpy() - final)) <= TOL * diam
    # 64-seed Voronoi from the first 64 samples
    dv = torch.empty(n, dtype=torch.float32, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    capi.ptp_voronoi(mesh, samples[:64], capi.ptp_params_default(), dv, lab)
    ov = oracle.ptp(V64, F, s[:64]).d
    assert np.max(np.abs(dv.cpu().numpy() - ov)) <= TOL * diam
    lab = lab.cpu().numpy()
    assert lab.min() >= 0 and lab.max() < 64
    assert np.array_equal(lab[s[:64]], np.arange(64))  # every seed labels itself
    assert len(np.unique(lab)) == 64  # every region is non-empty


def test_uneven_batch32_full_size(capi):
    probs = meshes.uneven_batch(32, seed=0)
    tops = [capi.ptp_toplesets(mesh_of(capi, V, F), S) for V, F, S in probs]
    sizes = [V.shape[0] for V, _, _ in probs]
    batch = capi.ptp_batch_create(tops)
    outs = [torch.empty(k, dtype=torch.float32, device="cuda") for k in sizes]
    bst = capi.ptp_distance_batch(batch, capi.ptp_params_default(), outs)
    capi.ptp_batch_destroy(batch)
    for b, (t, k) in enumerate(zip(tops, sizes)):
        d = torch.empty(k, dtype=torch.float32, device="cuda")
        st = capi.ptp_distance(t, capi.ptp_params_default(), d)
        assert torch.equal(outs[b], d), b
        assert bst[b]["iterations"] == st["iterations"] and bst[b]["band_updates"] == st["band_updates"], b
    small = int(np.argmin(sizes))
    V, F, S = probs[small]
    o = oracle.ptp(f32(V).astype(np.float64), F, S)
    assert bst[small]["iterations"] == o.K
    assert np.max(np.abs(outs[small].cpu().numpy() - o.d)) <= TOL * meshes.bbox_diagonal(f32(V))


def test_learned_band_torus_1m_gains_at_the_same_map(capi):
    """The benchmark mesh (not in the training set) in fixpoint mode through
    the fused launch: the learned multi-advance band needs fewer iterations
    and band updates than the plain band and gives the same map within
    1e-5 * diameter."""
    from paper_1810_08218_gb300 import learned

    w, meta = learned.load_weights()
    V, F, S = meshes.torus_1m()
    r = learned.compare(V, F, S, w, meta["margin"], reps=3, warm=1)
    assert r["plain"]["status"] == 0 and r["learned"]["status"] == 0
    assert r["learned"]["K"] < r["plain"]["K"] and r["learned"]["band_updates"] < r["plain"]["band_updates"], r
    assert r["max_abs_dd_over_diam"] <= TOL
