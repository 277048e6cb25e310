"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Toplesets are compared exactly (levels, rho, offsets; the order inside a
topleset is unspecified, so only its validity is checked).  Distances are
compared element by element at max |d_gpu - d_oracle| <= 1e-5 * diameter
(bounding-box diagonal), the tolerance the FP32 path must meet against the
FP64 oracle.  Both sides get the same float32 vertex positions.
"""
import numpy as np
import pytest

import oracle
from paper_1810_08218_gb300 import meshes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL_DIAM = 1e-5


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


def run_gpu(capi, V, F, S, eps=1e-3, max_iter=0, trace_cap=0, ok=(0,)):
    Vt = torch.from_numpy(f32(V)).cuda()
    Ft = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    mesh = capi.ptp_mesh_create(Vt, Ft)
    tops = capi.ptp_toplesets(mesh, np.atleast_1d(S).astype(np.int32))
    d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
    trace = None
    if trace_cap:
        trace = torch.zeros(trace_cap * capi.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    p = capi.ptp_params_default(eps=eps, max_iter=max_iter)
    if trace is not None:
        p.trace = trace.data_ptr()
        p.trace_cap = trace_cap
    st = capi.ptp_distance(tops, p, d, ok=ok)
    out = {"d": d.cpu().numpy(), "stats": st, "mesh": mesh, "tops": tops}
    if trace is not None:
        out["trace"] = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=capi.TRACE_DTYPE)[: st["iterations"]]
    return out


def run_oracle(V, F, S, eps=1e-3, max_iter=0, trace=False):
    return oracle.ptp(f32(V).astype(np.float64), F, np.atleast_1d(S), eps=eps, max_iter=max_iter, trace=trace)


def assert_close(dg, do, diam, tol=TOL_REL_DIAM):
    fin = np.isfinite(do)
    assert np.array_equal(np.isfinite(dg), fin)
    err = np.max(np.abs(dg[fin].astype(np.float64) - do[fin])) if fin.any() else 0.0
    assert err <= tol * diam, f"max |dd| = {err:.3e} > {tol * diam:.3e}"
    return err


# ---------------------------------------------------------------------------
# toplesets
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["flat65", "sphere_l5", "random", "multi"])
def test_toplesets_exact(capi, name):
    if name == "flat65":
        V, F, S = meshes.flat65()
    elif name == "sphere_l5":
        V, F = meshes.icosphere(5)
        S = [meshes.random_source(V.shape[0], 3)]
    elif name == "random":
        V, F = meshes.random_planar(3000, seed=1)
        S = [17]
    else:
        V, F = meshes.grid(80, 70, jitter=0.2, seed=2)
        S = [5, 5, 900, 4000, 5599]
    n = V.shape[0]
    level, rho = oracle.toplesets(n, F, S)
    Vt = torch.from_numpy(f32(V)).cuda()
    mesh = capi.ptp_mesh_create(Vt, torch.from_numpy(F).cuda())
    tops = capi.ptp_toplesets(mesh, np.asarray(S, dtype=np.int32))
    info = capi.ptp_toplesets_info(tops)
    assert info["rho"] == rho
    assert info["n_reached"] == n
    off = info["off"].cpu().numpy()
    perm = info["perm"].cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(level, minlength=rho))]))
    for r in range(rho):
        assert np.all(level[perm[off[r]:off[r + 1]]] == r)


def test_unreachable_vertices_are_last_and_infinite(capi):
    V1, F1 = meshes.grid(12, 12, jitter=0.1, seed=4)
    V = np.concatenate([V1, V1 + [2.0, 0.0, 0.0]])
    F = np.concatenate([F1, F1 + 144]).astype(np.int32)
    r = run_gpu(capi, V, F, [3])
    info = capi.ptp_toplesets_info(r["tops"])
    assert info["n_reached"] == 144
    perm = info["perm"].cpu().numpy()
    assert set(perm[144:]) == set(range(144, 288))
    assert np.all(np.isinf(r["d"][144:]))
    o = run_oracle(V, F, [3])
    assert_close(r["d"], o.d, meshes.bbox_diagonal(V))


# ---------------------------------------------------------------------------
# distances
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_flat65(capi, eps):
    V, F, S = meshes.flat65()
    g = run_gpu(capi, V, F, S, eps=eps)
    o = run_oracle(V, F, S, eps=eps)
    assert g["stats"]["rho"] == o.rho
    assert g["d"][S[0]] == 0.0
    assert_close(g["d"], o.d, meshes.bbox_diagonal(V))
    if eps >= 1e-3:
        # at the paper's threshold no relative change lies within FP32
        # rounding of eps on this mesh, so both sides take the same band
        # decisions; at 1e-6 a change is a few FP32 ulps and the decisions
        # may legitimately differ while the distances still agree
        assert g["stats"]["band_updates"] == o.updates
        assert g["stats"]["iterations"] == o.K
    else:
        assert abs(g["stats"]["iterations"] - o.K) <= max(3, o.K // 20)


def test_planar_front_exact(capi):
    """A line of sources: the exact answer is the linear field d = x."""
    V, F = meshes.grid(65, 65, jitter=0.2, seed=1)
    S = np.arange(0, 65 * 65, 65)
    g = run_gpu(capi, V, F, S, eps=1e-7)
    assert np.max(np.abs(g["d"] - f32(V)[:, 0])) < 1e-5


def test_sphere_l7(capi):
    V, F, S = meshes.sphere_l7()
    g = run_gpu(capi, V, F, S, eps=1e-3)
    o = run_oracle(V, F, S, eps=1e-3)
    err = assert_close(g["d"], o.d, meshes.bbox_diagonal(V))
    ex = np.arccos(np.clip(f32(V).astype(np.float64) @ f32(V)[S[0]].astype(np.float64), -1, 1))
    m = ex > 0
    mape = 100 * np.mean(np.abs(g["d"][m] - ex[m]) / ex[m])
    print(f"sphere_l7: max|dd|={err:.2e} K={g['stats']['iterations']} rho={g['stats']['rho']} MAPE={mape:.3f}%")
    assert mape < 1.0
    assert g["stats"]["iterations"] == o.K


@pytest.mark.parametrize("seed", [0, 1])
def test_irregular_general_vertices(capi, seed):
    """Delaunay meshes have valences above 7, which take the corner-list
    (GENERAL) path instead of the one-ring slots."""
    V, F = meshes.random_planar(5000, seed=seed)
    S = [meshes.random_source(V.shape[0], seed)]
    g = run_gpu(capi, V, F, S, eps=1e-3)
    o = run_oracle(V, F, S, eps=1e-3)
    assert_close(g["d"], o.d, meshes.bbox_diagonal(V))


def test_multi_source_with_duplicates(capi):
    V, F = meshes.grid(90, 77, jitter=0.2, seed=7)
    S = np.array([11, 11, 3000, 6500, 6929], dtype=np.int32)
    g = run_gpu(capi, V, F, S, eps=1e-3)
    o = run_oracle(V, F, S, eps=1e-3)
    assert np.all(g["d"][S] == 0.0)
    assert_close(g["d"], o.d, meshes.bbox_diagonal(V))


def test_iteration_cap_reports_not_converged(capi):
    V, F, S = meshes.flat65()
    g = run_gpu(capi, V, F, S, eps=1e-3, max_iter=10, ok=(0, 5))
    assert g["stats"]["status"] == 5 and g["stats"]["iterations"] == 10
    o = run_oracle(V, F, S, eps=1e-3, max_iter=10)
    assert_close(g["d"], o.d, meshes.bbox_diagonal(V))


def test_band_trace_matches_oracle(capi):
    V, F = meshes.grid(40, 33, jitter=0.2, seed=9)
    S = [600]
    o = run_oracle(V, F, S, eps=1e-3, trace=True)
    g = run_gpu(capi, V, F, S, eps=1e-3, trace_cap=4 * o.K + 64)
    t = g["trace"]
    assert len(t) == o.K
    assert np.array_equal(t["i"], o.trace_i)
    assert np.array_equal(t["j"], o.trace_j)
    np.testing.assert_allclose(t["maxrel"], o.trace_maxrel, rtol=1e-2, atol=1e-6)
    adv = np.r_[o.trace_i[1:], o.rho] == o.trace_i + 1
    assert np.array_equal(t["advanced"].astype(bool), adv)
    assert np.all(t["changed"] <= t["active"]) and t["active"].sum() == g["stats"]["active_updates"]


def test_deterministic_and_host_path_identical(capi):
    V, F, S = meshes.flat65(seed=3)
    a = run_gpu(capi, V, F, S)["d"]
    b = run_gpu(capi, V, F, S)["d"]
    assert np.array_equal(a, b)
    out = np.empty(V.shape[0], dtype=np.float32)
    p = capi.ptp_params_default()
    st = capi.ptp_geodesic(f32(V), F.astype(np.int32), np.asarray(S, np.int32), p, out)
    assert st["status"] == 0
    assert np.array_equal(out, a)


def test_tiny_meshes(capi):
    # one triangle
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    F = np.array([[0, 1, 2]], dtype=np.int32)
    g = run_gpu(capi, V, F, [0])
    np.testing.assert_allclose(g["d"], [0, 1, 1], atol=1e-6)
    # every vertex a source
    V, F = meshes.grid(5, 5)
    g = run_gpu(capi, V, F, np.arange(25))
    assert np.all(g["d"] == 0.0) and g["stats"]["rho"] == 1


def test_invalid_inputs(capi):
    V, F = meshes.grid(5, 5)
    Vt = torch.from_numpy(f32(V)).cuda()
    bad = F.copy()
    bad[3, 1] = 25
    with pytest.raises(capi.PTPError) as e:
        capi.ptp_mesh_create(Vt, torch.from_numpy(bad).cuda())
    assert e.value.status == capi.PTP_ERR_INDEX
    bad = F.copy()
    bad[4, 2] = bad[4, 0]
    with pytest.raises(capi.PTPError) as e:
        capi.ptp_mesh_create(Vt, torch.from_numpy(bad).cuda())
    assert e.value.status == capi.PTP_ERR_DEGENERATE_FACE
    mesh = capi.ptp_mesh_create(Vt, torch.from_numpy(F).cuda())
    with pytest.raises(capi.PTPError) as e:
        capi.ptp_toplesets(mesh, np.array([0, 25], dtype=np.int32))
    assert e.value.status == capi.PTP_ERR_INDEX
    with pytest.raises(capi.PTPError) as e:
        capi.ptp_toplesets(mesh, np.array([], dtype=np.int32))
    assert e.value.status == capi.PTP_ERR_ARG


def test_device_wait_limit_ends_an_unfinishable_wait(capi):
    """A barrier that can never complete (sized for one CTA more than the
    grid) ends by its ~10 ms limit with PTP_ERR_TIMEOUT, and the context
    stays usable: a map right after is still correct."""
    assert capi.ptp_selftest_wait_limit(20_000_000) == capi.PTP_ERR_TIMEOUT
    V, F, S = meshes.flat65()
    g = run_gpu(capi, V, F, S)
    o = run_oracle(V, F, S)
    assert_close(g["d"], o.d, meshes.bbox_diagonal(V))
