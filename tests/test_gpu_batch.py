"""Batched maps (one persistent launch for many meshes) against single maps.

Each map of a batch follows its own window, so its distances must equal,
bit for bit, those ptp_distance computes for it alone; the single-map path
is itself checked against the FP64 oracle elsewhere, and one batch here is
also compared with the oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_1810_08218_gb300 import meshes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def make_tops(capi, V, F, S):
    Vt = torch.from_numpy(f32(V)).cuda()
    Ft = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    mesh = capi.ptp_mesh_create(Vt, Ft)
    return capi.ptp_toplesets(mesh, np.atleast_1d(S).astype(np.int32))


def problems():
    out = meshes.uneven_batch(10, 200, 30000, seed=1)
    # two components: the second is unreachable (distances +inf)
    V1, F1 = meshes.grid(12, 12, jitter=0.1, seed=4)
    out.append((np.concatenate([V1, V1 + [2.0, 0.0, 0.0]]), np.concatenate([F1, F1 + 144]).astype(np.int32),
                np.array([3], dtype=np.int32)))
    # several sources, one repeated
    V, F = meshes.icosphere(4)
    out.append((V, F, np.array([5, 900, 5, 2000], dtype=np.int32)))
    # irregular valences (general vertices)
    V, F = meshes.random_planar(3000, seed=2)
    out.append((V, F, np.array([meshes.random_source(V.shape[0], 9)], dtype=np.int32)))
    # a single triangle
    out.append((np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64), np.array([[0, 1, 2]], dtype=np.int32),
                np.array([0], dtype=np.int32)))
    return out


def run_single(capi, tops, n, params, ok=(0,)):
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    st = capi.ptp_distance(tops, params, d, ok=ok)
    return d.cpu().numpy(), st


def run_batch(capi, tops, sizes, params, ok=(0,)):
    batch = capi.ptp_batch_create(tops)
    outs = [torch.full((n,), -1.0, dtype=torch.float32, device="cuda") for n in sizes]
    st = capi.ptp_distance_batch(batch, params, outs, ok=ok)
    capi.ptp_batch_destroy(batch)
    return [o.cpu().numpy() for o in outs], st


@pytest.mark.parametrize("band_mode", [0, 1])
def test_batch_equals_single_maps(capi, band_mode):
    probs = problems()
    tops = [make_tops(capi, *p) for p in probs]
    sizes = [p[0].shape[0] for p in probs]
    params = capi.ptp_params_default(band_mode=band_mode)
    outs, bst = run_batch(capi, tops, sizes, params)
    for b, (t, n) in enumerate(zip(tops, sizes)):
        d, st = run_single(capi, t, n, params)
        assert np.array_equal(outs[b], d, equal_nan=True), f"map {b}"
        assert bst[b]["iterations"] == st["iterations"], b
        assert bst[b]["band_updates"] == st["band_updates"], b
        assert bst[b]["rho"] == st["rho"], b
        assert bst[b]["status"] == 0


def test_batch_against_oracle(capi):
    probs = meshes.uneven_batch(4, 500, 5000, seed=7)
    tops = [make_tops(capi, *p) for p in probs]
    outs, bst = run_batch(capi, tops, [p[0].shape[0] for p in probs], capi.ptp_params_default())
    for b, (V, F, S) in enumerate(probs):
        o = oracle.ptp(f32(V).astype(np.float64), F, S)
        assert bst[b]["iterations"] == o.K
        fin = np.isfinite(o.d)
        assert np.array_equal(np.isfinite(outs[b]), fin)
        err = np.max(np.abs(outs[b][fin].astype(np.float64) - o.d[fin]))
        assert err <= 1e-5 * meshes.bbox_diagonal(V), (b, err)


def test_batch_iteration_cap(capi):
    probs = meshes.uneven_batch(4, 300, 3000, seed=3)
    tops = [make_tops(capi, *p) for p in probs]
    sizes = [p[0].shape[0] for p in probs]
    params = capi.ptp_params_default(max_iter=6)
    outs, bst = run_batch(capi, tops, sizes, params, ok=(0, capi.PTP_ERR_NOT_CONVERGED))
    for b, (t, n) in enumerate(zip(tops, sizes)):
        d, st = run_single(capi, t, n, params, ok=(0, capi.PTP_ERR_NOT_CONVERGED))
        assert np.array_equal(outs[b], d, equal_nan=True)
        assert bst[b]["status"] == st["status"]
        assert bst[b]["iterations"] == st["iterations"]


def test_batch_of_one_and_of_max_size_and_small_grid(capi):
    probs = meshes.uneven_batch(capi.PTP_BATCH_MAX, 30, 400, seed=5)
    tops = [make_tops(capi, *p) for p in probs]
    sizes = [p[0].shape[0] for p in probs]
    params = capi.ptp_params_default()
    single = [run_single(capi, t, n, params)[0] for t, n in zip(tops, sizes)]
    outs, _ = run_batch(capi, tops, sizes, params)
    assert all(np.array_equal(a, b) for a, b in zip(outs, single))
    outs, _ = run_batch(capi, tops[7:8], sizes[7:8], params)
    assert np.array_equal(outs[0], single[7])
    small = capi.ptp_params_default(grid=3)
    outs, _ = run_batch(capi, tops[:5], sizes[:5], small)
    assert all(np.array_equal(a, b) for a, b in zip(outs, single[:5]))


def test_batch_argument_errors(capi):
    probs = meshes.uneven_batch(2, 100, 200, seed=6)
    tops = [make_tops(capi, *p) for p in probs]
    with pytest.raises(capi.PTPError):
        capi.ptp_batch_create(tops * 17)  # 34 > PTP_BATCH_MAX
    batch = capi.ptp_batch_create(tops)
    p = capi.ptp_params_default()
    trace = torch.zeros(64 * capi.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    p.trace = trace.data_ptr()
    p.trace_cap = 64
    outs = [torch.empty(t.mesh.n, dtype=torch.float32, device="cuda") for t in tops]
    with pytest.raises(capi.PTPError):
        capi.ptp_distance_batch(batch, p, outs)
    capi.ptp_batch_destroy(batch)
