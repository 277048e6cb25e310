"""Launch shapes of the window kernels and the autotuner.

Threads per CTA and the number of CTAs change only how the band is spread
over the GPU: every shape must give bit-identical distances, iteration
counts, band windows and per-iteration change counts.  The number of
recomputed vertices is not fixed: a vertex whose change stamp another CTA
refreshes during the same iteration is recomputed once more than needed
(from unchanged inputs, so to the same value), and how often that happens
depends on timing.
"""
import numpy as np
import pytest

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


def make_tops(capi, V, F, S):
    Vt = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).cuda()
    Ft = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    mesh = capi.ptp_mesh_create(Vt, Ft)
    return capi.ptp_toplesets(mesh, np.atleast_1d(S).astype(np.int32))


def run(capi, tops, n, params, trace_cap=0):
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    tr = None
    if trace_cap:
        tr = torch.zeros(trace_cap * capi.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        params.trace = tr.data_ptr()
        params.trace_cap = trace_cap
    st = capi.ptp_distance(tops, params, d)
    out = d.cpu().numpy()
    if tr is not None:
        tr = np.frombuffer(tr.cpu().numpy().tobytes(), dtype=capi.TRACE_DTYPE)[: st["iterations"]]
    return out, st, tr


@pytest.mark.parametrize("shape", [(256, 0), (128, 0), (512, 7), (128, 3), (64, 1), (384, 152)])
def test_every_launch_shape_gives_the_same_map(capi, shape):
    V, F = meshes.random_planar(6000, seed=11)  # irregular valences, general vertices
    S = [meshes.random_source(V.shape[0], 2), meshes.random_source(V.shape[0], 3)]
    tops = make_tops(capi, V, F, S)
    d0, st0, tr0 = run(capi, tops, V.shape[0], capi.ptp_params_default(), trace_cap=4096)
    d1, st1, tr1 = run(capi, tops, V.shape[0], capi.ptp_params_default(block=shape[0], grid=shape[1]), trace_cap=4096)
    assert np.array_equal(d0, d1)
    for k in ("iterations", "band_updates", "changed", "checks"):
        assert st0[k] == st1[k], k
    assert abs(st0["active_updates"] - st1["active_updates"]) <= 1e-3 * st0["active_updates"]
    for f in ("i", "j", "changed", "maxrel", "advanced"):
        assert np.array_equal(tr0[f], tr1[f]), f
    assert np.allclose(tr0["errsum"], tr1["errsum"], rtol=1e-12, atol=0)


def test_invalid_block_rejected(capi):
    V, F, S = meshes.flat65()
    tops = make_tops(capi, V, F, S)
    d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
    for b in (32, 100, 1024):
        with pytest.raises(capi.PTPError):
            capi.ptp_distance(tops, capi.ptp_params_default(block=b), d)


def test_autotune_single_and_batch(capi):
    V, F, S = meshes.flat65()
    tops = make_tops(capi, V, F, S)
    p = capi.ptp_params_default()
    r = capi.ptp_autotune(tops, p, reps=3)
    assert r["tried"] >= 6 and r["ms"] > 0 and r["ms"] <= r["ms_default"]
    assert (p.block, p.grid) == (r["block"], r["grid"])
    d_tuned, _, _ = run(capi, tops, V.shape[0], p)
    d_default, _, _ = run(capi, tops, V.shape[0], capi.ptp_params_default())
    assert np.array_equal(d_tuned, d_default)

    probs = meshes.uneven_batch(6, 300, 5000, seed=4)
    tl = [make_tops(capi, *q) for q in probs]
    batch = capi.ptp_batch_create(tl)
    p = capi.ptp_params_default()
    r = capi.ptp_autotune(batch, p, reps=2)
    assert r["ms"] <= r["ms_default"]
    outs = [torch.empty(q[0].shape[0], dtype=torch.float32, device="cuda") for q in probs]
    capi.ptp_distance_batch(batch, p, outs)
    for t, q, o in zip(tl, probs, outs):
        ref, _, _ = run(capi, t, q[0].shape[0], capi.ptp_params_default())
        assert np.array_equal(o.cpu().numpy(), ref)
    capi.ptp_batch_destroy(batch)
