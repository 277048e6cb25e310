"""ptp_distance_from_sources (toplesets built inside the window launch)
against ptp_toplesets + ptp_distance.

Both run the same iteration from the same toplesets, so the distances must
be bit-identical and the iteration counts, band sizes and band windows
equal; the vertex order inside a topleset (which the fused BFS assigns in
its own order) does not enter any iterate.  The single-map path is itself
checked against the FP64 oracle in test_gpu_parity.py; the 1M torus is
also compared with the oracle here.
"""
import json
import os

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


def both(capi, V, F, S, trace_cap=0, **pk):
    Vt = torch.from_numpy(f32(V)).cuda()
    Ft = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    mesh = capi.ptp_mesh_create(Vt, Ft)
    S = np.atleast_1d(np.asarray(S, dtype=np.int32))
    ok = (0, capi.PTP_ERR_NOT_CONVERGED)
    out = []
    for fused in (False, True):
        d = torch.full((V.shape[0],), -1.0, dtype=torch.float32, device="cuda")
        tr = None
        p = capi.ptp_params_default(**pk)
        if trace_cap:
            tr = torch.zeros(trace_cap * capi.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            p.trace = tr.data_ptr()
            p.trace_cap = trace_cap
        if fused:
            st = capi.ptp_distance_from_sources(mesh, S, p, d, ok=ok)
        else:
            tops = capi.ptp_toplesets(mesh, S)
            st = capi.ptp_distance(tops, p, d, ok=ok)
        if tr is not None:
            tr = np.frombuffer(tr.cpu().numpy().tobytes(), dtype=capi.TRACE_DTYPE)[: st["iterations"]]
        out.append((d.cpu().numpy(), st, tr))
    return out


def assert_same(a, b, trace=False):
    (d0, s0, t0), (d1, s1, t1) = a, b
    assert np.array_equal(d0, d1, equal_nan=True)
    for k in ("iterations", "band_updates", "rho", "status", "checks"):
        assert s0[k] == s1[k], (k, s0[k], s1[k])
    if trace:
        for f in ("i", "j", "advanced", "changed"):
            assert np.array_equal(t0[f], t1[f]), f


@pytest.mark.parametrize("name", ["flat65", "sphere_l5", "random", "multi", "two_components", "triangle", "strip"])
def test_fused_equals_two_step(capi, name):
    if name == "flat65":
        V, F, S = meshes.flat65()
    elif name == "sphere_l5":
        V, F = meshes.icosphere(5)
        S = [meshes.random_source(V.shape[0], 3)]
    elif name == "random":
        V, F = meshes.random_planar(8000, seed=5)
        S = [meshes.random_source(V.shape[0], 6)]
    elif name == "multi":
        V, F = meshes.icosphere(4)
        S = [5, 900, 5, 2000, 17]
    elif name == "strip":
        # 2000 small toplesets: the copy CTAs trail the BFS and copy many per round
        V, F = meshes.grid(2000, 4, jitter=0.1, seed=7)
        S = [0]
    elif name == "two_components":
        V1, F1 = meshes.grid(12, 12, jitter=0.1, seed=4)
        V = np.concatenate([V1, V1 + [2.0, 0.0, 0.0]])
        F = np.concatenate([F1, F1 + 144]).astype(np.int32)
        S = [3]
    else:
        V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
        F = np.array([[0, 1, 2]], dtype=np.int32)
        S = [1]
    a, b = both(capi, V, F, S, trace_cap=8192)
    assert_same(a, b, trace=True)
    if name == "two_components":
        assert np.all(np.isinf(b[0][144:]))


@pytest.mark.parametrize("pk", [dict(block=128), dict(block=256, grid=40), dict(grid=7), dict(grid=3),
                                dict(band_mode=1), dict(max_iter=9), dict(eps=1e-6)])
def test_fused_launch_shapes_and_modes(capi, pk):
    V, F = meshes.torus(96, 64, 1.0, 0.4, noise=0.01, seed=2)
    S = [meshes.random_source(V.shape[0], 8)]
    a, b = both(capi, V, F, S, **pk)
    assert_same(a, b)


def test_fused_repeated_runs_bit_identical(capi):
    """The copy CTAs must copy every topleset position exactly once, in the
    same ranges in every copy CTA, and publish a topleset only after all of
    them have copied it; the window must not read a topleset before that.
    A range that differed between copy CTAs (a position remapped twice, or
    never) changed most distances of a map this size, and did so on some
    runs only, so the fused map is repeated and compared with the two-step
    map bit for bit each time."""
    V, F = meshes.torus(768, 512, 1.0, 0.4, noise=0.01, seed=3)
    S = [meshes.random_source(V.shape[0], 11)]
    ref, first = both(capi, V, F, S)
    assert_same(ref, first)
    Vt = torch.from_numpy(f32(V)).cuda()
    Ft = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    mesh = capi.ptp_mesh_create(Vt, Ft)
    for _ in range(4):
        d = torch.full((V.shape[0],), -1.0, dtype=torch.float32, device="cuda")
        st = capi.ptp_distance_from_sources(mesh, np.asarray(S, dtype=np.int32), capi.ptp_params_default(), d)
        assert_same(ref, (d.cpu().numpy(), st, None))


def test_fused_torus_1m_against_oracle(capi):
    V, F, S = meshes.torus_1m()
    a, b = both(capi, V, F, S)
    assert_same(a, b)
    with open(os.path.join(os.path.dirname(oracle.__file__), "workload_counts.json")) as f:
        c = json.load(f)["torus_1m"]
    assert b[1]["iterations"] == c["K"] and b[1]["rho"] == c["rho"] and b[1]["band_updates"] == c["updates"]


def test_fused_argument_errors(capi):
    V, F, S = meshes.flat65()
    mesh = capi.ptp_mesh_create(torch.from_numpy(f32(V)).cuda(), torch.from_numpy(F).cuda())
    d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
    with pytest.raises(capi.PTPError):
        capi.ptp_distance_from_sources(mesh, [V.shape[0]], capi.ptp_params_default(), d)
    p = capi.ptp_params_default()
    sched = torch.ones(100, dtype=torch.int32, device="cuda")
    p.schedule = sched.data_ptr()
    with pytest.raises(capi.PTPError):
        capi.ptp_distance_from_sources(mesh, S, p, d)
    # an empty source list, and a mesh with no faces
    with pytest.raises(capi.PTPError) as e:
        capi.ptp_distance_from_sources(mesh, np.array([], dtype=np.int32), capi.ptp_params_default(), d)
    assert e.value.status == capi.PTP_ERR_ARG
    with pytest.raises(capi.PTPError) as e:
        capi.ptp_mesh_create(torch.from_numpy(f32(V)).cuda(), torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    assert e.value.status == capi.PTP_ERR_ARG


def test_fused_device_sources_and_geodesic(capi):
    """Device source lists (validated on the host after a copy) and
    ptp_geodesic (mesh + fused launch) give the same map."""
    V, F = meshes.icosphere(5)
    S = np.array([11, 4000, 11], dtype=np.int32)
    mesh = capi.ptp_mesh_create(torch.from_numpy(f32(V)).cuda(), torch.from_numpy(F).cuda())
    d_host = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
    d_dev = torch.empty_like(d_host)
    capi.ptp_distance_from_sources(mesh, S, capi.ptp_params_default(), d_host)
    capi.ptp_distance_from_sources(mesh, torch.from_numpy(S).cuda(), capi.ptp_params_default(), d_dev)
    assert torch.equal(d_host, d_dev)
    tops = capi.ptp_toplesets(mesh, S)
    d_two = torch.empty_like(d_host)
    capi.ptp_distance(tops, capi.ptp_params_default(), d_two)
    assert torch.equal(d_host, d_two)
    out = np.empty(V.shape[0], dtype=np.float32)
    st = capi.ptp_geodesic(f32(V), F, S, capi.ptp_params_default(), out)
    assert st["status"] == 0 and np.array_equal(out, d_host.cpu().numpy())


def test_pool_reuse_and_release(capi):
    """Buffers reused from the library's pool, and buffers mapped again after
    ptp_release_memory, give the same map."""
    V, F = meshes.icosphere(5)
    S = np.array([7], dtype=np.int32)
    mesh = capi.ptp_mesh_create(torch.from_numpy(f32(V)).cuda(), torch.from_numpy(F).cuda())
    outs = []
    for r in range(3):
        d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
        capi.ptp_distance_from_sources(mesh, S, capi.ptp_params_default(), d)
        outs.append(d)
        if r == 1:
            torch.cuda.synchronize()
            capi.ptp_release_memory()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
