"""The 4096^2 heightfield (16,777,216 vertices, 33,538,050 triangles) at full
size, in the launch configuration the benchmark uses.

  * Against the oracle: tests/golden/terrain_4096_oracle_eps1e-3.txt holds
    the FP64 oracle's map at eps = 1e-3 on 4,500 seeded sample vertices
    (written offline by make_terrain_samples.py, which calls only the
    oracle).  The fused launch (toplesets built inside the window launch)
    and the two-step path must match it element by element within
    1e-5 * diameter, with the oracle's K, rho and vertex-update count.
  * Properties at the fixpoint (eps = 1e-7): d(S) = 0, every vertex
    reached, and for sampled vertices the oracle's FP64 update step
    (Sec. 3.2) applied once more from the GPU's final neighbour values may
    lower d(v) by at most 1e-5 * diameter; the paper-mode map lies above it
    (the iterates only decrease).
A cropped 256^2 heightfield of the same generator is compared with a whole
oracle map element by element.
"""
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


def gpu_map(capi, V32, F, S, eps):
    Vt = torch.from_numpy(V32).cuda()
    Ft = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    mesh = capi.ptp_mesh_create(Vt, Ft)
    tops = capi.ptp_toplesets(mesh, S)
    d = torch.empty(V32.shape[0], dtype=torch.float32, device="cuda")
    st = capi.ptp_distance(tops, capi.ptp_params_default(eps=eps), d)
    out = d.cpu().numpy()
    del tops, mesh, Vt, Ft, d
    torch.cuda.empty_cache()
    return out, st


def residuals(V, row, oa, ob, d, samples):
    r = np.empty(len(samples))
    for q, v in enumerate(samples):
        best = float(d[v])
        for c in range(row[v], row[v + 1]):
            best = min(best, oracle.update(V[v], V[oa[c]], V[ob[c]], float(d[oa[c]]), float(d[ob[c]])))
        r[q] = float(d[v]) - best
    return r


def test_cropped_terrain_matches_oracle(capi):
    V, F = meshes.terrain(256, 256, octaves=8, amplitude=0.1, seed=0)
    S = np.array([meshes.random_source(V.shape[0], 1)], dtype=np.int32)
    V32 = np.ascontiguousarray(V, dtype=np.float32)
    d, st = gpu_map(capi, V32, F, S, 1e-3)
    o = oracle.ptp(V32.astype(np.float64), F, S, eps=1e-3)
    assert st["iterations"] == o.K and st["band_updates"] == o.updates
    assert np.max(np.abs(d - o.d)) <= 1e-5 * meshes.bbox_diagonal(V)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "terrain_4096_oracle_eps1e-3.txt")


def read_golden():
    head = {}
    idx, val = [], []
    for line in open(GOLDEN):
        if line.startswith("# source"):
            t = line[1:].split()
            head = {t[q]: float(t[q + 1]) for q in range(0, len(t), 2)}
        elif not line.startswith("#"):
            a, b = line.split()
            idx.append(int(a))
            val.append(float(b))
    return head, np.array(idx), np.array(val)


@pytest.fixture(scope="module")
def terrain():
    V, F, S = meshes.terrain_4096()
    return np.ascontiguousarray(V, dtype=np.float32), F, S


def test_terrain_4096_matches_stored_oracle_samples(capi, terrain):
    V32, F, S = terrain
    head, idx, val = read_golden()
    assert int(head["source"]) == int(S[0])
    diam = meshes.bbox_diagonal(V32.astype(np.float64))
    assert abs(diam - head["diameter"]) <= 1e-12 * diam
    mesh = capi.ptp_mesh_create(torch.from_numpy(V32).cuda(), torch.from_numpy(np.ascontiguousarray(F)).cuda())
    d = torch.empty(V32.shape[0], dtype=torch.float32, device="cuda")
    p = capi.ptp_params_default(eps=1e-3)
    fused = capi.ptp_distance_from_sources(mesh, S, p, d)
    got_fused = d.cpu().numpy()[idx]
    tops = capi.ptp_toplesets(mesh, S)
    two = capi.ptp_distance(tops, p, d)
    got_two = d.cpu().numpy()[idx]
    del tops, mesh, d
    torch.cuda.empty_cache()
    for st, got in ((fused, got_fused), (two, got_two)):
        assert st["status"] == 0
        assert st["iterations"] == head["K"] and st["rho"] == head["rho"] and st["band_updates"] == head["updates"]
        err = float(np.max(np.abs(got.astype(np.float64) - val)))
        assert err <= 1e-5 * diam, f"max |dd| = {err:.3e} > {1e-5 * diam:.3e}"


def test_terrain_4096_fixpoint_properties(capi, terrain):
    V32, F, S = terrain
    n = V32.shape[0]
    diam = meshes.bbox_diagonal(V32.astype(np.float64))
    dfix, st = gpu_map(capi, V32, F, S, 1e-7)
    assert st["status"] == 0 and st["rho"] >= 2048  # at least half the lattice side
    assert dfix[S[0]] == 0.0 and np.all(np.isfinite(dfix))
    row, oa, ob = oracle.incident(n, F)
    rng = np.random.default_rng(0)
    samples = np.concatenate([rng.choice(n, 1500, replace=False),
                              np.argsort(dfix)[-200:],          # the far end of the front
                              rng.choice(np.argsort(dfix)[:5000], 300, replace=False)])  # near the source
    V64 = V32.astype(np.float64)
    r = residuals(V64, row, oa, ob, dfix, samples)
    assert r.min() >= 0.0
    assert r.max() <= 1e-5 * diam, r.max() / diam
    dpap, st2 = gpu_map(capi, V32, F, S, 1e-3)
    assert st2["status"] == 0 and st2["iterations"] <= st["iterations"]
    assert np.all(dpap >= dfix - 1e-6 * diam)
