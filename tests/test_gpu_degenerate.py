"""Near-degenerate triangles on the GPU: the FP64 solve of the update step.

The window kernels evaluate the update step (Sec. 3.2) in FP32, except for
triangles with an angle whose squared sine is below 1e-6, which they solve
in FP64 from the positions (ring-slot vertices) or from the corner lists
(vertices with more neighbours than a one-ring slot holds).  The sliver
plane is full of such triangles -- needles and obtuse caps with squared
sines from 1e-6 down to 1e-11, and about 650 vertices that use the corner
lists -- so these tests reach both FP64 branches (the run statistics count
the FP64 solves) and require the map to match the FP64 oracle element by
element within 1e-5 of the diameter, with the same iteration count, on the
two-step path and on the fused launch.
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


@pytest.fixture(scope="module")
def sliver():
    V, F = meshes.sliver_plane()
    return np.ascontiguousarray(V, dtype=np.float32), F


def _sources(n):
    return [meshes.random_source(n, 7), 0, n // 2]


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("eps", [1e-3, 1e-7])
def test_sliver_plane_matches_oracle_through_fp64_solves(capi, sliver, which, eps):
    V32, F = sliver
    n = V32.shape[0]
    S = np.array([_sources(n)[which]], dtype=np.int32)
    ref = oracle.ptp(V32.astype(np.float64), F, S, eps=eps if eps >= 1e-3 else 1e-12)
    mesh = capi.ptp_mesh_create(torch.from_numpy(V32).cuda(), torch.from_numpy(F).cuda())
    tops = capi.ptp_toplesets(mesh, S)
    p = capi.ptp_params_default(eps=eps)
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    st = capi.ptp_distance(tops, p, d)
    d2 = torch.empty_like(d)
    st2 = capi.ptp_distance_from_sources(mesh, S, p, d2)
    diam = meshes.bbox_diagonal(V32)
    for got, s in ((d.cpu().numpy(), st), (d2.cpu().numpy(), st2)):
        assert s["status"] == 0
        assert s["fp64_solves"] > 0, s
        assert np.all(np.isfinite(got))
        err = float(np.max(np.abs(got.astype(np.float64) - ref.d)))
        assert err <= TOL_REL_DIAM * diam, f"max |dd| = {err:.3e} > {TOL_REL_DIAM * diam:.3e}"
        if eps >= 1e-3:
            assert s["iterations"] == ref.K
    # the fused launch runs the same iteration
    assert torch.equal(d, d2) and st2["iterations"] == st["iterations"]


def test_sliver_plane_counts_fp64_solves(capi, sliver):
    """The mesh has over a thousand triangles below the FP64 threshold (over a
    hundred below 1e-10), and one map solves more than a thousand in FP64."""
    V32, F = sliver
    V = V32.astype(np.float64)
    e1, e2, e3 = V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 1]]
    det = (np.cross(e1, e2) ** 2).sum(1)
    a, c, A = (e1 ** 2).sum(1), (e2 ** 2).sum(1), (e3 ** 2).sum(1)
    s2 = np.minimum(np.minimum(det / (a * c), det / (a * A)), det / (c * A))
    assert (s2 < 1e-6).sum() > 1000 and (s2 < 1e-10).sum() > 100
    n = V32.shape[0]
    mesh = capi.ptp_mesh_create(torch.from_numpy(V32).cuda(), torch.from_numpy(F).cuda())
    tops = capi.ptp_toplesets(mesh, np.array([_sources(n)[0]], dtype=np.int32))
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    st = capi.ptp_distance(tops, capi.ptp_params_default(eps=1e-3), d)
    assert st["fp64_solves"] > 1000, st
