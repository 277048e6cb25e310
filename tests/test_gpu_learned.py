"""Learned iteration schedule: the GPU's fused MLP kernels against the FP64
reference, and the schedule's effect on PTP (with predictions that never
exceed the plain method's per-window counts the map is the plain map)."""
import numpy as np
import pytest

from oracle import mlp
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


def test_grad_and_forward_match_reference(capi):
    rng = np.random.default_rng(1)
    w32 = rng.normal(0.0, 0.3, mlp.NPARAM).astype(np.float32)
    w16 = w32.astype(np.float16)
    X = rng.uniform(0.0, 1.0, (3000, 6)).astype(np.float32)
    Y = rng.normal(3.0, 1.0, 3000).astype(np.float32)
    wh = torch.from_numpy(w16).cuda()
    g = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    capi.ptp_mlp_grad(wh, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), 3000, g, loss)
    wref = w16.astype(np.float64)  # the GPU computes with the FP16 weights
    gref = mlp.grad(wref, X, Y)
    np.testing.assert_allclose(g.cpu().numpy(), gref, rtol=2e-3, atol=2e-5 * np.abs(gref).max())
    assert abs(loss.item() - mlp.loss(wref, X, Y)) <= 1e-4 * mlp.loss(wref, X, Y)
    # inference: the schedule is floor(2^(y - margin)) clamped to [1, cap]
    sched = torch.empty(3000, dtype=torch.int32, device="cuda")
    capi.ptp_mlp_infer(wh, torch.from_numpy(X).cuda(), 3000, sched, margin=0.5, cap=1000)
    y = mlp.forward(wref, X)
    expect = np.clip(np.floor(2.0 ** (y - 0.5)), 1, 1000)
    got = sched.cpu().numpy()
    close = np.abs(2.0 ** (y - 0.5) - np.round(2.0 ** (y - 0.5))) > 1e-3  # away from integer boundaries
    assert np.array_equal(got[close], expect[close])


def test_training_lowers_the_loss(capi):
    from paper_1810_08218_gb300 import learned

    rng = np.random.default_rng(2)
    X = rng.uniform(0.0, 1.0, (2000, 6)).astype(np.float32)
    Y = (1.0 + 3.0 * X[:, 0] - 2.0 * X[:, 4] + X[:, 5] ** 2).astype(np.float32)
    w, hist = learned.train(X, Y, steps=400, lr=3e-3, log_every=100)
    assert hist[-1][1] < 0.05 * hist[0][1]
    assert mlp.loss(w.astype(np.float16).astype(np.float64), X, Y) < 0.05 * np.var(Y)


def test_schedule_at_or_below_plain_counts_gives_the_plain_map(capi):
    """Feed the plain method's own per-window counts as the schedule: every
    skipped test is one that failed in the plain run, so K, the band updates
    and the map are identical, with one test per window instead of one per
    iteration; a schedule below the counts also gives the plain map."""
    from paper_1810_08218_gb300 import learned

    V, F, S = meshes.sphere_l7()
    X, counts = learned.window_trace(V, F, S)
    n = V.shape[0]
    mesh = capi.ptp_mesh_create(torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(), torch.from_numpy(F).cuda())
    tops = capi.ptp_toplesets(mesh, S)
    d0 = torch.empty(n, dtype=torch.float32, device="cuda")
    d1 = torch.empty(n, dtype=torch.float32, device="cuda")
    s0 = capi.ptp_distance(tops, capi.ptp_params_default(), d0)
    for sch, expect_checks in ((counts, s0["rho"]), (np.maximum(counts // 2, 1), None)):
        sched = torch.from_numpy(sch.astype(np.int32)).cuda()
        p = capi.ptp_params_default()
        p.schedule = sched.data_ptr()
        s1 = capi.ptp_distance(tops, p, d1)
        assert torch.equal(d0, d1)
        assert s0["iterations"] == s1["iterations"] and s0["band_updates"] == s1["band_updates"]
        assert s1["checks"] <= s0["checks"]
        if expect_checks is not None:
            assert s1["checks"] == expect_checks
