"""Learned window schedule: traces of the plain method, training with the
library's own MLP kernels, the weight file, and plain-vs-learned runs.

The MLP predicts, for every topleset V_r, log2 of the number of iterations
after V_r enters the band (at iteration r) until it has converged, i.e. one
past the last iteration in which one of its vertices failed the relative-
change test of Eq. lower_band.  The learned multi-advance band (band_mode 2)
tests the toplesets whose predicted time has come as one group beside the
bottom topleset and retires them all when both pass; the plain band retires
at most one topleset per iteration.  Meant for fixpoint runs (eps = 1e-7),
where both give the same map within rounding.

All arithmetic runs in the CUDA library (window features, fused forward /
backward, Adam, inference, the schedule inside the fused launch); this module
assembles the training set from the plain method's convergence traces and
drives the kernels.  Weights are a flat float32 file (1313 values: W1[32][6],
b1, W2[32][32], b2, W3, b3) with a JSON header beside it.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np

from . import capi, meshes

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "schedule_mlp.f32")
FIXPOINT_EPS = 1e-7


def _torch():
    import torch

    return torch


def training_meshes(count: int = 200, seed: int = 0):
    """`count` seeded meshes of varied size and shape, one random source
    each: noisy tori, icospheres, bumpy icospheres, heightfields and jittered
    planes of 4k to 260k vertices (the training set's inputs)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        s = int(rng.integers(1 << 30))
        kind = q % 5
        if kind == 0:
            nu, nv = int(rng.integers(64, 513)), int(rng.integers(64, 513))
            V, F = meshes.torus(nu, nv, 1.0, float(rng.uniform(0.25, 0.5)), noise=float(rng.uniform(0.0, 0.02)), seed=s)
        elif kind == 1:
            V, F = meshes.icosphere(int(rng.integers(4, 8)))
        elif kind == 2:
            V, F = meshes.bumpy_icosphere(int(rng.integers(4, 8)), int(rng.integers(8, 65)),
                                          float(rng.uniform(0.02, 0.08)), float(rng.uniform(0.05, 0.2)), seed=s)
        elif kind == 3:
            side = int(rng.integers(64, 513))
            V, F = meshes.terrain(side, side, octaves=int(rng.integers(4, 9)), amplitude=float(rng.uniform(0.02, 0.2)),
                                  seed=s)
        else:
            nx, ny = int(rng.integers(64, 513)), int(rng.integers(64, 513))
            V, F = meshes.grid(nx, ny, jitter=0.2, seed=s)
        out.append((V, F, np.array([meshes.random_source(V.shape[0], s + 1)], dtype=np.int32)))
    return out


def _mesh_tops(V, F, S):
    torch = _torch()
    mesh = capi.ptp_mesh_create(torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(),
                                torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda())
    return mesh, capi.ptp_toplesets(mesh, np.ascontiguousarray(S, np.int32))


def features(tops):
    """Window features [rho, 6] of a toplesets handle (device tensor)."""
    torch = _torch()
    n = tops.mesh.n
    feat = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    capi.ptp_window_features(tops, feat)
    rho = capi.ptp_toplesets_info(tops)["rho"]
    return feat[: 6 * rho].view(rho, 6)


def window_trace(V, F, S, eps: float = FIXPOINT_EPS):
    """Features [rho - 1, 6] and convergence counts [rho - 1] of the plain
    method (band_mode 0) on one mesh, for the toplesets V_1 .. V_{rho-1}:
    count_r = (last iteration in which V_r failed the test) + 1 - r, at least 1."""
    torch = _torch()
    mesh, tops = _mesh_tops(V, F, S)
    X = features(tops)
    rho = X.shape[0]
    last = torch.full((rho,), -1, dtype=torch.int32, device="cuda")
    d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
    p = capi.ptp_params_default(eps=eps)
    p.conv_trace = last.data_ptr()
    capi.ptp_distance(tops, p, d)
    r = np.arange(rho)
    counts = np.maximum(last.cpu().numpy().astype(np.int64) + 1 - r, 1).astype(np.float64)
    return X.cpu().numpy()[1:], counts[1:]


def training_set(count: int = 200, seed: int = 0):
    """Stacked (features, log2 counts) over the training meshes."""
    Xs, Ys = [], []
    for V, F, S in training_meshes(count, seed):
        X, c = window_trace(V, F, S)
        Xs.append(X)
        Ys.append(np.log2(c))
    return np.concatenate(Xs).astype(np.float32), np.concatenate(Ys).astype(np.float32)


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style normal initialisation, zero biases."""
    rng = np.random.default_rng(seed)
    w = np.zeros(capi.PTP_MLP_NPARAM, dtype=np.float32)
    w[0:192] = rng.normal(0.0, np.sqrt(2.0 / 6), 192)
    w[224:1248] = rng.normal(0.0, np.sqrt(2.0 / 32), 1024)
    w[1280:1312] = rng.normal(0.0, np.sqrt(1.0 / 32), 32)
    return w


def train(X: np.ndarray, Y: np.ndarray, steps: int = 2000, lr: float = 3e-3, seed: int = 0, log_every: int = 0):
    """Full-batch Adam with the library's fused forward/backward kernel.
    Returns (FP32 weights, loss history)."""
    torch = _torch()
    w = torch.from_numpy(init_weights(seed)).cuda()
    wh = torch.empty(capi.PTP_MLP_NPARAM, dtype=torch.float16, device="cuda")
    capi.ptp_mlp_to_half(w, wh)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    g = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, np.float32)).cuda()
    hist = []
    for step in range(1, steps + 1):
        loss.zero_()
        capi.ptp_mlp_grad(wh, Xd, Yd, X.shape[0], g, loss)
        capi.ptp_mlp_adam(w, wh, m, v, g, lr, step)
        if log_every and (step % log_every == 0 or step == 1):
            hist.append((step, float(loss.item())))
    hist.append((steps, float(loss.item())))
    return w.cpu().numpy(), hist


def save_weights(w: np.ndarray, meta: dict, path: str = WEIGHTS) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.ascontiguousarray(w, dtype=np.float32).tofile(path)
    with open(path + ".json", "w") as f:
        json.dump(dict(meta, nparam=int(w.size), layout="W1[32][6] b1[32] W2[32][32] b2[32] W3[32] b3"), f, indent=1)


def load_weights(path: str = WEIGHTS):
    w = np.fromfile(path, dtype=np.float32)
    with open(path + ".json") as f:
        meta = json.load(f)
    assert w.size == capi.PTP_MLP_NPARAM == meta["nparam"]
    return w, meta


def half_weights(weights: np.ndarray):
    """FP16 copy of FP32 weights on the device (through the library)."""
    torch = _torch()
    w = torch.from_numpy(np.ascontiguousarray(weights, np.float32)).cuda()
    wh = torch.empty(capi.PTP_MLP_NPARAM, dtype=torch.float16, device="cuda")
    capi.ptp_mlp_to_half(w, wh)
    return wh


def schedule(tops, weights: np.ndarray, margin: float):
    """Device schedule [rho] of a toplesets handle (features -> MLP), the
    input of band_mode 2 in ptp_distance."""
    torch = _torch()
    X = features(tops)
    sched = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    capi.ptp_mlp_infer(half_weights(weights), X.contiguous(), X.shape[0], sched, margin=margin)
    return sched


def learned_params(wh, margin: float, eps: float = FIXPOINT_EPS):
    """Parameters of the learned band in ptp_distance_from_sources (the
    launch infers the schedule from the FP16 weights wh)."""
    p = capi.ptp_params_default(eps=eps, band_mode=2, mlp_margin=float(margin))
    p.mlp_half = wh.data_ptr()
    return p


def compare(V, F, S, weights: np.ndarray, margin: float, eps: float = FIXPOINT_EPS, reps: int = 10, warm: int = 2):
    """Plain band vs learned band through ptp_distance_from_sources on one
    mesh (resident), both at eps: median ms per map of `reps` runs, K, band
    updates and max |d_learned - d_plain| over the diameter."""
    torch = _torch()
    n = V.shape[0]
    V32 = np.ascontiguousarray(V, np.float32)
    mesh = capi.ptp_mesh_create(torch.from_numpy(V32).cuda(), torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda())
    Sh = np.ascontiguousarray(S, np.int32)
    wh = half_weights(weights)
    out = {}
    for name, p in (("plain", capi.ptp_params_default(eps=eps)), ("learned", learned_params(wh, margin, eps))):
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        ts = []
        st = None
        for r in range(warm + reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = capi.ptp_distance_from_sources(mesh, Sh, p, d)
            e1.record()
            e1.synchronize()
            if r >= warm:
                ts.append(e0.elapsed_time(e1))
        out[name] = {"ms": statistics.median(ts), "K": st["iterations"], "band_updates": st["band_updates"],
                     "status": st["status"], "d": d.cpu().numpy()}
    diam = meshes.bbox_diagonal(V32)
    dd = float(np.max(np.abs(out["learned"]["d"].astype(np.float64) - out["plain"]["d"])))
    res = {k: {kk: vv for kk, vv in v.items() if kk != "d"} for k, v in out.items()}
    res["max_abs_dd_over_diam"] = dd / diam
    return res
