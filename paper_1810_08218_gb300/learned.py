"""Learned iteration schedule: traces of the plain method, training with the
library's own MLP kernels, and the weight file.

All arithmetic runs in the CUDA library (window features, fused forward /
backward, Adam, inference); this module assembles the training set from the
plain method's per-iteration traces and drives the kernels.  Weights are a
flat float32 file (1313 values: W1[32][6], b1, W2[32][32], b2, W3, b3) with a
JSON header beside it.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import capi, meshes

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "schedule_mlp.f32")


def _torch():
    import torch

    return torch


def training_meshes(count: int = 200, seed: int = 0):
    """`count` seeded torus and sphere meshes of varied size and shape, one
    random source each: the training set's inputs."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        s = int(rng.integers(1 << 30))
        if q % 2 == 0:
            nu = int(rng.integers(48, 321))
            nv = int(rng.integers(48, 321))
            r = float(rng.uniform(0.25, 0.5))
            V, F = meshes.torus(nu, nv, 1.0, r, noise=float(rng.uniform(0.0, 0.02)), seed=s)
        else:
            level = int(rng.integers(3, 7))
            if rng.random() < 0.5:
                V, F = meshes.icosphere(level)
            else:
                V, F = meshes.bumpy_icosphere(level, int(rng.integers(8, 65)), float(rng.uniform(0.02, 0.08)),
                                              float(rng.uniform(0.05, 0.2)), seed=s)
        out.append((V, F, np.array([meshes.random_source(V.shape[0], s + 1)], dtype=np.int32)))
    return out


def window_trace(V, F, S, eps: float = 1e-3):
    """Features [rho, 6] and per-window iteration counts [rho] of the plain
    method on one mesh (the count of iterations whose lower bound was r)."""
    torch = _torch()
    n = V.shape[0]
    mesh = capi.ptp_mesh_create(torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(),
                                torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda())
    tops = capi.ptp_toplesets(mesh, S)
    feat = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    capi.ptp_window_features(tops, feat)
    rho = capi.ptp_toplesets_info(tops)["rho"]
    cap = 16 * rho + 64
    trace = torch.zeros(cap * capi.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    p = capi.ptp_params_default(eps=eps)
    p.trace = trace.data_ptr()
    p.trace_cap = cap
    st = capi.ptp_distance(tops, p, d)
    tr = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=capi.TRACE_DTYPE)[: st["iterations"]]
    counts = np.bincount(tr["i"], minlength=rho)[:rho].astype(np.float64)
    X = feat[: 6 * rho].cpu().numpy().reshape(rho, 6)
    return X, counts


def training_set(count: int = 200, seed: int = 0):
    """Stacked (features, log2 counts) over the training meshes; windows that
    the plain method left after a single iteration are kept too."""
    Xs, Ys = [], []
    for V, F, S in training_meshes(count, seed):
        X, c = window_trace(V, F, S)
        keep = c > 0
        Xs.append(X[keep])
        Ys.append(np.log2(c[keep]))
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


def schedule(tops, weights: np.ndarray, margin: float):
    """Device schedule [rho] for a toplesets handle (features -> MLP)."""
    torch = _torch()
    n = tops.mesh.n
    feat = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    capi.ptp_window_features(tops, feat)
    w = torch.from_numpy(np.ascontiguousarray(weights, np.float32)).cuda()
    wh = torch.empty(capi.PTP_MLP_NPARAM, dtype=torch.float16, device="cuda")
    capi.ptp_mlp_to_half(w, wh)
    sched = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = capi.ptp_toplesets_info(tops)["rho"]
    capi.ptp_mlp_infer(wh, feat, rho, sched, margin=margin)
    return sched
