"""Train the learned iteration schedule and evaluate it.

  python -m paper_1810_08218_gb300.train_schedule [--meshes 200] [--steps 3000] [--out DIR]

1. Runs the plain method with traces on `--meshes` seeded torus and sphere
   meshes and collects, per topleset window, the six window features and
   log2 of the number of iterations the band's lower bound stayed there.
2. Trains the MLP with the library's fused forward/backward and Adam kernels.
3. Picks the safety margin on held-out meshes: the smallest margin with at
   most 1% of windows predicted above the plain count (a prediction above
   the plain count is the only way the schedule can change the map).
4. Saves the weights (flat float32 + JSON header) and reports, on the 1M
   noisy torus, plain vs learned: iterations, band updates, tests of
   Eq. lower_band, ms per map and max |d_learned - d_plain|.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1810_08218_gb300 import build, capi, learned, meshes  # noqa: E402


def evaluate(weights, margin, V, F, S, reps=10):
    import torch

    n = V.shape[0]
    mesh = capi.ptp_mesh_create(torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(), torch.from_numpy(F).cuda())
    tops = capi.ptp_toplesets(mesh, S)
    sched = learned.schedule(tops, weights, margin)
    out = {}
    for name, sch in (("plain", None), ("learned", sched)):
        p = capi.ptp_params_default()
        if sch is not None:
            p.schedule = sch.data_ptr()
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        st = capi.ptp_distance(tops, p, d)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            ev0.record()
            capi.ptp_distance(tops, p, d, stats=False)
            ev1.record()
            torch.cuda.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        out[name] = {"d": d.cpu().numpy(), "ms": float(np.median(ts)), "K": st["iterations"],
                     "band_updates": st["band_updates"], "checks": st["checks"]}
    diam = meshes.bbox_diagonal(np.asarray(V, np.float32))
    dd = float(np.max(np.abs(out["learned"]["d"].astype(np.float64) - out["plain"]["d"])))
    return {k: {kk: vv for kk, vv in v.items() if kk != "d"} for k, v in out.items()} | {
        "max_abs_diff": dd, "tolerance": 1e-5 * diam}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--meshes", type=int, default=200)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=os.path.dirname(learned.WEIGHTS))
    args = ap.parse_args()
    build.build()
    capi.load()
    t = time.time()
    X, Y = learned.training_set(args.meshes, seed=0)
    t_collect = time.time() - t
    t = time.time()
    w, hist = learned.train(X, Y, steps=args.steps, lr=args.lr, seed=0, log_every=500)
    t_train = time.time() - t
    # margin on held-out meshes
    Xh, Yh = learned.training_set(24, seed=1)
    import torch

    wh = torch.from_numpy(w).cuda()
    w16 = torch.empty(capi.PTP_MLP_NPARAM, dtype=torch.float16, device="cuda")
    capi.ptp_mlp_to_half(wh, w16)
    yh = torch.empty(Xh.shape[0], dtype=torch.int32, device="cuda")
    chosen = None
    rows = []
    for margin in (0.0, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0):
        capi.ptp_mlp_infer(w16, torch.from_numpy(Xh).cuda(), Xh.shape[0], yh, margin=margin)
        pred = yh.cpu().numpy()
        cnt = np.round(2.0 ** Yh).astype(np.int64)
        over = float(np.mean(pred > cnt))
        saved = float(np.sum(np.minimum(pred, cnt) - 1) / np.sum(cnt))
        rows.append({"margin": margin, "over_fraction": over, "tests_saved_fraction": saved})
        if chosen is None and over <= 0.01:
            chosen = margin
    if chosen is None:
        chosen = 3.0
    meta = {"trained_on": f"{args.meshes} seeded torus and sphere meshes (learned.training_meshes, seed 0)",
            "samples": int(X.shape[0]), "steps": args.steps, "lr": args.lr, "final_loss": hist[-1][1],
            "loss_history": hist, "margin": chosen, "margin_table": rows,
            "collect_s": round(t_collect, 1), "train_s": round(t_train, 1)}
    path = os.path.join(args.out, os.path.basename(learned.WEIGHTS))
    learned.save_weights(w, meta, path)
    V, F, S = meshes.torus_1m()
    ev = evaluate(w, chosen, V, F, S)
    print(json.dumps({"weights": path, "samples": int(X.shape[0]), "final_loss": hist[-1][1], "margin": chosen,
                      "margin_table": rows, "torus_1m": ev}, indent=1))


if __name__ == "__main__":
    main()
