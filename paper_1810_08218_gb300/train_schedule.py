"""Train the learned window schedule and evaluate it.

  python -m paper_1810_08218_gb300.train_schedule [--meshes 200] [--steps 3000] [--out DIR]

1. Runs the plain method (fixpoint mode, eps = 1e-7) with convergence traces
   on `--meshes` seeded meshes (tori, spheres, bumpy spheres, heightfields,
   jittered planes) and collects, per topleset, the six window features and
   log2 of the iterations from its entry into the band to its convergence.
2. Trains the MLP with the library's fused forward/backward and Adam kernels.
3. Picks the inference margin on 24 held-out meshes: the one with the fewest
   iterations of the learned band in total.
4. Saves the weights (flat float32 + JSON header) and reports, on the 1M
   noisy torus and the level-7 sphere (neither in the training set), plain
   vs learned band through ptp_distance_from_sources: ms per map, K, band
   updates and max |d_learned - d_plain| / diameter.
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

MARGINS = (-1.0, -0.5, -0.25, 0.0, 0.25, 0.5, 1.0)


def held_out_iterations(w, probs, margins=MARGINS):
    """Total K of the plain band and of the learned band per margin (two-step
    path, the schedule from ptp_window_features + ptp_mlp_infer)."""
    import torch

    tot = {"plain": 0, **{m: 0 for m in margins}}
    upd = {"plain": 0, **{m: 0 for m in margins}}
    for V, F, S in probs:
        mesh, tops = learned._mesh_tops(V, F, S)
        d = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
        st = capi.ptp_distance(tops, capi.ptp_params_default(eps=learned.FIXPOINT_EPS), d)
        tot["plain"] += st["iterations"]
        upd["plain"] += st["band_updates"]
        for m in margins:
            sched = learned.schedule(tops, w, m)
            p = capi.ptp_params_default(eps=learned.FIXPOINT_EPS, band_mode=2)
            p.schedule = sched.data_ptr()
            st = capi.ptp_distance(tops, p, d)
            tot[m] += st["iterations"]
            upd[m] += st["band_updates"]
    return tot, upd


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
    tot, upd = held_out_iterations(w, learned.training_meshes(24, seed=1))
    chosen = min(MARGINS, key=lambda m: (tot[m], upd[m], abs(m)))
    rows = [{"margin": m, "iterations": tot[m], "band_updates": upd[m]} for m in MARGINS]
    meta = {"trained_on": f"{args.meshes} seeded meshes (learned.training_meshes, seed 0), eps {learned.FIXPOINT_EPS}",
            "target": "log2(iterations from a topleset's entry into the band until one past its last failed test)",
            "samples": int(X.shape[0]), "steps": args.steps, "lr": args.lr, "final_loss": hist[-1][1],
            "loss_history": hist, "margin": chosen, "held_out_plain_iterations": tot["plain"],
            "held_out_plain_band_updates": upd["plain"], "margin_table": rows,
            "collect_s": round(t_collect, 1), "train_s": round(t_train, 1)}
    path = os.path.join(args.out, os.path.basename(learned.WEIGHTS))
    learned.save_weights(w, meta, path)
    ev = {}
    for name in ("torus_1m", "sphere_l7"):
        V, F, S = getattr(meshes, name)()
        ev[name] = learned.compare(V, F, S, w, chosen)
    print(json.dumps({"weights": path, "samples": int(X.shape[0]), "final_loss": hist[-1][1], "margin": chosen,
                      "held_out": {"plain_iterations": tot["plain"], "margin_table": rows}, "eval": ev}, indent=1))


if __name__ == "__main__":
    main()
