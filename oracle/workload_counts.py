"""Write oracle/workload_counts.json: for each named single-map benchmark
workload, the oracle's own iteration count K, topleset count rho and total
vertex updates (sum over k of |B_k minus S|) at the paper's eps = 1e-3.  The
full-size GPU tests compare the fused launch's statistics with them.

Calls only the oracle and the seeded input generators.
Run: python -m oracle.workload_counts
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1810_08218_gb300 import meshes  # noqa: E402

OUT = os.path.join(HERE, "workload_counts.json")
WORKLOADS = {"torus_1m": meshes.torus_1m, "sphere_l7": meshes.sphere_l7, "flat65": meshes.flat65,
             "terrain_4096": meshes.terrain_4096}


def counts(name: str, eps: float = 1e-3) -> dict:
    V, F, S = WORKLOADS[name]()
    V = np.ascontiguousarray(V, dtype=np.float32).astype(np.float64)
    r = oracle.ptp(V, F, S, eps=eps, trace=True)
    level, rho = oracle.toplesets(V.shape[0], F, S)
    off = np.concatenate([[0], np.cumsum(np.bincount(level[level >= 0], minlength=rho))])
    nsrc = int(off[1])
    per_k = np.array([off[j + 1] - max(off[i], nsrc) for i, j in zip(r.trace_i, r.trace_j)], dtype=np.int64)
    assert int(per_k.sum()) == r.updates
    return {"eps": eps, "K": r.K, "rho": r.rho, "updates": r.updates}


def main() -> None:
    data = {name: counts(name) for name in WORKLOADS}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps({k: {kk: v[kk] for kk in ("K", "rho", "updates")} for k, v in data.items()}))


if __name__ == "__main__":
    main()
