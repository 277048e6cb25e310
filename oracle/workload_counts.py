"""Write oracle/workload_counts.json: for each named benchmark workload, the
oracle's own iteration count K, topleset count rho, total vertex updates
(sum over k of |B_k minus S|) and the cumulative updates after every 25
iterations.  The benchmark's CPU-reference leg times a bounded prefix of the
oracle's iterations and scales it to a whole map with these counts.

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
WORKLOADS = {"torus_1m": meshes.torus_1m, "sphere_l7": meshes.sphere_l7, "flat65": meshes.flat65}


def counts(name: str, eps: float = 1e-3) -> dict:
    V, F, S = WORKLOADS[name]()
    V = np.ascontiguousarray(V, dtype=np.float32).astype(np.float64)
    r = oracle.ptp(V, F, S, eps=eps, trace=True)
    level, rho = oracle.toplesets(V.shape[0], F, S)
    off = np.concatenate([[0], np.cumsum(np.bincount(level[level >= 0], minlength=rho))])
    nsrc = int(off[1])
    per_k = np.array([off[j + 1] - max(off[i], nsrc) for i, j in zip(r.trace_i, r.trace_j)], dtype=np.int64)
    cum = np.cumsum(per_k)
    assert int(cum[-1]) == r.updates
    return {"eps": eps, "K": r.K, "rho": r.rho, "updates": r.updates,
            "cumulative_every_25": [int(cum[min(k, r.K) - 1]) for k in range(25, r.K + 25, 25)]}


def main() -> None:
    data = {name: counts(name) for name in WORKLOADS}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps({k: {kk: v[kk] for kk in ("K", "rho", "updates")} for k, v in data.items()}))


if __name__ == "__main__":
    main()
