"""Write terrain_4096_oracle_eps1e-3.txt: the FP64 oracle's PTP map of the
4096^2 heightfield (paper_1810_08218_gb300.meshes.terrain_4096, seed 0) at
the paper's eps = 1e-3 (Sec. 4.2, Eq. lower_band; update step of Sec. 3.2),
stored at 4,500 seeded sample vertices, with the oracle's K, rho and vertex
update count.  Calls only oracle/ and the seeded input generator; one map
takes a few minutes on one host core.

    python tests/golden/make_terrain_samples.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1810_08218_gb300 import meshes  # noqa: E402

OUT = os.path.join(HERE, "terrain_4096_oracle_eps1e-3.txt")


def main():
    V, F, S = meshes.terrain_4096()
    V = np.ascontiguousarray(V, dtype=np.float32).astype(np.float64)
    r = oracle.ptp(V, F, S, eps=1e-3)
    n = V.shape[0]
    rng = np.random.default_rng(2024)
    order = np.argsort(r.d, kind="stable")
    idx = np.concatenate([rng.choice(n, 4000, replace=False),      # anywhere
                          order[-200:],                              # the far end of the front
                          rng.choice(order[:20000], 300, replace=False)])  # near the source
    idx = np.unique(idx)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle PTP map of meshes.terrain_4096(seed=0) at eps = 1e-3 (Sec. 4.2, Eq. lower_band;\n")
        f.write("# the update step of Sec. 3.2), float32 vertex positions, written by make_terrain_samples.py.\n")
        f.write(f"# source {int(S[0])} K {r.K} rho {r.rho} updates {r.updates} diameter {meshes.bbox_diagonal(V)!r}\n")
        f.write("# vertex distance\n")
        for v in idx:
            f.write(f"{int(v)} {float(r.d[v])!r}\n")
    print(OUT, len(idx), r.K, r.rho, r.updates)


if __name__ == "__main__":
    main()
