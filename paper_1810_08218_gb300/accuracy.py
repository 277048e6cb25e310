"""Accuracy of the stopping rule against the fixpoint (the ε–error relation
the paper leaves open, Sec. 6 / Sec. 5.2).

For each mesh and each ε of Eq. lower_band (and the fixed band whose lower
bound is ceil(k/2), Sec. 6.1), one map through ptp_distance_from_sources:
the iterations K, the time per map (mesh resident, CUDA events, median of
5 after 2 warm-ups), the deviation from the fixpoint (the same map at
ε = 1e-7, where every band update has stopped changing in FP32) and, where
the exact geodesic distance has a closed form, the error against it:
Euclidean distance on the plane, great-circle distance on the unit sphere
(the quantities of Sec. 5.2).  Prints a markdown table.

    python -m paper_1810_08218_gb300.accuracy [flat65 sphere_l7 torus_1m]
"""
from __future__ import annotations

import statistics
import sys

import numpy as np

from . import build, capi, meshes

EPS = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5)
FIXPOINT_EPS = 1e-7


def _exact(name: str, V: np.ndarray, S: np.ndarray):
    if name == "flat65":
        return np.linalg.norm(V - V[S[0]], axis=1)
    if name == "sphere_l7":
        return np.arccos(np.clip(V @ V[S[0]], -1.0, 1.0))
    return None


def _run(torch, mesh, S, n, params, reps=5, warm=2):
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    ok = (capi.PTP_OK, capi.PTP_ERR_NOT_CONVERGED)
    times = []
    st = None
    for r in range(warm + reps):
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record()
        st = capi.ptp_distance_from_sources(mesh, S, params, d, ok=ok)
        z.record()
        z.synchronize()
        if r >= warm:
            times.append(a.elapsed_time(z))
    return d.cpu().numpy().astype(np.float64), st, statistics.median(times)


def report(names) -> str:
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required")
    build.build()
    capi.load()
    lines = ["| mesh | stopping rule | K | ms per map | max \\|d - d_fix\\| / diam | mean \\|d - d_fix\\| / mean d_fix "
             "| MAPE vs exact | max \\|d - exact\\| / diam |",
             "|---|---|---:|---:|---:|---:|---:|---:|"]
    for name in names:
        V, F, S = getattr(meshes, name)()
        V32 = np.ascontiguousarray(V, dtype=np.float32)
        n = V.shape[0]
        diam = meshes.bbox_diagonal(V32)
        mesh = capi.ptp_mesh_create(torch.from_numpy(V32).cuda(), torch.from_numpy(np.ascontiguousarray(F)).cuda())
        Sh = np.ascontiguousarray(S, dtype=np.int32)
        d_fix, st_fix, ms_fix = _run(torch, mesh, Sh, n, capi.ptp_params_default(eps=FIXPOINT_EPS))
        exact = _exact(name, V32.astype(np.float64), S)
        rules = [(f"ε = {e:g}", capi.ptp_params_default(eps=e)) for e in EPS]
        rules.append(("fixed band ceil(k/2)", capi.ptp_params_default(band_mode=1)))
        rules.append((f"ε = {FIXPOINT_EPS:g} (fixpoint)", None))
        for label, p in rules:
            if p is None:
                d, st, ms = d_fix, st_fix, ms_fix
            else:
                d, st, ms = _run(torch, mesh, Sh, n, p)
            dev = np.abs(d - d_fix)
            row = [name, label, str(st["iterations"]), f"{ms:.3f}", f"{dev.max() / diam:.2e}",
                   f"{dev.mean() / d_fix.mean():.2e}"]
            if exact is not None:
                m = exact > 0
                row += [f"{100 * np.mean(np.abs(d[m] - exact[m]) / exact[m]):.4f}%",
                        f"{np.abs(d - exact).max() / diam:.2e}"]
            else:
                row += ["—", "—"]
            if st["status"] != capi.PTP_OK:
                row[2] += " (cap)"
            lines.append("| " + " | ".join(row) + " |")
        capi.ptp_mesh_destroy(mesh)
    return "\n".join(lines)


if __name__ == "__main__":
    print(report(sys.argv[1:] or ["flat65", "sphere_l7", "torus_1m"]))
