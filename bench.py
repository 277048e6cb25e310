#!/usr/bin/env python3
"""Benchmark: ms per geodesic distance map on the 1M-vertex noisy torus.

One step = one pass of the whole PTP hot path on device-resident inputs:
ptp_mesh_create (corner lists) -> ptp_toplesets (BFS toplesets and
renumbering) -> ptp_distance (window iteration, convergence test, band
sliding, scatter to the original order).  L2 is flushed (a 256 MiB write)
between steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica of the map on its own
GPU (the method does not shard within one map); value = total time (max over
ranks) / maps processed by all ranks.  Rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on the host cores instead
(rank 0 only), each step a bounded prefix of the oracle's iterations scaled
to a whole map by the oracle's own update count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "torus_1m": "noisy torus R=1 r=0.4, 1024x1024 lattice (1,048,576 vertices, 2,097,152 triangles), "
                "radial noise +-0.01r, one seeded source, eps=1e-3",
    "sphere_l7": "unit icosphere level 7 (163,842 vertices, 327,680 triangles), one seeded source, eps=1e-3",
    "flat65": "65x65 jittered unit square (4,225 vertices, 8,192 triangles), centre source, eps=1e-3",
}
# Algorithmic bytes per band vertex-update (the per-update traffic model): its
# float4 position 16 B + d_{k-1} 4 B + d_k 4 B + row offset 4 B + six incident
# pairs 48 B.  Neighbour data is counted once, under the neighbour's own update.
BYTES_PER_UPDATE = 76
FALLBACK_HBM_GBS = 6800.0


def _mesh(name):
    from paper_1810_08218_gb300 import meshes

    return {"torus_1m": meshes.torus_1m, "sphere_l7": meshes.sphere_l7, "flat65": meshes.flat65}[name]()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _config(workload: str, world: int) -> dict:
    return {"workload": WORKLOADS[workload], "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"independent replicas x{world}" if world > 1 else "single GPU",
            "step": "mesh_create + toplesets + distance (all hot-path stages)"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("ptp_distance.cu", "ptp_update.cuh", "ptp_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1810_08218_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(workload: str):
    """DRAM bytes per launch of the window kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "ptp_window_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[workload]
        if e.get("kernel_source_sha256") == _kernel_source_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_full_map(workload: str) -> dict:
    """The FP64 oracle as it stands, one full map, single thread."""
    import oracle

    V, F, S = _mesh(workload)
    V = np.ascontiguousarray(V, dtype=np.float32).astype(np.float64)
    t = time.perf_counter()
    r = oracle.ptp(V, F, S, eps=1e-3)
    dt = time.perf_counter() - t
    return {"value": round(dt * 1e3, 3), "unit": "ms per map", "cores": 1, "kind": "oracle",
            "sample": f"one full map of the workload on 1 host core (K={r.K}, {r.updates} vertex updates, "
                      f"{dt:.1f} s)"}


def run_reference(args) -> None:
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import oracle

    with open(os.path.join(ROOT, "oracle", "workload_counts.json")) as f:
        counts = json.load(f)[args.workload]
    V, F, S = _mesh(args.workload)
    V = np.ascontiguousarray(V, dtype=np.float32).astype(np.float64)
    # bounded prefix: about 150 s of oracle work over all steps, at ~300 ns per update
    budget_s = max(0.5, 150.0 / max(1, args.steps + args.warmup))
    target = budget_s / 300e-9
    cum = counts["cumulative_every_25"]
    m_iter = 25
    for q, c in enumerate(cum):
        if c <= target:
            m_iter = min(25 * (q + 1), counts["K"])
    times = []
    upd = None
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oracle.ptp(V, F, S, eps=1e-3, max_iter=m_iter)
        dt = time.perf_counter() - t
        upd = r.updates
        if s >= args.warmup:
            times.append(dt)
    scale = counts["updates"] / upd
    ms = 1e3 * statistics.mean(times) * scale
    line = {"metric": "ms per geodesic map", "value": round(ms, 3), "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(args.workload, args.gpus),
            "cpu_baseline": {"value": round(ms, 3), "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": f"first {m_iter} of {counts['K']} iterations ({upd} of {counts['updates']} "
                                       f"vertex updates) per step, scaled by the oracle's own update count"},
            "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    from paper_1810_08218_gb300 import build, capi

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    capi.load()

    V, F, S = _mesh(args.workload)
    n, nf, m = V.shape[0], F.shape[0], S.shape[0]
    V32 = np.ascontiguousarray(V, dtype=np.float32)
    Vt = torch.from_numpy(V32).to(dev)
    Ft = torch.from_numpy(F).to(dev)
    St = torch.from_numpy(S).to(dev)
    d = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    kb = torch.cuda.Event(enable_timing=True)
    ke = torch.cuda.Event(enable_timing=True)
    kb.record(stream)  # torch creates the CUDA event on first record
    ke.record(stream)
    torch.cuda.synchronize()
    params = capi.ptp_params_default(eps=1e-3)

    def step(with_kernel_events: bool):
        if with_kernel_events:
            params.ev_begin = kb.cuda_event
            params.ev_end = ke.cuda_event
        else:
            params.ev_begin = None
            params.ev_end = None
        mesh = capi.ptp_mesh_create(Vt, Ft)
        tops = capi.ptp_toplesets(mesh, St)
        capi.ptp_distance(tops, params, d, stats=False)
        return mesh, tops

    for _ in range(args.warmup):
        mesh, tops = step(False)
        stats = capi.ptp_last_stats(tops)
        capi.ptp_toplesets_destroy(tops)
        capi.ptp_mesh_destroy(mesh)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = capi.ptp_kernel_launches()
    step_ms, kern_ms = [], []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        mesh, tops = step(True)
        s1.record(stream)
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        kern_ms.append(kb.elapsed_time(ke))
        stats = capi.ptp_last_stats(tops)
        capi.ptp_toplesets_destroy(tops)
        capi.ptp_mesh_destroy(mesh)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    launches = capi.ptp_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None

    total_ms = float(sum(step_ms))
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    value = total_ms / (args.steps * world)

    # end to end through the public API with pinned host buffers: the H2D
    # copies of vertices, faces and sources and the D2H copy of the map are
    # inside the timed region
    Vh = torch.from_numpy(V32).pin_memory()
    Fh = torch.from_numpy(F).pin_memory()
    Sh = torch.from_numpy(S).pin_memory()
    dh = torch.empty(n, dtype=torch.float32).pin_memory()
    e2e_ms = []
    for s in range(args.warmup + min(args.steps, 20)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        capi.ptp_geodesic(Vh, Fh, Sh, capi.ptp_params_default(eps=1e-3), dh)
        dt = (time.perf_counter() - t) * 1e3
        if s >= args.warmup:
            e2e_ms.append(dt)
    e2e_val = statistics.mean(e2e_ms)
    if world > 1:
        tt = torch.tensor([e2e_val], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_val = float(tt.item()) / world

    if rank == 0:
        peak, peak_kind = _peaks()
        kavg = statistics.mean(kern_ms)
        bytes_launch = BYTES_PER_UPDATE * stats["band_updates"]
        achieved = bytes_launch / (kavg * 1e-3) / 1e9
        line = {
            "metric": "ms per geodesic map", "value": round(value, 4), "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": _config(args.workload, world),
            "window_kernel_ms": round(kavg, 4),
            "vertex_updates_per_s": round(stats["band_updates"] / (kavg * 1e-3), 1),
            "ptp": {"K": stats["iterations"], "rho": stats["rho"], "band_updates": stats["band_updates"],
                    "active_updates": stats["active_updates"], "fp64_solves": stats["fp64_solves"]},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                         "traffic": _traffic(args.workload),
                         "bytes_model": f"{BYTES_PER_UPDATE} B x {stats['band_updates']} band vertex-updates"},
            "e2e": {"value": round(e2e_val, 4), "unit": "ms", "h2d_bytes_per_step": 12 * n + 12 * nf + 4 * m,
                    "d2h_bytes_per_step": 4 * n},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s": round(wall, 3),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_full_map(args.workload)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="torus_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
