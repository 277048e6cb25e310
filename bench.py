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
(rank 0 only): every step is one whole oracle map, the steps run as
independent single-threaded processes on all host cores, and the line
reports the whole run's wall time per map.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
    "bumpy_l8_fps": "level-8 icosphere with 64 Gaussian bumps (655,362 vertices, 1,310,720 triangles): 1,000-sample "
                    "farthest-point sampling from a seeded first vertex (999 multi-source maps, one captured CUDA "
                    "graph relaunched per sample) plus a 64-seed geodesic Voronoi map from the first 64 samples, "
                    "eps=1e-3",
    "uneven_batch32": "32 meshes, even ones jittered unit squares and odd ones noisy tori, vertex counts log-uniform "
                      "in 10k-2M (9,007,687 in total), one seeded source each, all maps in one persistent launch, "
                      "eps=1e-3",
    "terrain_4096": "4096x4096 heightfield (16,777,216 vertices, 33,538,050 triangles), 8-octave value-noise height "
                    "of amplitude 0.1, one seeded source, eps=1e-3",
}
# workloads of several maps per step (their own step functions below)
MULTI_MAP = ("bumpy_l8_fps", "uneven_batch32")
# Algorithmic bytes per band vertex-update (the per-update traffic model): its
# float4 position 16 B + d_{k-1} 4 B + d_k 4 B + row offset 4 B + six incident
# pairs 48 B.  Neighbour data is counted once, under the neighbour's own update.
BYTES_PER_UPDATE = 76
FALLBACK_HBM_GBS = 6800.0


def _mesh(name):
    from paper_1810_08218_gb300 import meshes

    return {"torus_1m": meshes.torus_1m, "sphere_l7": meshes.sphere_l7, "flat65": meshes.flat65,
            "terrain_4096": meshes.terrain_4096}[name]()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


STEPS = {
    "uneven_batch32": "32 x (ptp_mesh_create + ptp_toplesets) on 8 streams, largest mesh first to the least "
                      "loaded stream (BFS, renumbering), ptp_batch_create, ptp_distance_batch (all 32 windows in "
                      "one launch)",
    "bumpy_l8_fps": "ptp_mesh_create, ptp_fps (1,000 samples: per sample BFS, window, device argmax, "
                    "one captured CUDA graph), ptp_voronoi (64 seeds)",
}
SINGLE_STEP = ("ptp_mesh_create + ptp_distance_from_sources (corner lists and slots; BFS toplesets, "
               "renumbering and the window iteration in one launch: all hot-path stages)")


TWO_STEP = ("ptp_mesh_create + ptp_toplesets (cluster BFS, renumbering) + ptp_distance (the window iteration "
            "in its own launch)")


def _config(workload: str, world: int, path: str = "fused") -> dict:
    return {"workload": WORKLOADS[workload], "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"independent replicas x{world}" if world > 1 else "single GPU",
            "step": STEPS.get(workload, TWO_STEP if path == "two_step" else SINGLE_STEP)}


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (x itself without a process
    group); `device` holds the reduction tensor (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(total_ms: float, steps: int, world: int) -> tuple[float, float]:
    """(ms per step, ms per map) for `world` independent replicas that each
    ran `steps` maps in total_ms (the slowest rank's time): every rank's maps
    count, so the whole job's time per map is total_ms / (steps * world)."""
    return total_ms / steps, total_ms / (steps * world)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _kernel_source_hash() -> str:
    """Hash of the window kernel's code (its sources without comments and
    whitespace), so a recorded traffic figure is dropped when the code changes
    but not when only a comment does."""
    import re

    h = hashlib.sha256()
    for f in ("ptp_distance.cu", "ptp_update.cuh", "ptp_internal.cuh", "ptp_schedule.cuh"):
        with open(os.path.join(ROOT, "paper_1810_08218_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
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


# the oracle's map at stored sample vertices, for maps too large for the
# CPU-baseline leg to run whole
STORED_SAMPLES = {"terrain_4096": os.path.join(ROOT, "tests", "golden", "terrain_4096_oracle_eps1e-3.txt")}

# one full oracle map takes about this long on one host core; larger maps are
# timed on a bounded prefix of their iterations (the CPU baseline leg)
CPU_BASELINE_BUDGET_S = 30.0


def cpu_oracle_full_map(workload: str, V=None, F=None, S=None) -> tuple[dict, np.ndarray | None]:
    """The FP64 oracle as it stands on one host core: one full map when the
    oracle's update count for the workload fits the budget (the map is
    returned for the accuracy report), else the first iterations of the map,
    scaled to the whole map by the oracle's own update count."""
    import oracle

    if V is None:
        V, F, S = _mesh(workload)
    V = np.ascontiguousarray(V, dtype=np.float32).astype(np.float64)
    with open(os.path.join(ROOT, "oracle", "workload_counts.json")) as f:
        counts = json.load(f).get(workload)
    if counts is None or counts["updates"] * 150e-9 <= CPU_BASELINE_BUDGET_S:
        t = time.perf_counter()
        r = oracle.ptp(V, F, S, eps=1e-3)
        dt = time.perf_counter() - t
        return ({"value": round(dt * 1e3, 3), "unit": "ms per map", "cores": 1, "kind": "oracle",
                 "sample": f"one full map of the workload on 1 host core (K={r.K}, {r.updates} vertex updates, "
                           f"{dt:.1f} s)"}, r.d)
    # a prefix of the map's iterations, doubled until it takes a third of
    # the budget (early iterations have narrow bands and cost little)
    m_iter = max(1, counts["K"] // 32)
    while True:
        t = time.perf_counter()
        r = oracle.ptp(V, F, S, eps=1e-3, max_iter=m_iter)
        dt = time.perf_counter() - t
        if dt >= CPU_BASELINE_BUDGET_S / 3 or m_iter >= counts["K"]:
            break
        m_iter = min(2 * m_iter, counts["K"])
    ms = dt * 1e3 * counts["updates"] / r.updates
    return ({"value": round(ms, 3), "unit": "ms per map", "cores": 1, "kind": "oracle",
             "sample": f"the first {m_iter} of the map's {counts['K']} iterations on 1 host core ({r.updates} of "
                       f"{counts['updates']} vertex updates, {dt:.1f} s), scaled by the update count"}, None)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_ORACLE_JOB = {}


def _oracle_init(workload: str) -> None:
    V, F, S = _mesh(workload)
    _ORACLE_JOB["args"] = (np.ascontiguousarray(V, dtype=np.float32).astype(np.float64), F, S)


def _oracle_worker(_step: int) -> tuple[float, int]:
    """One whole FP64 oracle map in this worker process: (seconds, K)."""
    import oracle

    V, F, S = _ORACLE_JOB["args"]
    t = time.perf_counter()
    r = oracle.ptp(V, F, S, eps=1e-3)
    return time.perf_counter() - t, r.K


def run_reference(args) -> None:
    """The reference arm: the FP64 oracle as it stands.  Each step is one
    whole map; the W warm-up maps and then the K timed maps run as
    independent single-threaded processes, as many at once as the host has
    cores.  value = wall time of the K timed maps / K."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = host_cores()
    procs = max(1, min(cores, args.steps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_oracle_init, initargs=(args.workload,)) as pool:
        pool.map(_oracle_worker, range(min(args.warmup, procs)), chunksize=1)
        t = time.perf_counter()
        res = pool.map(_oracle_worker, range(args.steps), chunksize=1)
        wall = time.perf_counter() - t
    ms = wall * 1e3 / args.steps
    per_map = statistics.mean(r[0] for r in res)
    line = {"metric": "ms per geodesic map", "value": round(ms, 3), "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(args.workload, args.gpus),
            "cpu_baseline": {"value": round(ms, 3), "unit": "ms", "cores": procs, "kind": "oracle",
                             "sample": f"{args.steps} whole maps (K={res[0][1]}) in {procs} single-threaded "
                                       f"processes on {cores} host cores, {wall * 1e3:.1f} ms wall; "
                                       f"{per_map * 1e3:.1f} ms per map in each process"},
            "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


LEARNED_WORKLOADS = ("torus_1m", "sphere_l7")


def learned_vs_plain(V, F, S) -> dict:
    """The learned multi-advance band against the plain band, both in
    fixpoint mode (eps = 1e-7) through the fused launch on the resident
    mesh: median ms per map of 10 runs (CUDA events), K, band updates and
    max |d_learned - d_plain| / diameter."""
    from paper_1810_08218_gb300 import learned

    w, meta = learned.load_weights()
    r = learned.compare(V, F, S, w, meta["margin"], eps=learned.FIXPOINT_EPS, reps=10, warm=3)
    out = {"eps": learned.FIXPOINT_EPS, "margin": meta["margin"], "unit": "ms per map"}
    for k in ("plain", "learned"):
        out[k] = {"ms": round(r[k]["ms"], 4), "K": r[k]["K"], "band_updates": r[k]["band_updates"]}
    out["learned_over_plain_ms"] = round(r["learned"]["ms"] / r["plain"]["ms"], 4)
    out["max_abs_dd_over_diam"] = r["max_abs_dd_over_diam"]
    return out


def map_accuracy(workload: str, d_gpu: np.ndarray, V32: np.ndarray, S, d_oracle) -> dict:
    """max |d_gpu - d_oracle| / diameter against the oracle's map at the same
    eps, and the mean relative error against the exact distance where the
    workload has one (Euclidean on the plane, great circle on the sphere)."""
    from paper_1810_08218_gb300 import accuracy, meshes

    diam = meshes.bbox_diagonal(V32)
    out = {"diameter": round(diam, 6)}
    g = d_gpu.astype(np.float64)
    if d_oracle is not None:
        fin = np.isfinite(d_oracle)
        out["max_abs_dd_over_diam_vs_oracle"] = float(np.max(np.abs(g[fin] - d_oracle[fin])) / diam)
        out["tolerance_over_diam"] = 1e-5
    elif workload in STORED_SAMPLES and os.path.exists(STORED_SAMPLES[workload]):
        # a map too large for the CPU-baseline leg: the oracle's values stored
        # at seeded sample vertices (tests/golden, written offline)
        idx, val = [], []
        for line in open(STORED_SAMPLES[workload]):
            if not line.startswith("#"):
                a, b = line.split()
                idx.append(int(a))
                val.append(float(b))
        out["max_abs_dd_over_diam_vs_oracle"] = float(np.max(np.abs(g[np.array(idx)] - np.array(val))) / diam)
        out["oracle_samples"] = len(idx)
        out["tolerance_over_diam"] = 1e-5
    exact = accuracy._exact(workload, V32.astype(np.float64), np.asarray(S))
    if exact is not None:
        m = exact > 0
        out["mre_vs_exact"] = float(np.mean(np.abs(g[m] - exact[m]) / exact[m]))
        out["exact"] = "Euclidean distance" if workload == "flat65" else "great-circle distance"
    return out


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
    d = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    kb = torch.cuda.Event(enable_timing=True)
    ke = torch.cuda.Event(enable_timing=True)
    kb.record(stream)  # torch creates the CUDA event on first record
    ke.record(stream)
    torch.cuda.synchronize()
    params = capi.ptp_params_default(eps=1e-3)

    S_host = np.ascontiguousarray(S, dtype=np.int32)  # host source list: no host wait for its validation

    def step(with_kernel_events: bool):
        if with_kernel_events:
            params.ev_begin = kb.cuda_event
            params.ev_end = ke.cuda_event
        else:
            params.ev_begin = None
            params.ev_end = None
        mesh = capi.ptp_mesh_create(Vt, Ft)
        if args.path == "two_step":
            # toplesets (cluster BFS, renumbering), then the window launch
            tops = capi.ptp_toplesets(mesh, S_host)
            capi.ptp_distance(tops, params, d, stats=False)
            capi.ptp_toplesets_destroy(tops)
        else:
            # toplesets (BFS, renumbering) and the iteration in one launch
            capi.ptp_distance_from_sources(mesh, S_host, params, d, stats=False)
        return mesh

    for _ in range(args.warmup):
        mesh = step(False)
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
        mesh = step(True)
        s1.record(stream)
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        kern_ms.append(kb.elapsed_time(ke))
        capi.ptp_mesh_destroy(mesh)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    launches = capi.ptp_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None

    # the map's statistics (one more untimed run with them)
    mesh = capi.ptp_mesh_create(Vt, Ft)
    params.ev_begin = None
    params.ev_end = None
    if args.path == "two_step":
        tops = capi.ptp_toplesets(mesh, S_host)
        stats = capi.ptp_distance(tops, params, d, stats=True)
        capi.ptp_toplesets_destroy(tops)
    else:
        stats = capi.ptp_distance_from_sources(mesh, S_host, params, d, stats=True)
    capi.ptp_mesh_destroy(mesh)
    d_map = d.cpu().numpy()
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    ms_per_step, value = replica_throughput(total_ms, args.steps, world)

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
    e2e_val = max_over_ranks(statistics.mean(e2e_ms), dev) / world

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
            "config": _config(args.workload, world, args.path),
            "window_kernel_ms": round(kavg, 4),
            "timed_kernel": ("ptp_window, fused: BFS toplesets, renumbering and the iteration in one launch"
                             if args.path == "fused" else "ptp_window, the iteration alone (toplesets built before)"),
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
        if args.workload in LEARNED_WORKLOADS:
            line["learned_schedule"] = learned_vs_plain(V, F, S)
        d_oracle = None
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], d_oracle = cpu_oracle_full_map(args.workload, V, F, S)
        line["accuracy"] = map_accuracy(args.workload, d_map, V32, S, d_oracle)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _multi_line(args, metric_maps, step_ms, e2e_ms, h2d, d2h, launches, clocks, stats_ptp, extra, kern_ms=None):
    """The JSON line of a several-maps workload (rank 0, N = 1)."""
    peak, peak_kind = _peaks()
    value = step_ms / metric_maps
    t_ms = kern_ms if kern_ms is not None else step_ms
    achieved = BYTES_PER_UPDATE * stats_ptp["band_updates"] / (t_ms * 1e-3) / 1e9
    line = {
        "metric": "ms per geodesic map", "value": round(value, 4), "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(_config(args.workload, 1), maps_per_step=metric_maps),
        "ptp": stats_ptp,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_kind, "traffic": None,
                     "scope": "window kernel" if kern_ms is not None else "whole step",
                     "bytes_model": f"{BYTES_PER_UPDATE} B x {stats_ptp['band_updates']} band vertex-updates"},
        "e2e": {"value": round(e2e_ms / metric_maps, 4), "unit": "ms", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    line.update(extra)
    return line


def _timed_steps(torch, stream, flush, step, n):
    out = []
    for _ in range(n):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def stream_schedule(sizes, lanes):
    """Largest first to the least loaded lane, the load of a mesh being
    sqrt(n) (its BFS levels).  Returns the issue order and lane per mesh."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0.0] * lanes
    lane_of = {}
    for i in order:
        j = min(range(lanes), key=lambda q: (load[q], q))
        lane_of[i] = j
        load[j] += math.sqrt(sizes[i])
    return order, lane_of


def run_batch(args) -> None:
    """32 uneven maps: all hot-path stages per map (mesh, toplesets), then
    the batched window in one launch; beside it the same 32 maps one after
    another through ptp_distance."""
    import torch

    from paper_1810_08218_gb300 import build, capi, meshes

    rank, _, local = _dist_env()
    torch.cuda.set_device(local)
    build.build()
    capi.load()
    probs = meshes.uneven_batch(32, seed=0)
    host = [(torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).pin_memory(),
             torch.from_numpy(F).pin_memory(), torch.from_numpy(S)) for V, F, S in probs]
    dev = [(v.cuda(), f.cuda(), q.cuda()) for v, f, q in host]
    sizes = [V.shape[0] for V, _, _ in probs]
    outs = [torch.empty(n, dtype=torch.float32, device="cuda") for n in sizes]
    houts = [torch.empty(n, dtype=torch.float32).pin_memory() for n in sizes]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    kb = torch.cuda.Event(enable_timing=True)
    ke = torch.cuda.Event(enable_timing=True)
    kb.record(stream)
    ke.record(stream)
    torch.cuda.synchronize()
    params = capi.ptp_params_default(eps=1e-3)
    params.ev_begin = kb.cuda_event
    params.ev_end = ke.cuda_event
    res = {}
    # The meshes and their toplesets are independent: each BFS occupies one
    # 8-SM cluster, so they are built on 8 streams at once (host source lists,
    # so no toplesets call waits for the device) and joined before the batch
    # is created.  A BFS takes time in proportion to its levels, about
    # sqrt(n), so the meshes go largest first to the least loaded stream; a
    # mesh is created on its own stream, so its validation read-back waits
    # only for that stream while the others run.
    side = [torch.cuda.Stream() for _ in range(8)]
    srcs = [np.ascontiguousarray(S, dtype=np.int32) for _, _, S in probs]
    order, lane_of = stream_schedule(sizes, len(side))

    def batched(src=dev, out_host=False):
        ready = torch.cuda.Event()
        ready.record(stream)
        for ss in side:
            ss.wait_event(ready)
        tops = [None] * len(src)
        for i in order:
            ss = side[lane_of[i]]
            tops[i] = capi.ptp_toplesets(capi.ptp_mesh_create(src[i][0], src[i][1], stream=ss), srcs[i], stream=ss)
        for ss in side:
            ev = torch.cuda.Event()
            ev.record(ss)
            stream.wait_event(ev)
        batch = capi.ptp_batch_create(tops, stream=stream)
        res["st"] = capi.ptp_distance_batch(batch, params, outs)
        capi.ptp_batch_destroy(batch)
        if out_host:
            for o, h in zip(outs, houts):
                h.copy_(o, non_blocking=True)

    seq_params = capi.ptp_params_default(eps=1e-3)

    def sequential():
        # the same maps one after another, each through the single-map
        # benchmark path (mesh, then the fused launch)
        for (v, f, _), src, o in zip(dev, srcs, outs):
            capi.ptp_distance_from_sources(capi.ptp_mesh_create(v, f), src, seq_params, o, stats=False)

    for _ in range(args.warmup):
        batched()
        sequential()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = capi.ptp_kernel_launches()
    kern, t_batch = [], []
    for _ in range(args.steps):
        t_batch += _timed_steps(torch, stream, flush, batched, 1)
        kern.append(kb.elapsed_time(ke))
    launches = capi.ptp_kernel_launches() - l0
    clocks = sampler.stop()
    t_seq = _timed_steps(torch, stream, flush, sequential, max(3, args.steps // 2))
    # end to end: inputs from pinned host memory, maps back to pinned host memory
    e2e = []
    for s_ in range(args.warmup + min(args.steps, 10)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        batched(src=host, out_host=True)
        torch.cuda.synchronize()
        if s_ >= args.warmup:
            e2e.append((time.perf_counter() - t) * 1e3)
    st = res["st"]
    stats_ptp = {"K_max": max(x["iterations"] for x in st), "K_sum": sum(x["iterations"] for x in st),
                 "band_updates": sum(x["band_updates"] for x in st), "vertices": sum(sizes)}
    line = _multi_line(args, 32, statistics.mean(t_batch), statistics.mean(e2e),
                       sum(12 * V.shape[0] + 12 * F.shape[0] + 4 for V, F, _ in probs), 4 * sum(sizes), launches,
                       clocks, stats_ptp,
                       {"window_kernel_ms": round(statistics.mean(kern), 4),
                        "sequential_ms_per_map": round(statistics.mean(t_seq) / 32, 4),
                        "batch_speedup": round(statistics.mean(t_seq) / statistics.mean(t_batch), 3)},
                       kern_ms=statistics.mean(kern))
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fps(args) -> None:
    """1,000-sample farthest-point sampling (999 multi-source maps under one
    captured CUDA graph) plus a 64-seed Voronoi map, mesh creation included."""
    import torch

    from paper_1810_08218_gb300 import build, capi, meshes

    rank, _, local = _dist_env()
    torch.cuda.set_device(local)
    build.build()
    capi.load()
    V, F, S = meshes.bumpy_l8()
    n = V.shape[0]
    Vh = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).pin_memory()
    Fh = torch.from_numpy(F).pin_memory()
    Vt, Ft = Vh.cuda(), Fh.cuda()
    ns, nv = 1000, 64
    samples = torch.empty(ns, dtype=torch.int32, device="cuda")
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    hs = torch.empty(ns, dtype=torch.int32).pin_memory()
    hl = torch.empty(n, dtype=torch.int32).pin_memory()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    params = capi.ptp_params_default(eps=1e-3)
    res = {}

    def step(src=(Vt, Ft), out_host=False):
        mesh = capi.ptp_mesh_create(*src)
        res["fps"] = capi.ptp_fps(mesh, int(S[0]), ns, params, samples, use_graph=True)
        res["vor"] = capi.ptp_voronoi(mesh, samples[:nv], params, d, lab)
        if out_host:
            hs.copy_(samples, non_blocking=True)
            hl.copy_(lab, non_blocking=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = capi.ptp_kernel_launches()
    t = _timed_steps(torch, stream, flush, step, args.steps)
    launches = capi.ptp_kernel_launches() - l0
    clocks = sampler.stop()
    e2e = []
    for s_ in range(args.warmup + min(args.steps, 5)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(src=(Vh, Fh), out_host=True)
        torch.cuda.synchronize()
        if s_ >= args.warmup:
            e2e.append((time.perf_counter() - t0) * 1e3)
    maps = (ns - 1) + 1
    stats_ptp = {"fps_iterations": res["fps"]["iterations"], "band_updates": res["fps"]["band_updates"]
                 + res["vor"]["band_updates"], "voronoi_K": res["vor"]["iterations"]}
    line = _multi_line(args, maps, statistics.mean(t), statistics.mean(e2e), 12 * n + 12 * F.shape[0],
                       4 * ns + 4 * n, launches, clocks, stats_ptp,
                       {"fps_ms_per_sample": round(statistics.mean(t) / ns, 4)})
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="torus_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", choices=["fused", "two_step"], default="fused",
                    help="single-map workloads: the fused launch (default) or ptp_toplesets + ptp_distance")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if args.workload in MULTI_MAP:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle timing is defined for the single-map "
                              "workloads (torus_1m, sphere_l7, flat65, terrain_4096)"}), flush=True)
        else:
            run_reference(args)
    elif args.workload == "uneven_batch32":
        run_batch(args)
    elif args.workload == "bumpy_l8_fps":
        run_fps(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
