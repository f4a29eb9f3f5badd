"""Benchmark of the Flood complex filtration hot path on one B300 (or N replicas).

One step = FPS landmarks -> cell grid over X -> flood values of every simplex
of Del(L) (interior samples, face-max), i.e. every GPU stage of the method.
The host Delaunay of L is input and is not timed: it is computed once from
the first FPS result and reused (FPS is bit-exact, so every step picks the
same landmarks; the bench checks that).

Prints one JSON line (rank 0). Default workload: 1,000,000-point noisy torus
(R=1, r=0.3, uniform in angles, sigma=0.005), 2,000 FPS landmarks, m=10.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "torus-1M": dict(gen="torus_cloud", n=1_000_000, n_l=2000, m=10, seed=2),
    "shapes-5M": dict(gen="shape_mix_cloud", n=5_000_000, n_l=10_000, m=12, seed=3),
    "sphere-10k": dict(gen="sphere_cloud", n=10_000, n_l=128, m=6, seed=1),
    # the setting of the paper's runtime comparison (§5.3, Table 2): 1M swiss cheese, 2k landmarks,
    # 20 points per edge
    "swisscheese-1M": dict(gen="swisscheese_cloud", n=1_000_000, n_l=2000, m=19, seed=6),
}
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (Blackwell)
FLOPS_PER_PAIR = 6               # one pair = 3 FMAs: |x'|^2 - 2 p'.x'
# DRAM bytes (read + write) of the flood kernels of one filtration on torus-1M
# (k_flood_heavy and k_flood, dimensions 1-3: six launches), from one ncu
# capture at the given launch parameters; valid only while the filtration
# source is the one captured and the step runs at those parameters, else
# reported as null.
FLOOD_DRAM_CAPTURE = {"workload": "torus-1M", "bytes": 153_770_752 + 205_568,
                      "cell_factor": 0.5, "heavy_shells": 9,
                      "filtration_cu_sha256": "53db2d106bcc29a3664dc4dec60e438a221c5cda84e13873b12ec62fe1837d2e"}


def _source_sha(name: str):
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_2509_22432_b300", "csrc", name), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None


def _flood_traffic(workload: str, tuned: dict):
    cap = FLOOD_DRAM_CAPTURE
    if cap["bytes"] is None or workload != cap["workload"]:
        return None
    if (tuned["cell_factor"], tuned["heavy_shells"]) != (cap["cell_factor"], cap["heavy_shells"]):
        return None
    if _source_sha("filtration.cu") != cap["filtration_cu_sha256"]:
        return None
    return float(cap["bytes"])


def _golden_landmarks(workload: str, X):
    """The oracle's FPS picks for this workload (tests/golden), if stored and X is the stored cloud."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", f"fps_{workload}_oracle.txt")
    if not os.path.exists(path):
        return None
    head, rows = {}, []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) == 2:
                    head[parts[0]] = parts[1]
            elif line.strip():
                rows.append(int(line))
    if hashlib.sha256(np.ascontiguousarray(X, np.float32).tobytes()).hexdigest() != head.get("x_sha256"):
        return None
    return np.array(rows, dtype=np.int64)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []       # (arrival time, csv line)
        self.window = None    # (start, end) of the timed region, monotonic seconds

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, start: float, end: float):
        """Keep only the samples that arrived inside [start, end]."""
        self.window = (start, end)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if self.window and not (self.window[0] <= t <= self.window[1]):
                continue
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(ms_local: float, units_local: float, device=None):
    """Whole-job numbers across ranks: (max step time over ranks, total units).

    Replicas (each rank runs its own cloud) report weak scaling: the job's
    throughput is the units of all ranks divided by the slowest rank's time.
    """
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local), float(units_local)
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def make_inputs(wl: dict, seed_offset: int = 0):
    from paper_2509_22432_b300 import data
    gen = getattr(data, wl["gen"])
    return gen(wl["n"], seed=wl["seed"] + seed_offset)


def oracle_workload(X, wl, workload):
    """Landmarks and complex of the workload for the oracle: the oracle's own FPS picks.

    For the full-size workloads they are stored under tests/golden (written by a
    script that runs only the oracle); small clouds run the oracle's FPS here.
    Returns (L, complex, where the landmarks came from).
    """
    import oracle
    from paper_2509_22432_b300 import delaunay_complex
    idx = _golden_landmarks(workload, X)
    where = f"tests/golden/fps_{workload}_oracle.txt"
    if idx is None:
        if X.shape[0] * wl["n_l"] > 5e8:
            return None, None, "no stored oracle picks for this cloud"
        idx, _ = oracle.fps(X, wl["n_l"], 0)
        where = "oracle.fps in this run"
    L = X[idx]
    return L, delaunay_complex(L), where


def oracle_sample_costs(X, L, cx, m, fps_iters, n_simplices, seed, index=None):
    """Time the oracle on a bounded sample of the workload itself.

    FPS: `fps_iters` iterations of oracle.fps over all of X (each pick costs one
    pass over X, the same for every pick). Flood values: `n_simplices` simplices
    drawn uniformly from the workload's own complex (dimensions 1-3, FP64 k-d
    tree over the full grid). Returns per-pick and per-simplex seconds.
    """
    import oracle
    t0 = time.perf_counter()
    oracle.fps(X, fps_iters + 1, 0)
    t_pick = (time.perf_counter() - t0) / fps_iters
    counts = [cx.simplices[k].shape[0] for k in (1, 2, 3)]
    rng = np.random.default_rng(seed)
    draw = rng.choice(sum(counts), min(sum(counts), n_simplices), replace=False)
    bounds = np.cumsum([0] + counts)
    subset = [np.zeros(0, np.int64)] + [np.sort(draw[(draw >= bounds[i]) & (draw < bounds[i + 1])] - bounds[i])
                                        for i in range(3)]
    t1 = time.perf_counter()
    oracle.flood_values(X, L, cx.simplices, m, index=index, subset=subset)
    t_simplex = (time.perf_counter() - t1) / max(1, len(draw))
    return t_pick, t_simplex, len(draw)


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo), for the CPU-baseline record."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(X, wl, workload):
    """The oracle as it stands, timed on a bounded sample of the workload's own complex.

    Extrapolated to one step: per-pick FPS cost x (n_L - 1) + k-d tree build +
    per-simplex cost x the complex's simplices (dimensions 1-3).
    """
    import oracle
    L, cx, where = oracle_workload(X, wl, workload)
    if cx is None:
        return None
    t0 = time.perf_counter()
    index = oracle.flood.KDIndex(X, "kdtree")
    t_build = time.perf_counter() - t0
    fps_iters = max(8, int(2e8 // X.shape[0]))                  # a few seconds of FPS passes
    t_pick, t_simplex, sampled = oracle_sample_costs(X, L, cx, wl["m"], fps_iters, 1500, seed=0, index=index)
    n_simp = sum(cx.counts[1:])
    step_s = t_pick * (wl["n_l"] - 1) + t_build + t_simplex * n_simp
    return {"value": n_simp / step_s, "unit": "simplices/s", "cores": os.cpu_count(), "cpu_model": cpu_model(),
            "kind": "oracle", "estimate": True, "step_s_estimated": step_s,
            "threads": "FPS: numpy on one core; k-d tree queries: scipy cKDTree with workers=-1 (all cores)",
            "sample": f"sample of the workload itself, extrapolated to one step: {fps_iters} FPS iterations over all "
                      f"{X.shape[0]} points ({1e3 * t_pick:.1f} ms per pick, x {wl['n_l'] - 1} picks); FP64 k-d tree "
                      f"build ({t_build:.2f} s); flood values of {sampled} simplices drawn uniformly from the "
                      f"workload's own complex of {n_simp} ({1e3 * t_simplex:.2f} ms per simplex); landmarks: "
                      f"{where}"}


def serving_clouds(n_clouds: int, seed: int = 4):
    """Clouds of the batched-serving workload: sizes log-uniform in [2000, 200000],
    shapes from the 8-surface mix (cloud i draws with seed 4000 + i)."""
    from paper_2509_22432_b300 import data
    sizes = data.serving_sizes(n_clouds, seed=seed)
    return [data.shape_mix_cloud(int(n), seed=4000 + i) for i, n in enumerate(sizes)]


def warm_serving(clouds, m: int = 8):
    """Run a few clouds through both server modes first: the first requests of a process pay
    one-time costs (kernel loading, memory-pool growth, imports) that are not serving latency."""
    for batched in (True, False):
        run_serving(clouds[:16], 2000.0, batched, m=m, device_faces=True)


def precompute_tets(clouds, landmark_fraction: float = 0.02) -> dict:
    """Tetrahedra of every serving cloud's landmarks (the server's own FPS picks, computed here by
    flood_fps with the server's landmark count), keyed by the landmarks' float32 bytes: with them
    the server's triangulation callback does no Qhull work, so runs can exclude the host Delaunay."""
    import torch
    from paper_2509_22432_b300 import ops
    from paper_2509_22432_b300.serve import delaunay_tets
    cache = {}
    for X in clouds:
        n = X.shape[0]
        # the server's count: lround of the binary32 fraction times N
        n_l = min(max(int(math.floor(float(np.float32(landmark_fraction)) * n + 0.5)), 4), n)
        idx, _ = ops.fps(torch.from_numpy(X).cuda(), n_l, 0)
        L = np.ascontiguousarray(X[idx.cpu().numpy()], dtype=np.float32)
        cache[L.tobytes()] = delaunay_tets(L)
    return cache


def run_serving(clouds, rate: float, batched: bool, m: int = 8, seed: int = 4, device_faces: bool = False,
                tets_cache: dict | None = None, triangulation_workers: int | None = None) -> dict:
    """Submit the clouds at Poisson arrival times; return clouds/s and latency percentiles.

    batched: the continuous-batching server; otherwise the plain path, one
    cloud at a time through the same kernels (one slot, one worker, batch 1).
    Latency = arrival -> values on the host, host Delaunay included unless
    tets_cache holds every cloud's tetrahedra (precompute_tets).
    device_faces: the host hands over tetrahedra only; faces are built on the device.
    triangulation_workers: host threads running Qhull in the batched server
    (default: one per host core, the measured best; fewer leave the host
    Delaunay the bottleneck at 500 clouds/s).
    """
    from paper_2509_22432_b300 import data
    from paper_2509_22432_b300.serve import Server
    arrivals = data.poisson_arrivals(len(clouds), rate, seed=seed)
    if triangulation_workers is None:
        triangulation_workers = os.cpu_count() or 8
    kw = (dict(max_inflight=64, max_batch=64, gpu_workers=4, triangulation_workers=triangulation_workers) if batched else
          dict(max_inflight=1, max_batch=1, gpu_workers=1, triangulation_workers=1))
    with Server(device_budget_bytes=32 << 30, device_faces=device_faces, tets_cache=tets_cache, **kw) as srv:
        t0 = time.perf_counter()
        tickets = []
        for X, t in zip(clouds, arrivals):
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(X, 0, m))
        res = [srv.result(t, timeout_ms=600_000) for t in tickets]
        st = srv.stats()
        misses = srv.cache_misses
    lat = np.array([r["latency_ms"] for r in res if r["status"] == 0])
    return {"clouds_per_s": st["clouds_per_s"], "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "failed": int(st["failed"]), "batches": int(st["batches"]),
            "mean_batch": float(st["mean_batch"]), "rate_per_s": rate, "clouds": len(clouds),
            "host_delaunay": "excluded (precomputed)" if tets_cache is not None else "included",
            **({"delaunay_cache_misses": int(misses)} if tets_cache is not None else {})}


def run_reference(args, wl):
    """--impl reference: the FP64 oracle, timed on the host cores, on this workload's own complex.

    A full oracle step takes minutes (about 20 ms per FPS pick and a millisecond
    per simplex on one host), so each timed step is a bounded sample of the
    workload: a few FPS passes over all of X and a few dozen simplices of the
    workload's complex. `value` extrapolates the measured per-pick and
    per-simplex costs to one full step (marked as an estimate); ms_per_step is
    the measured time of one sample step.
    """
    import oracle
    X = make_inputs(wl)
    L, cx, where = oracle_workload(X, wl, args.workload)
    if cx is None:
        print(json.dumps({"impl": "reference", "unavailable": f"{where}: the oracle's FPS on this cloud takes too "
                                                              "long to run here"}))
        return
    t0 = time.perf_counter()
    index = oracle.flood.KDIndex(X, "kdtree")
    t_build = time.perf_counter() - t0
    fps_iters, n_sample = 4, 40
    picks, simps, step_ms = [], [], []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        tp, ts, _ = oracle_sample_costs(X, L, cx, wl["m"], fps_iters, n_sample, seed=100 + it, index=index)
        if it >= args.warmup:
            picks.append(tp)
            simps.append(ts)
            step_ms.append(1e3 * (time.perf_counter() - t0))
    n_simp = sum(cx.counts[1:])
    step_s = float(np.mean(picks)) * (wl["n_l"] - 1) + t_build + float(np.mean(simps)) * n_simp
    v = n_simp / step_s
    sample = (f"each step: {fps_iters} oracle FPS iterations over all {X.shape[0]} points and flood values of "
              f"{n_sample} simplices drawn from the workload's own complex ({n_simp} simplices, landmarks: {where}); "
              f"value extrapolates the mean per-pick and per-simplex costs to one full step "
              f"({step_s:.1f} s estimated)")
    line = {"impl": "reference", "metric": "flood simplices/s", "value": v, "unit": "simplices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)),
            "ms_per_step_is": "measured time of one sample step (not a full oracle step)",
            "full_step_s_estimated": step_s, "estimate": True,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_points": wl["n"], "n_landmarks": wl["n_l"], "m": wl["m"]},
            "cpu_baseline": {"value": v, "unit": "simplices/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "simplices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def measure_second_workload(name: str, steps: int, warmup: int, dev, flush) -> dict:
    """The whole step on another workload (the 5M-point shape mix by default), same rules as the main line.

    Landmarks: the CUDA FPS of every step; its picks are compared with the oracle's
    stored picks for this cloud (tests/golden), index for index. The complex is the
    host Delaunay of those landmarks (input, untimed); launch parameters come from
    the autotuner, run first on this workload.
    """
    import torch
    from paper_2509_22432_b300 import delaunay_complex, ops, tune
    wl = WORKLOADS[name]
    X = make_inputs(wl)
    n_l, m = wl["n_l"], wl["m"]
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream(dev)
    idx0, key0 = ops.fps(Xd, n_l, 0)
    golden = _golden_landmarks(name, X)
    exact = None if golden is None else bool(np.array_equal(idx0.cpu().numpy(), golden))
    cx = delaunay_complex(X[idx0.cpu().numpy()])
    dcx = ops.to_device(cx, dev)
    cover = float(np.sqrt(key0[-1].item()))
    tuned = tune.tune_workload(Xd, Xd[idx0], dcx, m, cover, reps=1)
    cell = tuned["cell_factor"] * cover
    times, ph = [], []
    for it in range(warmup + steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        idx, _ = ops.fps(Xd, n_l, 0, sync=False)
        ev[1].record(stream)
        grid = ops.build_grid(Xd, cell, sync=False)
        ev[2].record(stream)
        ops.filtration(grid, ops.gather_rows(Xd, idx, sync=False), dcx, m, want_src=False, sync=False)
        ev[3].record(stream)
        ops.check(dev)
        grid.close()
        if it >= warmup:
            times.append(ev[0].elapsed_time(ev[3]))
            ph.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]),
                       sum(ops.last_filtration_stats()["flood_kernel_ms"])])
    n_simp = sum(cx.counts[1:])
    ms = float(np.mean(times))
    ph = np.mean(np.array(ph), axis=0)
    return {"workload": name, "n_points": wl["n"], "n_landmarks": n_l, "m": m, "simplices_per_step": n_simp,
            "metric": "flood simplices/s", "value": n_simp / (ms * 1e-3), "unit": "simplices/s", "ms_per_step": ms,
            "steps": steps, "warmup": warmup,
            "phase_ms": {"fps": float(ph[0]), "grid": float(ph[1]), "filtration": float(ph[2]),
                         "flood_kernels": float(ph[3])},
            "fps_equals_oracle_picks": exact, "tuning": {"cell_factor": tuned["cell_factor"],
                                                         "heavy_shells": tuned["heavy_shells"]},
            "l2": "flushed between steps", "delaunay": "host, untimed, computed once"}


AMBIENT_DIMS = (2, 3, 4, 5)


def measure_ambient_dimensions(dims, steps: int, warmup: int, dev, flush, peak_tflops: float,
                               cpu_sample: bool) -> dict:
    """The scaling study in the ambient dimension (§5.3, Fig. 4c): swisscheese-like clouds in [0,5]^d,
    |X| = 1M, |L| = 1k, m = 10, through the general-dimension path (flood_fps_nd, flood_build_grid_nd,
    flood_filtration_nd).

    A step is FPS + grid + filtration of every simplex of Del(L) (dimensions 0..d), timed with CUDA
    events, L2 flushed between steps; Del(L) is host input (Qhull), computed once and untimed. The
    picks of d = 4, 5 are compared with the oracle's stored picks (tests/golden). The flood kernels'
    FP32 rate counts the evaluated (sample, point) pairs at 3d - 1 flops each (d differences, one
    product, d - 1 fused multiply-adds). cpu_sample: the oracle (k-d tree, full grid of each simplex)
    timed on 10 simplices per dimension, scaled to the whole complex.
    """
    import torch
    import oracle
    from paper_2509_22432_b300 import data, delaunay_complex, ops
    stream = torch.cuda.current_stream(dev)
    out = {}
    for d in dims:
        n, n_l, m = 1_000_000, 1000, 10
        X = data.swisscheese_cloud(n, seed=6, dim=d)
        Xd = torch.from_numpy(X).to(dev)
        idx0, _ = ops.fps_nd(Xd, n_l, 0)
        golden = _golden_landmarks(f"swisscheese{d}d-1M", X)
        exact = None if golden is None else bool(np.array_equal(idx0.cpu().numpy(), golden))
        L = X[idx0.cpu().numpy()]
        cx = delaunay_complex(L)
        dcx = ops.to_device(cx, dev)
        times, ph = [], []
        for it in range(warmup + steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            idx, _ = ops.fps_nd(Xd, n_l, 0, sync=False)
            ev[1].record(stream)
            grid = ops.build_grid_nd(Xd, 0.0, sync=False)
            ev[2].record(stream)
            ops.filtration_nd(grid, ops.gather_rows(Xd, idx, sync=False), dcx, m, sync=False)
            ev[3].record(stream)
            ops.check(dev)
            if it >= warmup:
                times.append(ev[0].elapsed_time(ev[3]))
                ph.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
            info = grid.info()
            grid.close()
        st = ops.last_filtration_nd_stats()
        ms = float(np.mean(times))
        ph = np.mean(np.array(ph), axis=0)
        pairs = int(sum(st["pairs"]) + sum(st["pairs_fallback"]))
        achieved = pairs * (3 * d - 1) / (ph[2] * 1e-3) / 1e12
        n_simp = int(sum(cx.counts[1:]))
        rec = {"workload": f"swisscheese{d}d-1M", "d": d, "n_points": n, "n_landmarks": n_l, "m": m,
               "simplices": cx.counts, "simplices_per_step": n_simp, "items": int(sum(st["items"])),
               "metric": "flood simplices/s", "value": n_simp / (ms * 1e-3), "unit": "simplices/s",
               "ms_per_step": ms, "steps": steps, "warmup": warmup,
               "phase_ms": {"fps": float(ph[0]), "grid": float(ph[1]), "filtration": float(ph[2])},
               "fps_equals_oracle_picks": exact,
               "grid": {"cell_size": info["cell_size"], "n_cells": info["n_cells"]},
               "work": {k: int(sum(v)) for k, v in st.items() if k != "dim"},
               "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                            "frac": achieved / peak_tflops, "evaluated_pairs": pairs, "flops_per_pair": 3 * d - 1,
                            "kernel": "k_nd_resolve + k_nd_fallback (all dimensions of one filtration)"},
               "l2": "flushed between steps", "delaunay": "host, untimed, computed once"}
        if cpu_sample:
            rng = np.random.default_rng(5)
            subset = [np.arange(0)] + [rng.choice(c, min(10, c), replace=False) for c in cx.counts[1:]]
            index = oracle.flood.KDIndex(X, "kdtree")
            t0 = time.perf_counter()
            oracle.flood_values(X, L, cx.simplices, m, method="kdtree", index=index, subset=subset)
            t = time.perf_counter() - t0
            est = sum(t / sum(len(x) for x in subset[1:]) * c for c in cx.counts[1:])
            rec["cpu_baseline"] = {"kind": "oracle", "cores": 1, "sample": f"{sum(len(x) for x in subset[1:])} "
                                   "simplices (10 per dimension, full grid, k-d tree over X), scaled to the complex",
                                   "seconds_estimate": est, "simplices_per_s": n_simp / est}
        out[f"d{d}"] = rec
        del Xd
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus-1M", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--second-workload", default="shapes-5M", choices=sorted(WORKLOADS) + ["none"],
                    help="a second workload timed the same way and reported beside the main line")
    ap.add_argument("--ambient-dims", default=",".join(str(d) for d in AMBIENT_DIMS),
                    help="ambient dimensions of the Fig. 4c scaling leg (comma list, or 'none')")
    ap.add_argument("--no-tune", action="store_true",
                    help="take the tuning table's parameters instead of sweeping them first (profiling runs)")
    ap.add_argument("--serving", action="store_true",
                    help="sweep the batched-serving workload (512 clouds, Poisson rates 50..2000/s)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    import torch
    import torch.distributed as dist

    from paper_2509_22432_b300 import data, delaunay_complex, ops

    if args.serving:
        if rank == 0:
            clouds = serving_clouds(512)
            warm_serving(clouds)
            cache = precompute_tets(clouds)
            for rate in (50, 100, 200, 500, 1000, 2000):
                for batched in (True, False):
                    for tc in (None, cache):
                        r = run_serving(clouds, rate, batched, device_faces=True, tets_cache=tc)
                        print(json.dumps({"serving": "batched" if batched else "per-cloud", "faces": "device",
                                          "device_budget_bytes": 32 << 30, **r}), flush=True)
        return

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    X = make_inputs(wl, seed_offset=rank)
    n_l, m = wl["n_l"], wl["m"]
    Xd = torch.from_numpy(X).to(dev)
    idx0, key0 = ops.fps(Xd, n_l, 0)
    L_host = X[idx0.cpu().numpy()]
    cx = delaunay_complex(L_host)
    dcx = ops.to_device(cx, dev)
    # launch parameters by the project's autotuner (untimed): grid cell factor and
    # heavy-group threshold, measured on this workload and kept in the tuning table
    from paper_2509_22432_b300 import tune
    cover = float(np.sqrt(key0[-1].item()))                # FPS covering radius
    if args.no_tune:
        t = tune.lookup(wl["n"], n_l, m)
        tuned = {"cell_factor": t["cell_factor"], "heavy_shells": t["heavy_shells"], "ms": None, "default_ms": None}
    else:
        tuned = tune.tune_workload(Xd, Xd[idx0], dcx, m, cover)
    cell = tuned["cell_factor"] * cover
    n_simp = sum(cx.counts[1:])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)

    phase_events = []

    def step(record=False):
        # every call is asynchronous (no host wait inside the step); the stream's
        # status is checked once at the end of the step (ops.check)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
        if record:
            ev[0].record(stream)
        idx, key = ops.fps(Xd, n_l, 0, sync=False)
        if record:
            ev[1].record(stream)
        grid = ops.build_grid(Xd, cell, sync=False)
        if record:
            ev[2].record(stream)
        L = ops.gather_rows(Xd, idx, sync=False)
        vals, _ = ops.filtration(grid, L, dcx, m, want_src=False, sync=False)
        if record:
            ev[3].record(stream)
            phase_events.append(ev)
        return idx, vals, grid

    clocks = ClockSampler(local).__enter__()  # running before the timed region; samples filtered to it
    for _ in range(args.warmup):
        idx, vals, grid = step()
        ops.check(dev)
        grid.close()
    assert torch.equal(idx, idx0), "FPS must be deterministic"
    stats = ops.last_filtration_stats()

    # ---- device-timed steps (inputs resident in HBM; L2 flushed between steps)
    times, flood_ms = [], []
    launches0 = ops.kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    time.sleep(0.3)  # the sampler's first lines arrive after a short start-up
    t_region0 = time.monotonic()
    try:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, grid = step(record=True)
            e1.record(stream)
            ops.check(dev)                  # waits for the step; raises if any call of it failed
            grid.close()
            times.append(e0.elapsed_time(e1))
            flood_ms.append(sum(ops.last_filtration_stats()["flood_kernel_ms"]))
        torch.cuda.synchronize()
    finally:
        clocks.mark(t_region0, time.monotonic())
        clocks.__exit__(None, None, None)
    launches = ops.kernel_launches() - launches0
    ms, total_simplices = aggregate(float(np.mean(times)), float(n_simp), dev)

    # ---- end to end through the public API with host buffers
    Xh = torch.from_numpy(X).pin_memory()
    # the complex's int32 arrays packed in one pinned buffer: one upload per step, device views
    cx_parts = [t.cpu() for t in dcx.simplices] + [t.cpu() for t in dcx.facets]
    cx_h = torch.cat([t.reshape(-1) for t in cx_parts]).pin_memory()
    cx_offs = np.concatenate([[0], np.cumsum([t.numel() for t in cx_parts])]).tolist()
    n_simp_parts = len(dcx.simplices)
    h2d = Xh.numel() * 4 + cx_h.numel() * 4
    d2h = n_l * 8 + sum(cx.counts) * 4
    e2e_times = []
    idx_out = torch.empty(n_l, dtype=torch.int64).pin_memory()
    val_out = torch.empty(sum(cx.counts), dtype=torch.float32).pin_memory()
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xg = Xh.to(dev, non_blocking=True)
        idx, key = ops.fps(Xg, n_l, 0, sync=False)
        idx_out.copy_(idx, non_blocking=True)  # the landmarks go to the host (the triangulation's input)
        stream.synchronize()
        cx_d = cx_h.to(dev, non_blocking=True)
        views = [cx_d[cx_offs[i]:cx_offs[i + 1]].view(cx_parts[i].shape) for i in range(len(cx_parts))]
        dc = ops.DeviceComplex(cx.n_vertices, views[:n_simp_parts], views[n_simp_parts:])
        grid = ops.build_grid(Xg, cell, sync=False)
        vals, _ = ops.filtration(grid, ops.gather_rows(Xg, idx, sync=False), dc, m, want_src=False, sync=False)
        off = 0
        for v in vals:                      # the values go to the host: one pinned buffer, one wait
            val_out[off:off + v.numel()].copy_(v, non_blocking=True)
            off += v.numel()
        ops.check(dev)                      # waits for the stream; raises if any call of the step failed
        if it >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
        grid.close()
    e2e_s = float(np.mean(e2e_times))
    # the last end-to-end step's results equal the resident-input step's, bit for bit
    grid_r = ops.build_grid(Xd, cell)
    vals_r, _ = ops.filtration(grid_r, Xd[idx0], dcx, m, want_src=False)
    grid_r.close()
    e2e_exact = bool(torch.equal(idx_out, idx0.cpu()) and
                     torch.equal(val_out.view(torch.int32), torch.cat([v.cpu() for v in vals_r]).view(torch.int32)))
    if not e2e_exact:
        raise RuntimeError("end-to-end step results differ from the resident-input step")

    # ---- the same step with uniform random point sets P_sigma (§4.1, Lemma 4)
    # in place of the grid: as many points per simplex as the grid's interior
    # samples at this m, drawn independently per simplex.
    S_rand = [math.comb(m - 1, k) for k in (1, 2, 3)]
    w_rand = [None] + [torch.from_numpy(data.random_barycentric(cx.counts[k], S_rand[k - 1], k, seed=7)).to(dev)
                       for k in (1, 2, 3)]
    rs_times, rs_filt, rs_flood = [], [], []
    for it in range(args.warmup + min(args.steps, 10)):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        idx, key = ops.fps(Xd, n_l, 0)
        grid = ops.build_grid(Xd, cell)
        e[1].record(stream)
        vals, _ = ops.filtration_given(grid, ops.gather_rows(Xd, idx), dcx, w_rand, want_src=False)
        e[2].record(stream)
        e[2].synchronize()
        grid.close()
        if it >= args.warmup:
            rs_times.append(e[0].elapsed_time(e[2]))
            rs_filt.append(e[1].elapsed_time(e[2]))
            rs_flood.append(sum(ops.last_filtration_stats()["flood_kernel_ms"]))
    rs_stats = ops.last_filtration_stats()
    del w_rand

    peaks, peak_kind = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    fps_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in phase_events]))

    # ---- FP32 peak of this GPU, measured: a pure-FMA kernel (scalar and packed
    # forms) timed with CUDA events, clocks sampled while it runs
    def probe(packed, iters=40_000):
        ops.fp32_peak_probe(dev, packed, 2000)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl = ops.fp32_peak_probe(dev, packed, iters)
            b.record(stream)
            b.synchronize()
            best = max(best, fl / (a.elapsed_time(b) * 1e-3) / 1e12)
        return best

    pclk = ClockSampler(local).__enter__()
    time.sleep(0.3)
    tp0 = time.monotonic()
    peak_scalar, peak_packed = probe(False), probe(True)
    pclk.mark(tp0, time.monotonic())
    pclk.__exit__(None, None, None)
    peak_tflops = max(peak_scalar, peak_packed)

    # ---- flood kernels on the FP32 pipe: evaluated pairs x 6 flops / their event time
    pairs = sum(stats["pairs"])
    fk = float(np.mean(flood_ms))
    achieved = pairs * FLOPS_PER_PAIR / (fk * 1e-3) / 1e12
    queries = sum(stats["samples"][1:])
    # the method's own work (§8(d)): interior samples x points of X in each
    # simplex's Lemma 2 masking ball, counted on the device
    gb = ops.build_grid(Xd, cell)
    ball = ops.masking_ball_counts(gb, Xd[idx0], dcx)
    gb.close()
    interior = [0] + [math.comb(m - 1, k) for k in (1, 2, 3)]
    alg_pairs = sum(interior[k] * ball[k] for k in (1, 2, 3))

    # ---- FPS: latency of the exchange rounds. Floor: the same launch width on
    # a cloud of one chunk per block (the exchange with almost no chunk work).
    fst = ops.fps_stats()
    rounds = max(1, fst["rounds"])
    Xd_fps = torch.from_numpy(X).to(dev)

    def fps_time(Xs, k, nb=0):
        best = float("inf")
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops.fps(Xs, k, 0, n_blocks=nb)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best, ops.fps_stats()

    late_us = 1e3 * (fps_time(Xd_fps, n_l)[0] - fps_time(Xd_fps, n_l // 2)[0]) / (n_l - n_l // 2)
    small = torch.from_numpy(data.sphere_cloud(fst["blocks"] * 256, seed=77)).to(dev)
    n_floor = min(n_l, small.shape[0])
    floor_ms, floor_st = fps_time(small, n_floor, nb=fst["blocks"])
    floor_round_us = 1e3 * floor_ms / max(1, floor_st["rounds"])
    floor_pick_us = 1e3 * floor_ms / max(1, n_floor - 1)
    round_us = 1e3 * fps_ms / rounds
    pick_us = 1e3 * fps_ms / max(n_l - 1, 1)
    del Xd_fps, small
    line = {
        "metric": "flood simplices/s", "value": total_simplices / (ms * 1e-3), "unit": "simplices/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_points": wl["n"], "n_landmarks": n_l, "m": m,
                   "simplices_per_step": n_simp, "simplex_counts": cx.counts, "cell_size": cell,
                   "tuning": {"cell_factor": tuned["cell_factor"], "heavy_shells": tuned["heavy_shells"],
                              "grid_and_filtration_ms": tuned["ms"], "at_defaults_ms": tuned["default_ms"],
                              "by": "paper_2509_22432_b300.tune: every (cell factor, heavy threshold) candidate "
                                    "timed with CUDA events on this workload before the timed steps"},
                   "l2": "flushed between steps (256 MB write)", "delaunay": "host, untimed, computed once",
                   "parallelism": f"replicas x{world}"},
        "nn_queries_per_s": world * queries / (ms * 1e-3),
        "pairs_per_step": pairs,
        "phase_ms": {"fps": fps_ms,
                     "grid": float(np.mean([e[1].elapsed_time(e[2]) for e in phase_events])),
                     "filtration": float(np.mean([e[2].elapsed_time(e[3]) for e in phase_events])),
                     "flood_kernels": fk},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": _flood_traffic(args.workload, tuned),
                     "traffic_unit": "DRAM bytes of the six flood launches of one filtration (ncu, at cell factor "
                                     f"{FLOOD_DRAM_CAPTURE['cell_factor']:g} and heavy threshold "
                                     f"{FLOOD_DRAM_CAPTURE['heavy_shells']}; null when the step runs at other "
                                     "parameters or another filtration source)",
                     "kernel": "k_flood_heavy + k_flood (dimensions 1-3), the largest stage of the step",
                     "flops_per_pair": FLOPS_PER_PAIR,
                     "evaluated_pairs": pairs,
                     "algorithmic_pairs": alg_pairs,
                     "algorithmic_pairs_are": "sum over simplices of C(m-1,k) interior samples x |X in the Lemma 2 "
                                              "masking ball| (the method's own work); the kernels evaluate "
                                              "evaluated_pairs of them after exact pruning",
                     "algorithmic_over_evaluated": alg_pairs / max(1, pairs),
                     "peak_kind": "measured in this run: pure-FMA kernel (flood_fp32_peak_probe), best of scalar "
                                  "and packed forms",
                     "peak_scalar": peak_scalar, "peak_packed": peak_packed, "peak_clocks": pclk.summary(),
                     "nominal_peak": sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12},
        "roofline_fps": {"bound": "latency", "kernel": "k_fps_resident" if fst["resident"] else "k_fps_global",
                         "rounds": rounds, "picks": n_l, "blocks": fst["blocks"],
                         "per_round_us": round_us, "per_pick_us": pick_us, "late_per_pick_us": late_us,
                         "floor_per_round_us": floor_round_us, "floor_per_pick_us": floor_pick_us,
                         "floor_rounds": floor_st["rounds"],
                         "picks_per_round": (n_l - 1) / rounds,
                         "floor_picks_per_round": (n_floor - 1) / max(1, floor_st["rounds"]),
                         "floor_note": "per pick the floor is a floor; per round it need not be (its rounds "
                                       "can make more picks, each costing selection time)",
                         "floor_is": f"the same kernel and launch width ({fst['blocks']} blocks) on a cloud of one "
                                    f"256-point chunk per block, {n_floor} picks: the grid exchange and pick "
                                    "selection with almost no chunk work",
                         "frac": floor_pick_us / pick_us,
                         "frac_is": "floor per pick / this workload's per pick"},
        "e2e": {"value": world * n_simp / e2e_s, "unit": "simplices/s", "results_equal_resident_step": e2e_exact,
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
    }
    # ---- the paper's own design on the same GPU (§4.2, App. A.1): every full-grid
    # sample against every point in its simplex's masking ball, no pruning
    grid = ops.build_grid(Xd, cell)
    L_dev = Xd[idx0]
    mk_ms, mk_pairs = [], 0
    # the comparator holds the full grid of a tetrahedron in shared memory: C(m+3, 3) <= 1024
    for it in range(3 if math.comb(m + 3, 3) <= 1024 else 0):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, mk_pairs = ops.filtration_masked(grid, L_dev, dcx, m)
        e1.record(stream)
        e1.synchronize()
        if it >= 1:
            mk_ms.append(e0.elapsed_time(e1))
    grid.close()
    mk = float(np.median(mk_ms)) if mk_ms else float("nan")

    # ---- faces and facet incidence of the workload's tetrahedra: device vs host builder
    from paper_2509_22432_b300.complex import complex_from_simplices
    tets_h = np.ascontiguousarray(cx.simplices[3], dtype=np.int32)
    tets_d = torch.from_numpy(tets_h).to(dev)
    fc_dev = []
    for it in range(args.warmup + min(args.steps, 10)):
        t0 = time.perf_counter()
        ops.complex_faces(tets_d, n_l)                 # synchronises its stream
        if it >= args.warmup:
            fc_dev.append(1e3 * (time.perf_counter() - t0))
    t0 = time.perf_counter()
    complex_from_simplices([tets_h], n_l, top_dim=3)
    fc_host = 1e3 * (time.perf_counter() - t0)
    rs_ms, _ = aggregate(float(np.mean(rs_times)), float(n_simp), dev)
    rs_pairs = sum(rs_stats["pairs"])
    rs_fk = float(np.mean(rs_flood))
    rs_tflops = rs_pairs * FLOPS_PER_PAIR / (rs_fk * 1e-3) / 1e12
    line["random_sets"] = {
        "metric": "flood simplices/s", "value": world * n_simp / (rs_ms * 1e-3), "unit": "simplices/s",
        "ms_per_step": rs_ms, "steps": len(rs_times),
        "points_per_simplex": S_rand, "draw": "uniform on each simplex, independent per simplex (seed 7)",
        "nn_queries_per_s": world * sum(rs_stats["samples"][1:]) / (rs_ms * 1e-3),
        "phase_ms": {"fps_and_grid": float(np.mean(rs_times)) - float(np.mean(rs_filt)),
                     "filtration": float(np.mean(rs_filt)), "flood_kernels": rs_fk},
        "pairs_per_step": rs_pairs,
        "roofline_flood": {"bound": "alu", "achieved": rs_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                           "frac": rs_tflops / peak_tflops}}
    filt_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in phase_events]))
    line["paper_masked"] = {"skipped": f"m = {m}: the comparator holds at most 1024 full-grid samples per "
                                       "simplex (m <= 15)"} if not mk_ms else {
        "what": "the paper's evaluation on this GPU: full grid (faces included) x points in the Lemma 2 "
                "masking ball, no pruning (flood_filtration_masked)",
        "filtration_ms": mk, "pairs": int(mk_pairs), "simplices_per_s": world * n_simp / (mk * 1e-3),
        "pruned_filtration_ms": filt_ms, "pruned_pairs": pairs, "speedup_of_pruned": mk / filt_ms,
        "pair_rate_per_s": mk_pairs / (mk * 1e-3),
        # implementation-independent floor: its pairs at the FP32 ALU peak (direct form |x - p|^2:
        # 3 FSUB + 2 FFMA + 1 FMUL + 1 FMNMX = 7 instructions per pair and lane)
        "alu_floor_ms": 1e3 * mk_pairs * 7 / (sms * FP32_LANES_PER_SM * sm_max * 1e6),
        "pair_ratio": mk_pairs / max(pairs, 1)}
    # ---- persistence pairs of the step's filtration on the device (§2; the PH share of Table 1)
    gph = ops.build_grid(Xd, cell)
    ph_vals, _ = ops.filtration(gph, Xd[idx0], dcx, m, want_src=False)
    gph.close()
    ph_ms = []
    for it in range(args.warmup + min(args.steps, 10)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ph = ops.persistence(dcx, ph_vals)            # synchronises its stream
        if it >= args.warmup:
            ph_ms.append(1e3 * (time.perf_counter() - t0))
    line["persistence"] = {"device_ms": float(np.median(ph_ms)), "pairs": [int(p.shape[0]) for p in ph["pairs"]],
                           "essential": [int(e.numel()) for e in ph["essential"]], "rounds": ph["rounds"],
                           "what": "flood_persistence on the step's values: per-dimension bitonic order, parallel "
                                   "Z/2 column reduction with clearing (call to return, synchronised)"}
    ph_values = [v.cpu().numpy().astype(np.float64) for v in ph_vals]
    if args.second_workload not in ("none", args.workload):
        line["second_workload"] = measure_second_workload(args.second_workload, min(args.steps, 10), args.warmup,
                                                          dev, flush)
    if rank == 0 and args.ambient_dims != "none":
        dims = [int(x) for x in args.ambient_dims.split(",") if x]
        line["ambient_dimension"] = measure_ambient_dimensions(dims, min(args.steps, 5), args.warmup, dev, flush,
                                                               peak_tflops, not args.no_cpu_baseline)
    line["complex_faces"] = {"tetrahedra": int(cx.counts[3]), "device_ms": float(np.median(fc_dev)),
                             "host_ms": fc_host, "what": "triangles, edges and facet incidence from the "
                             "tetrahedra: flood_complex_faces (call to return, synchronised) vs the host "
                             "numpy builder"}
    if rank == 0 and not args.no_serving:
        clouds = serving_clouds(512)
        warm_serving(clouds)
        cache = precompute_tets(clouds)
        runs = {}
        for rate in (50.0, 500.0):
            runs[f"{rate:g}"] = {"batched": run_serving(clouds, rate, True, device_faces=True),
                                 "per_cloud": run_serving(clouds, rate, False, device_faces=True),
                                 "batched_no_delaunay": run_serving(clouds, rate, True, device_faces=True,
                                                                    tets_cache=cache)}
        line["serving"] = {"workload": "512 clouds, 2k-200k points (log-uniform), shape mix, Poisson arrivals, "
                                       f"n_L = 2% of points, m = 8, device budget 32 GB, host Delaunay (Qhull, {os.cpu_count()} "
                                       "threads for the batched server) included except in batched_no_delaunay "
                                       "(tetrahedra precomputed from the same landmarks), faces built on the "
                                       "device in every arm",
                           "by_rate": runs,
                           "arms": "batched: continuous batching (64 slots, batches of up to 64 clouds); per_cloud: "
                                   "the same kernels one cloud at a time (one slot, batch 1)",
                           "warm_up": "16 clouds through each server mode before the timed runs"}
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(X, wl, args.workload)
        if cb is not None:
            line["cpu_baseline"] = cb
        # the oracle's host reduction of the same filtration, beside the device's
        import oracle
        t0 = time.perf_counter()
        oracle.persistence_pairs(cx.simplices, cx.facets, ph_values)
        line["persistence"]["host_oracle_ms"] = 1e3 * (time.perf_counter() - t0)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
