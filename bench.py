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
# DRAM bytes (read + write) of one k_fps_resident launch on torus-1M, from one
# ncu capture (profiles/k_fps_resident_torus-1M.md), valid only while the FPS
# source is the one captured: reported as null once fps.cu changes.
FPS_DRAM_CAPTURE = {"workload": "torus-1M", "bytes": 16_084_736 + 10_752,
                    "fps_cu_sha256": "f7d7282ff41ccb5c33e4f7c3cae06bcc10b9f14969de5dd912944eeb780dcb36"}


def _fps_traffic(workload: str):
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_2509_22432_b300", "csrc", "fps.cu"), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    cap = FPS_DRAM_CAPTURE
    if workload != cap["workload"] or digest != cap["fps_cu_sha256"]:
        return None
    return float(cap["bytes"])


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


def cpu_baseline(X, wl, budget_s: float = 20.0):
    """The oracle as it stands, on a bounded sample of the same workload.

    Sample: FPS for a fixed number of iterations on all of X, the FP64 k-d
    tree over X, and flood values (full barycentric grid, FP64) of a random
    sample of simplices; extrapolated to one full step in simplices/s.
    """
    import oracle
    from paper_2509_22432_b300 import delaunay_complex

    t0 = time.perf_counter()
    j = 24
    idx, _ = oracle.fps(X, j, 0)
    t_fps_iter = (time.perf_counter() - t0) / (j - 1)
    t_fps = t_fps_iter * (wl["n_l"] - 1)
    idx, _ = oracle.fps(X, min(wl["n_l"], 400), 0)     # landmarks for a representative complex
    L = X[idx]
    cx = delaunay_complex(L)
    t1 = time.perf_counter()
    index = oracle.flood.KDIndex(X, "kdtree")
    t_build = time.perf_counter() - t1
    rng = np.random.default_rng(0)
    per_dim, sampled = [], 0
    remaining = max(1.0, budget_s - (time.perf_counter() - t0))
    sub = [None] * 4
    for k in (1, 2, 3):
        n = cx.simplices[k].shape[0]
        sub[k] = rng.choice(n, min(n, 300), replace=False)
    t2 = time.perf_counter()
    res = oracle.flood_values(X, L, cx.simplices, wl["m"], index=index,
                              subset=[np.zeros(0, np.int64)] + sub[1:])
    t_sample = time.perf_counter() - t2
    sampled = sum(len(s) for s in sub[1:])
    per_simplex = t_sample / sampled
    return {"per_simplex_s": per_simplex, "t_fps_s": t_fps, "t_build_s": t_build, "sampled": sampled,
            "note": f"FPS {j} iterations on all {X.shape[0]} points; k-d tree build; "
                    f"flood values of {sampled} random simplices (dims 1-3) of a {L.shape[0]}-landmark Delaunay"}


def serving_clouds(n_clouds: int, seed: int = 4):
    """Clouds of the batched-serving workload: sizes log-uniform in [2000, 200000],
    shapes from the 8-surface mix (cloud i draws with seed 4000 + i)."""
    from paper_2509_22432_b300 import data
    sizes = data.serving_sizes(n_clouds, seed=seed)
    return [data.shape_mix_cloud(int(n), seed=4000 + i) for i, n in enumerate(sizes)]


def run_serving(clouds, rate: float, batched: bool, m: int = 8, seed: int = 4, device_faces: bool = False) -> dict:
    """Submit the clouds at Poisson arrival times; return clouds/s and latency percentiles.

    batched: the continuous-batching server; otherwise the plain path, one
    cloud at a time through the same kernels (one slot, one worker, batch 1).
    Latency = arrival -> values on the host, host Delaunay included.
    device_faces: the host hands over tetrahedra only; faces are built on the device.
    """
    from paper_2509_22432_b300 import data
    from paper_2509_22432_b300.serve import Server
    arrivals = data.poisson_arrivals(len(clouds), rate, seed=seed)
    kw = (dict(max_inflight=64, max_batch=64, gpu_workers=4, triangulation_workers=8) if batched else
          dict(max_inflight=1, max_batch=1, gpu_workers=1, triangulation_workers=1))
    with Server(device_budget_bytes=32 << 30, device_faces=device_faces, **kw) as srv:
        t0 = time.perf_counter()
        tickets = []
        for X, t in zip(clouds, arrivals):
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(X, 0, m))
        res = [srv.result(t, timeout_ms=600_000) for t in tickets]
        st = srv.stats()
    lat = np.array([r["latency_ms"] for r in res if r["status"] == 0])
    return {"clouds_per_s": st["clouds_per_s"], "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "failed": int(st["failed"]), "batches": int(st["batches"]),
            "mean_batch": float(st["mean_batch"]), "rate_per_s": rate, "clouds": len(clouds)}


def run_reference(args, wl):
    """--impl reference: the FP64 oracle timed on the host cores."""
    X = make_inputs(wl)
    res = cpu_baseline(X, wl)
    # simplex count of the full workload's complex, estimated from the landmark count
    n_simplices = 28.1 * wl["n_l"]
    step_s = res["t_fps_s"] + res["t_build_s"] + res["per_simplex_s"] * n_simplices
    v = n_simplices / step_s
    line = {"impl": "reference", "metric": "flood simplices/s", "value": v, "unit": "simplices/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_points": wl["n"], "n_landmarks": wl["n_l"], "m": wl["m"]},
            "cpu_baseline": {"value": v, "unit": "simplices/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": res["note"]},
            "e2e": {"value": v, "unit": "simplices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus-1M", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
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
            for rate in (50, 100, 200, 500, 1000, 2000):
                for batched in (True, False):
                    r = run_serving(clouds, rate, batched, device_faces=True)
                    print(json.dumps({"serving": "batched" if batched else "per-cloud", "faces": "device", **r}),
                          flush=True)
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
    grid0 = ops.build_grid(Xd, 0.0)
    cell = 0.5 * float(np.sqrt(key0[-1].item()))           # half the FPS covering radius
    grid0.close()
    n_simp = sum(cx.counts[1:])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)

    phase_events = []

    def step(record=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
        if record:
            ev[0].record(stream)
        idx, key = ops.fps(Xd, n_l, 0)
        if record:
            ev[1].record(stream)
        grid = ops.build_grid(Xd, cell)
        if record:
            ev[2].record(stream)
        L = Xd[idx]
        vals, _ = ops.filtration(grid, L, dcx, m, want_src=False)
        if record:
            ev[3].record(stream)
            phase_events.append(ev)
        grid.close()
        return idx, vals

    clocks = ClockSampler(local).__enter__()  # running before the timed region; samples filtered to it
    for _ in range(args.warmup):
        idx, vals = step()
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
            step(record=True)
            e1.record(stream)
            e1.synchronize()
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
    simp_h = [t.cpu().pin_memory() for t in dcx.simplices]
    fac_h = [t.cpu().pin_memory() for t in dcx.facets]
    h2d = Xh.numel() * 4 + sum(t.numel() * 4 for t in simp_h + fac_h)
    d2h = n_l * 8 + sum(cx.counts) * 4
    e2e_times = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xg = Xh.to(dev, non_blocking=True)
        idx, key = ops.fps(Xg, n_l, 0)
        idx_h = idx.cpu()
        dc = ops.DeviceComplex(cx.n_vertices, [t.to(dev, non_blocking=True) for t in simp_h],
                               [t.to(dev, non_blocking=True) for t in fac_h])
        grid = ops.build_grid(Xg, cell)
        vals, _ = ops.filtration(grid, Xg[idx_h.to(dev)], dc, m, want_src=False)
        out = [v.cpu() for v in vals]
        grid.close()
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_times))

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
        vals, _ = ops.filtration_given(grid, Xd[idx], dcx, w_rand, want_src=False)
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
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    pairs = sum(stats["pairs"])
    fk = float(np.mean(flood_ms))
    achieved = pairs * FLOPS_PER_PAIR / (fk * 1e-3) / 1e12
    queries = sum(stats["samples"][1:])
    # FPS: algorithmic bytes of one iteration = 12N (coordinates) + 8N (read and
    # write the running minimum); the kernel keeps them on chip, so this is an
    # effective bandwidth against the measured HBM copy bandwidth.
    fps_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in phase_events]))
    fps_bytes = 20.0 * wl["n"] * (n_l - 1)
    fps_gbs = fps_bytes / (fps_ms * 1e-3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    # Per-pick cost of the late picks (few chunks still change; the grid-wide
    # exchange dominates): difference of two FPS calls, n_l and n_l / 2 picks.
    Xd_fps = torch.from_numpy(X).to(dev)

    def fps_time(k):
        best = float("inf")
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops.fps(Xd_fps, k, 0)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    late_us = 1e3 * (fps_time(n_l) - fps_time(n_l // 2)) / (n_l - n_l // 2)
    del Xd_fps
    line = {
        "metric": "flood simplices/s", "value": total_simplices / (ms * 1e-3), "unit": "simplices/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_points": wl["n"], "n_landmarks": n_l, "m": m,
                   "simplices_per_step": n_simp, "simplex_counts": cx.counts, "cell_size": cell,
                   "l2": "flushed between steps (256 MB write)", "delaunay": "host, untimed, computed once",
                   "parallelism": f"replicas x{world}"},
        "nn_queries_per_s": world * queries / (ms * 1e-3),
        "pairs_per_step": pairs,
        "phase_ms": {"fps": float(np.mean([e[0].elapsed_time(e[1]) for e in phase_events])),
                     "grid": float(np.mean([e[1].elapsed_time(e[2]) for e in phase_events])),
                     "filtration": float(np.mean([e[2].elapsed_time(e[3]) for e in phase_events])),
                     "flood_kernels": fk},
        "roofline": {"bound": "hbm", "achieved": fps_gbs, "peak": hbm, "unit": "GB/s", "frac": fps_gbs / hbm,
                     "traffic": _fps_traffic(args.workload), "traffic_unit": "bytes per launch",
                     "kernel": "k_fps_resident (FPS, dominant by time)", "effective": True,
                     "algorithmic_bytes": "20 N per pick (12N coordinates + 8N running minima) of the streaming "
                                          "algorithm; effective: points stay on chip and chunks whose minima "
                                          "provably cannot change are skipped (exact)",
                     "per_pick_us": 1e3 * fps_ms / max(n_l - 1, 1), "late_per_pick_us": late_us,
                     "peak_kind": f"{peak_kind} hbm_gbs"},
        "roofline_flood": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                           "frac": achieved / peak_tflops, "kernel": "k_flood + k_flood_heavy (all dims)",
                           "flops_per_pair": FLOPS_PER_PAIR,
                           "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz"},
        "e2e": {"value": world * n_simp / e2e_s, "unit": "simplices/s", "h2d_bytes_per_step": int(h2d),
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
    line["complex_faces"] = {"tetrahedra": int(cx.counts[3]), "device_ms": float(np.median(fc_dev)),
                             "host_ms": fc_host, "what": "triangles, edges and facet incidence from the "
                             "tetrahedra: flood_complex_faces (call to return, synchronised) vs the host "
                             "numpy builder"}
    if rank == 0 and not args.no_serving:
        clouds = serving_clouds(128)
        b = run_serving(clouds, 500.0, True, device_faces=False)
        bd = run_serving(clouds, 500.0, True, device_faces=True)
        p = run_serving(clouds, 500.0, False, device_faces=False)
        line["serving"] = {"workload": "128 clouds, 2k-200k points (log-uniform), shape mix, Poisson 500/s, "
                                       "n_L = 2% of points, m = 8, host Delaunay included",
                           "batched": b, "batched_device_faces": bd, "per_cloud": p,
                           "modes": "batched and per_cloud: whole complex built on the host; "
                                    "batched_device_faces (the server's default): tetrahedra from the host, "
                                    "faces built on the device"}
    if rank == 0 and not args.no_cpu_baseline:
        res = cpu_baseline(X, wl)
        step_s = res["t_fps_s"] + res["t_build_s"] + res["per_simplex_s"] * n_simp
        line["cpu_baseline"] = {"value": n_simp / step_s, "unit": "simplices/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": res["note"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
