"""Autotuner of the filtration's launch parameters (the tuning table of libflood).

Two parameters change the speed of a filtration but never its results: the
grid cell edge as a multiple of the FPS covering radius, and the shell count
from which a sample group runs on a whole CTA (see flood_tuning in
include/flood.h). This module measures them on a workload: for every
candidate pair it builds the grid and runs the filtration, timed with CUDA
events on the current stream, keeps the fastest, and records it in the
library's table under the workload's bucket (SM count, log2 points, log2
landmarks, m). The table is written to and read from a plain text file
(FLOOD_TUNE_CACHE, else ~/.cache/paper_2509_22432_b300/tune.txt).

Usage:
    python -m paper_2509_22432_b300.tune --serving      # buckets of the serving workload (shape mix, 2k-200k)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _lib

__all__ = ["Entry", "cache_path", "lookup", "set_entry", "entries", "clear", "load", "save", "bucket",
           "choose", "tune_workload", "tune_cloud"]

CELL_FACTORS = (0.35, 0.5, 0.7, 1.0)
HEAVY_SHELLS = (7, 8, 9, 10, 12)
DEFAULTS = (0.5, 9)        # the library's parameters when a bucket has no entry
KEEP_DEFAULTS_WITHIN = 0.02  # a candidate must beat the defaults by more than this to replace them


Entry = _lib.TuningEntry


def _lib_tune():
    return _lib.get()


def cache_path() -> str:
    return os.environ.get("FLOOD_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                              "paper_2509_22432_b300", "tune.txt")


def _log2(v: int) -> int:
    return 0 if v <= 1 else int(round(np.log2(float(v))))


def bucket(n_points: int, n_landmarks: int, m: int, sm_count: int) -> tuple:
    """The table key of a workload: (SM count, round(log2 points), round(log2 landmarks), m)."""
    return (int(sm_count), _log2(n_points), _log2(n_landmarks), int(m))


def lookup(n_points: int, n_landmarks: int, m: int) -> dict:
    """Parameters the library uses for this workload on the current device."""
    t = _lib.Tuning()
    _lib.check(_lib_tune().flood_tuning_lookup(int(n_points), int(n_landmarks), int(m), C.byref(t)),
               "flood_tuning_lookup")
    return {"cell_factor": float(t.cell_factor), "heavy_shells": int(t.heavy_shells), "tuned": bool(t.tuned)}


def set_entry(key: tuple, cell_factor: float, heavy_shells: int) -> None:
    e = Entry(*key, float(cell_factor), int(heavy_shells))
    _lib.check(_lib_tune().flood_tuning_set(C.byref(e)), "flood_tuning_set")


def entries() -> list:
    lib = _lib_tune()
    n = C.c_int32(0)
    _lib.check(lib.flood_tuning_entries(None, 0, C.byref(n)), "flood_tuning_entries")
    arr = (Entry * max(1, n.value))()
    _lib.check(lib.flood_tuning_entries(arr, n.value, C.byref(n)), "flood_tuning_entries")
    return [(tuple(int(getattr(e, f)) for f in ("sm_count", "log2_points", "log2_landmarks", "m")),
             float(e.cell_factor), int(e.heavy_shells)) for e in arr[:n.value]]


def clear() -> None:
    _lib.check(_lib_tune().flood_tuning_clear(), "flood_tuning_clear")


def load(path: str | None = None) -> int:
    n = C.c_int32(0)
    _lib.check(_lib_tune().flood_tuning_load((path or cache_path()).encode(), C.byref(n)), "flood_tuning_load")
    return int(n.value)


def save(path: str | None = None) -> str:
    path = path or cache_path()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path + ".tmp", "w") as f:
        f.write("# sm_count log2_points log2_landmarks m cell_factor heavy_shells\n")
        for key, cf, hs in sorted(entries()):
            f.write(f"{key[0]} {key[1]} {key[2]} {key[3]} {cf:.6g} {hs}\n")
    os.replace(path + ".tmp", path)
    return path


def choose(timings: dict):
    """The tuned pair from {(cell factor, heavy threshold): ms}: the fastest, except that the
    defaults stay when they were measured and are within KEEP_DEFAULTS_WITHIN of it.
    Returns ((cell factor, heavy threshold), ms)."""
    best, ms = min(timings.items(), key=lambda kv: kv[1])
    d_ms = timings.get(DEFAULTS)
    if d_ms is not None and d_ms <= ms * (1.0 + KEEP_DEFAULTS_WITHIN):
        return DEFAULTS, d_ms
    return best, ms


def tune_workload(X, L, cx, m: int, cover: float, cell_factors=CELL_FACTORS, heavy_shells=HEAVY_SHELLS,
                  reps: int = 3) -> dict:
    """Measure grid build + filtration for every (cell factor, heavy threshold) pair on one workload.

    X, L: float32 CUDA tensors; cx: ops.DeviceComplex; cover: FPS covering radius
    (sqrt of the last FPS key). Each pair is timed `reps` times (best kept) with
    CUDA events on the current stream. The fastest pair is recorded in the
    table under the workload's bucket and returned with every timing; the
    defaults stay when they are measured and within KEEP_DEFAULTS_WITHIN of
    the fastest (near-ties are timing noise, and a stable choice keeps
    profiles taken at the defaults valid for the workload).
    """
    import torch
    from . import ops

    dev = X.device
    stream = torch.cuda.current_stream(dev)
    key = bucket(X.shape[0], L.shape[0], m, torch.cuda.get_device_properties(dev).multi_processor_count)
    timings = {}
    for cf in cell_factors:
        for hs in heavy_shells:
            set_entry(key, cf, hs)
            best = float("inf")
            for _ in range(reps + 1):                   # one untimed pass first
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                grid = ops.build_grid(X, cf * cover)
                ops.filtration(grid, L, cx, m, want_src=False)
                b.record(stream)
                b.synchronize()
                grid.close()
                best = min(best, a.elapsed_time(b))
            timings[(cf, hs)] = best
    (cf, hs), ms = choose(timings)
    d_ms = timings.get(DEFAULTS)
    set_entry(key, cf, hs)
    return {"bucket": key, "cell_factor": cf, "heavy_shells": hs, "ms": ms,
            "default_ms": d_ms, "timings_ms": {f"{a:g}/{b}": t for (a, b), t in timings.items()}}


def tune_cloud(X_host: np.ndarray, n_landmarks: int, m: int, **kw) -> dict:
    """tune_workload on a host cloud: FPS on the device, host Delaunay of the landmarks."""
    import torch
    from . import ops
    from .complex import delaunay_complex

    Xd = torch.from_numpy(np.ascontiguousarray(X_host, np.float32)).cuda()
    idx, key = ops.fps(Xd, n_landmarks, 0)
    L = Xd[idx]
    cx = ops.to_device(delaunay_complex(L.cpu().numpy()), Xd.device)
    return tune_workload(Xd, L, cx, m, float(np.sqrt(key[-1].item())), **kw)


def _main():
    import argparse
    from . import data

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--serving", action="store_true", help="tune the serving workload's size buckets")
    ap.add_argument("--out", default=None, help="table file (default: FLOOD_TUNE_CACHE or ~/.cache/...)")
    args = ap.parse_args()
    if os.path.exists(args.out or cache_path()):
        load(args.out)
    if args.serving:
        for n in (2_000, 5_000, 11_000, 23_000, 45_000, 91_000, 181_000):
            X = data.shape_mix_cloud(n, seed=900 + n % 97)
            r = tune_cloud(X, max(4, round(0.02 * n)), 8)
            print(f"{n:>8} points: cell factor {r['cell_factor']:g}, heavy shells {r['heavy_shells']}, "
                  f"{r['ms']:.3f} ms (defaults {r['default_ms']:.3f} ms)")
    print("wrote", save(args.out))


if __name__ == "__main__":
    _main()
