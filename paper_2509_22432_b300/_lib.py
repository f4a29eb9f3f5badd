"""ctypes loader for libflood.so: declares every C entry point of include/flood.h.

The library is loaded from this package directory only (never a system
copy). A missing library raises at first use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# FLOOD_LIBRARY=checked loads the bounds-checked build (libflood_checked.so).
CHECKED = os.environ.get("FLOOD_LIBRARY", "") == "checked"
LIB_PATH = os.path.join(HERE, "libflood_checked.so" if CHECKED else "libflood.so")

STATUS = {
    0: "FLOOD_OK", -1: "FLOOD_EINVAL", -2: "FLOOD_ENOMEM", -3: "FLOOD_ECUDA", -4: "FLOOD_ETIMEOUT",
    -5: "FLOOD_EDEGENERATE", -6: "FLOOD_ECAPACITY", -7: "FLOOD_EINTERNAL",
}


class FloodError(RuntimeError):
    def __init__(self, status: int, message: str, where: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {message}" if where else f"{self.name}: {message}")


class GridInfo(C.Structure):
    _fields_ = [
        ("n_points", C.c_int64), ("n_cells", C.c_int64), ("dims", C.c_int32 * 3), ("cell_size", C.c_float),
        ("origin", C.c_float * 3), ("bbox_lo", C.c_float * 3), ("bbox_hi", C.c_float * 3),
        ("device_bytes", C.c_int64),
    ]


class FiltrationStats(C.Structure):
    _fields_ = [
        ("simplices", C.c_int64 * 4), ("samples", C.c_int64 * 4), ("pairs", C.c_int64 * 4),
        ("work_items", C.c_int64 * 4), ("active_samples", C.c_int64 * 4), ("shells", C.c_int64 * 4),
        ("tiles", C.c_int64 * 4),
        ("flood_kernel_ms", C.c_float * 4),
    ]


class FpsStats(C.Structure):
    _fields_ = [("picks", C.c_int64), ("rounds", C.c_int64), ("blocks", C.c_int32), ("resident", C.c_int32)]


class TuningEntry(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("log2_points", C.c_int32), ("log2_landmarks", C.c_int32),
                ("m", C.c_int32), ("cell_factor", C.c_float), ("heavy_shells", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("cell_factor", C.c_float), ("heavy_shells", C.c_int32), ("tuned", C.c_int32)]


P4 = C.c_void_p * 4
I64x4 = C.c_int64 * 4
I32x4 = C.c_int32 * 4
ND_MAX_DIM = 5
P6 = C.c_void_p * (ND_MAX_DIM + 1)
I64x6 = C.c_int64 * (ND_MAX_DIM + 1)


class GridNdInfo(C.Structure):
    _fields_ = [
        ("n_points", C.c_int64), ("n_cells", C.c_int64), ("dim", C.c_int32), ("dims", C.c_int32 * ND_MAX_DIM),
        ("cell_size", C.c_float), ("bbox_lo", C.c_float * ND_MAX_DIM), ("bbox_hi", C.c_float * ND_MAX_DIM),
        ("device_bytes", C.c_int64),
    ]


class NdStats(C.Structure):
    _fields_ = [("dim", C.c_int32)] + [
        (name, C.c_int64 * (ND_MAX_DIM + 1))
        for name in ("items", "pruned", "resolved", "exact", "fallback", "pairs", "pairs_fallback", "cells")]


class FiltrationJob(C.Structure):
    _fields_ = [
        ("grid", C.c_void_p), ("L", C.c_void_p), ("n_landmarks", C.c_int32), ("m", C.c_int32),
        ("simplices", C.c_void_p * 4), ("facets", C.c_void_p * 4), ("n_simplices", C.c_int64 * 4),
        ("values", C.c_void_p * 4), ("src", C.c_void_p * 4),
    ]

class HostComplex(C.Structure):
    _fields_ = [("n_simplices", C.c_int64 * 4), ("simplices", C.c_void_p * 4), ("facets", C.c_void_p * 4),
                ("owner", C.c_void_p)]


TRIANGULATE = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_float), C.c_int32, C.POINTER(HostComplex))
RELEASE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ServeConfig(C.Structure):
    _fields_ = [("device_budget_bytes", C.c_int64), ("max_inflight", C.c_int32), ("max_batch", C.c_int32),
                ("gpu_workers", C.c_int32), ("triangulation_workers", C.c_int32),
                ("landmark_fraction", C.c_float), ("cell_factor", C.c_float),
                ("triangulate", TRIANGULATE), ("release", RELEASE), ("user", C.c_void_p)]


class ServeResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_landmarks", C.c_int32), ("n_simplices", C.c_int64 * 4),
                ("values", C.POINTER(C.c_float) * 4), ("landmarks", C.POINTER(C.c_int64)),
                ("latency_ms", C.c_double), ("simplices", C.POINTER(C.c_int32) * 4)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("inflight", C.c_int64),
                ("batches", C.c_int64), ("mean_batch", C.c_double), ("clouds_per_s", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("device_bytes_in_use", C.c_int64), ("device_bytes_peak", C.c_int64)]


_SERVE_SIGNATURES = {
    "flood_serve_create": (C.c_int, [C.POINTER(ServeConfig), C.POINTER(C.c_void_p)]),
    "flood_serve_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                     C.POINTER(C.c_uint64)]),
    "flood_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(ServeResult)]),
    "flood_serve_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "flood_serve_stats": (C.c_int, [C.c_void_p, C.POINTER(ServeStats)]),
    "flood_serve_destroy": (None, [C.c_void_p]),
}


_SIGNATURES = {
    "flood_fps": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "flood_fps_blocks": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "flood_fps_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "flood_last_fps_stats": (C.c_int, [C.POINTER(FpsStats)]),
    "flood_fps_scratch_bytes": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(C.c_int64)]),
    "flood_fps_wait_test": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_uint32,
                                      C.c_void_p, C.c_void_p]),
    "flood_masking_ball_counts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P4, I64x4, C.POINTER(C.c_int64),
                                            C.c_void_p]),
    "flood_fp32_peak_probe": (C.c_int, [C.c_int32, C.c_int64, C.POINTER(C.c_double), C.c_void_p]),
    "flood_build_grid": (C.c_int, [C.c_void_p, C.c_int64, C.c_float, C.POINTER(C.c_void_p), C.c_void_p]),
    "flood_grid_get_info": (C.c_int, [C.c_void_p, C.POINTER(GridInfo)]),
    "flood_grid_destroy": (None, [C.c_void_p]),
    "flood_filtration": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P4, P4, I64x4, C.c_int32, P4, P4,
                                   C.c_void_p]),
    "flood_filtration_given": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P4, P4, I64x4, P4, I32x4, P4, P4,
                                         C.c_void_p]),
    "flood_filtration_given_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P4, I64x4, P4, I32x4, P4,
                                                  P4, C.c_void_p, C.c_void_p, C.c_void_p]),
    "flood_filtration_masked": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P4, I64x4, C.c_int32, P4,
                                          C.POINTER(C.c_int64), C.c_void_p]),
    "flood_complex_faces": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.c_void_p]),
    "flood_last_filtration_stats": (C.c_int, [C.POINTER(FiltrationStats)]),
    "flood_filtration_batch": (C.c_int, [C.POINTER(FiltrationJob), C.c_int32, C.c_void_p]),
    "flood_filtration_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P4, I64x4, C.c_int32, P4, P4,
                                            C.c_void_p, C.c_void_p, C.c_void_p]),
    "flood_tuning_lookup": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.POINTER(Tuning)]),
    "flood_tuning_set": (C.c_int, [C.POINTER(TuningEntry)]),
    "flood_tuning_load": (C.c_int, [C.c_char_p, C.POINTER(C.c_int32)]),
    "flood_tuning_entries": (C.c_int, [C.POINTER(TuningEntry), C.c_int32, C.POINTER(C.c_int32)]),
    "flood_tuning_clear": (C.c_int, []),
    "flood_check": (C.c_int, [C.c_void_p]),
    "flood_persistence": (C.c_int, [P4, P4, I64x4, P4, C.c_void_p * 3, C.c_int64 * 3, P4, I64x4,
                                    C.POINTER(C.c_int64), C.c_void_p]),
    "flood_gather_rows": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "flood_fps_nd": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "flood_build_grid_nd": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.POINTER(C.c_void_p),
                                      C.c_void_p]),
    "flood_grid_nd_get_info": (C.c_int, [C.c_void_p, C.POINTER(GridNdInfo)]),
    "flood_grid_nd_destroy": (None, [C.c_void_p]),
    "flood_filtration_nd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, P6, P6, I64x6, C.c_int32, P6,
                                      C.c_void_p]),
    "flood_last_filtration_nd_stats": (C.c_int, [C.POINTER(NdStats)]),
    "flood_last_error": (C.c_char_p, []),
    "flood_version": (C.c_char_p, []),
    "flood_kernel_launches": (C.c_int64, []),
}
_SIGNATURES.update(_SERVE_SIGNATURES)

_lock = threading.Lock()
_lib = None


def exported_symbols() -> list:
    return list(_SIGNATURES)


def get() -> C.CDLL:
    """Load libflood.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            if _build.needs_build(CHECKED):
                _build.build(checked=CHECKED)
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libflood.so not found at {LIB_PATH}; run paper_2509_22432_b300/build.py")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        msg = get().flood_last_error().decode(errors="replace")
        raise FloodError(status, msg, where)
