"""Serving loop: continuous batching of many point clouds (flood_serve_* in libflood).

The library admits clouds by in-flight slots and a device-memory budget, runs
FPS and the grid build per cloud on its own streams, asks this module to
triangulate the landmarks (scipy/Qhull on the host, as the paper does with
CGAL/qhull), and runs every cloud that is ready through one batched flood
filtration. All device work happens in libflood; Python only supplies the
triangulation callback and marshals results.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
# imported here, not inside the callback: a first import from the library's
# triangulation threads would hold up the first requests behind the import lock
from scipy.spatial import Delaunay

from . import _lib
from ._lib import RELEASE, ServeConfig, ServeResult, ServeStats, TRIANGULATE
from .complex import delaunay_complex

__all__ = ["Server", "delaunay_tets"]


def delaunay_tets(L: np.ndarray) -> np.ndarray:
    """Tetrahedra of Del(L) (scipy/Qhull), ascending vertex ids, int32."""
    return np.ascontiguousarray(np.sort(Delaunay(np.asarray(L, np.float64)).simplices, axis=1), dtype=np.int32)


def _lib_serve():
    return _lib.get()


class Server:
    """Continuous-batching flood server on the current CUDA device.

    triangulate(L) -> SimplexLists (default: scipy Delaunay of the landmarks).
    max_batch = 1 gives the plain one-cloud-at-a-time path.
    triangulation_workers: host threads running the triangulation callback
    (default: one per host core).
    device_faces (default when no triangulate is given): the callback hands
    over the tetrahedra of the scipy Delaunay triangulation only, and the
    library builds the triangles, edges and facet incidence on the device;
    results list the rows of every dimension ("simplices"), whose order is then
    the device's, not lexicographic. device_faces=False builds the whole
    complex on the host (rows in lexicographic order).
    tets_cache (device_faces only): tetrahedra by the landmarks' float32 bytes,
    used instead of running Qhull when present (to time the server without
    the host Delaunay); `cache_misses` counts the landmark sets it lacked.
    """

    def __init__(self, device_budget_bytes: int = 16 << 30, max_inflight: int = 64, max_batch: int = 32,
                 gpu_workers: int = 4, triangulation_workers: int | None = None, landmark_fraction: float = 0.02,
                 cell_factor: float = 0.5, triangulate=None, device_faces: bool | None = None,
                 tets_cache: dict | None = None):
        self._lib = _lib_serve()
        if triangulation_workers is None:
            triangulation_workers = os.cpu_count() or 4
        if device_faces is None:
            device_faces = triangulate is None
        if device_faces and triangulate is not None:
            raise ValueError("device_faces uses the built-in tetrahedralisation; pass no triangulate")
        self._fn = triangulate or delaunay_complex
        self._device_faces = bool(device_faces)
        self._tets_cache = tets_cache
        self.cache_misses = 0
        self._keep = {}
        self._next = 1
        self._lock = threading.Lock()
        self._tri_cb = TRIANGULATE(self._triangulate)
        self._rel_cb = RELEASE(self._release)
        cfg = ServeConfig(int(device_budget_bytes), int(max_inflight), int(max_batch), int(gpu_workers),
                          int(triangulation_workers), float(landmark_fraction), float(cell_factor),
                          self._tri_cb, self._rel_cb, None)
        h = C.c_void_p(0)
        _lib.check(self._lib.flood_serve_create(C.byref(cfg), C.byref(h)), "flood_serve_create")
        self._h = h

    # called from library threads (ctypes takes the GIL)
    def _triangulate(self, user, L_ptr, n, out):
        try:
            L = np.ctypeslib.as_array(L_ptr, shape=(int(n) * 3,)).reshape(int(n), 3).copy()
            arrays = []
            o = out.contents
            if self._device_faces:
                tets = self._tets_cache.get(L.tobytes()) if self._tets_cache is not None else None
                if tets is None:
                    if self._tets_cache is not None:
                        with self._lock:
                            self.cache_misses += 1
                    tets = delaunay_tets(L)
                arrays.append(tets)
                for k in range(3):
                    o.n_simplices[k] = 0
                o.n_simplices[3] = tets.shape[0]
                o.simplices[3] = tets.ctypes.data if tets.size else None
                with self._lock:
                    key = self._next
                    self._next += 1
                    self._keep[key] = arrays
                o.owner = key
                return 0
            cx = self._fn(L)
            for k in range(4):
                if k < len(cx.simplices):
                    s = np.ascontiguousarray(cx.simplices[k], dtype=np.int32)
                    f = np.ascontiguousarray(cx.facets[k], dtype=np.int32)
                    arrays += [s, f]
                    o.n_simplices[k] = s.shape[0]
                    o.simplices[k] = s.ctypes.data if s.size else None
                    o.facets[k] = f.ctypes.data if f.size else None
                else:
                    o.n_simplices[k] = 0
            with self._lock:
                key = self._next
                self._next += 1
                self._keep[key] = arrays
            o.owner = key
            return 0
        except Exception:
            return 1

    def _release(self, user, owner):
        with self._lock:
            self._keep.pop(owner, None)

    def submit(self, X: np.ndarray, n_landmarks: int = 0, m: int = 8) -> int:
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != 3:
            raise ValueError("X must be (n, 3)")
        t = C.c_uint64(0)
        _lib.check(self._lib.flood_serve_submit(self._h, X.ctypes.data, X.shape[0], int(n_landmarks), int(m),
                                                C.byref(t)), "flood_serve_submit")
        return int(t.value)

    def result(self, ticket: int, timeout_ms: int = -1) -> dict:
        """Wait for a result; returns values per dimension, landmark rows, latency, status."""
        r = ServeResult()
        _lib.check(self._lib.flood_serve_poll(self._h, int(ticket), int(timeout_ms), C.byref(r)), "flood_serve_poll")
        out = {"status": int(r.status), "latency_ms": float(r.latency_ms), "values": [], "landmarks": None,
               "simplices": [None]}
        if r.status == 0:
            out["landmarks"] = np.ctypeslib.as_array(r.landmarks, shape=(r.n_landmarks,)).copy()
            for k in range(4):
                n = int(r.n_simplices[k])
                out["values"].append(np.ctypeslib.as_array(r.values[k], shape=(n,)).copy() if n else
                                     np.zeros(0, np.float32))
                if k >= 1:
                    out["simplices"].append(
                        np.ctypeslib.as_array(r.simplices[k], shape=(n, k + 1)).copy() if n and r.simplices[k]
                        else np.zeros((0, k + 1), np.int32))
        return out

    def release(self, ticket: int) -> None:
        _lib.check(self._lib.flood_serve_release(self._h, int(ticket)), "flood_serve_release")

    def stats(self) -> dict:
        st = ServeStats()
        _lib.check(self._lib.flood_serve_stats(self._h, C.byref(st)), "flood_serve_stats")
        return {name: getattr(st, name) for name, _ in ServeStats._fields_}

    def close(self) -> None:
        if self._h:
            self._lib.flood_serve_destroy(self._h)
            self._h = C.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
