"""Torch-facing wrappers of libflood (argument marshalling only).

Every step runs in the CUDA kernels of libflood.so; these functions only
check shapes and dtypes, pass device pointers and the current CUDA stream,
and raise FloodError on a non-OK status. Inputs must already live on a CUDA
device; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import FloodError, P4, I64x4, I32x4

__all__ = ["check", "fps", "fps_noalloc", "fps_stats", "fps_scratch_bytes", "fps_wait_test", "masking_ball_counts",
           "fp32_peak_probe", "Grid", "build_grid", "DeviceComplex", "to_device", "filtration",
           "filtration_batch", "filtration_backward", "filtration_given", "filtration_given_backward",
           "complex_faces", "filtration_masked", "persistence", "diagrams_from_pairs",
           "last_filtration_stats", "FloodFunction", "flood_values", "GivenFloodFunction", "flood_values_given",
           "fps_nd", "GridNd", "build_grid_nd", "filtration_nd", "last_filtration_nd_stats", "gather_rows"]


def _stream_ptr(device: torch.device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor | None) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


def _points(X: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if X.dtype != torch.float32 or X.dim() != 2 or X.shape[1] != 3:
        raise ValueError(f"{name} must be float32 of shape (n, 3)")
    return X.contiguous()


def check(device: torch.device | None = None) -> None:
    """Wait for the current stream and raise FloodError if an asynchronous call on it failed (flood_check)."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(device):
        st = _lib.get().flood_check(_stream_ptr(device))
    _lib.check(st, "flood_check")


def _finish(st: int, where: str, device: torch.device, sync: bool) -> None:
    _lib.check(st, where)
    if sync:
        check(device)


def fps(X: torch.Tensor, n_landmarks: int, start: int = 0, n_blocks: int = 0, sync: bool = True):
    """Farthest point sampling (§3.2). Returns (idx int64[n], key float32[n]).

    n_blocks: launch width (0 automatic, 1 one SM, k blocks); the picks are
    the same for every width. sync=False leaves the call asynchronous: its
    device-side status is then reported by check() or by the next call.
    """
    X = _points(X, "X")
    idx = torch.empty(n_landmarks, dtype=torch.int64, device=X.device)
    key = torch.empty(n_landmarks, dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_fps_blocks(_ptr(X), X.shape[0], int(n_landmarks), int(start), int(n_blocks), _ptr(idx),
                                         _ptr(key), _stream_ptr(X.device))
    _finish(st, "flood_fps", X.device, sync)
    return idx, key


def fps_noalloc(X: torch.Tensor, n_landmarks: int, start: int = 0):
    """fps() for callers that must not allocate device memory inside the library.

    Same picks as fps(); the library takes its scratch from a fixed array
    compiled into it, so X may hold at most 2^20 points, and calls that
    overlap on the GPU must be serialised by the caller. (The output tensors
    here are allocated by torch before the call; a caller without an
    allocator passes its own buffers to the C entry point directly.)
    """
    X = _points(X, "X")
    idx = torch.empty(n_landmarks, dtype=torch.int64, device=X.device)
    key = torch.empty(n_landmarks, dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_fps_noalloc(_ptr(X), X.shape[0], int(n_landmarks), int(start), _ptr(idx),
                                          _ptr(key), _stream_ptr(X.device))
    _lib.check(st, "flood_fps_noalloc")
    return idx, key


def fps_stats() -> dict:
    """Counters of this thread's last successful FPS call: picks, exchange rounds, blocks, resident."""
    st = _lib.FpsStats()
    _lib.check(_lib.get().flood_last_fps_stats(C.byref(st)), "flood_last_fps_stats")
    return {"picks": int(st.picks), "rounds": int(st.rounds), "blocks": int(st.blocks),
            "resident": bool(st.resident)}


def fps_scratch_bytes(n_points: int, n_blocks: int = 0) -> int:
    """Device scratch bytes flood_fps_blocks takes for n_points at launch width n_blocks (host arithmetic)."""
    out = C.c_int64(0)
    _lib.check(_lib.get().flood_fps_scratch_bytes(int(n_points), int(n_blocks), C.byref(out)),
               "flood_fps_scratch_bytes")
    return int(out.value)


def fps_wait_test(X: torch.Tensor, n_landmarks: int, n_blocks: int, extra_blocks: int, poll_limit: int) -> int:
    """Run FPS with an exchange that waits for never-launched blocks; returns the raw status (test support)."""
    X = _points(X, "X")
    idx = torch.full((n_landmarks,), -1, dtype=torch.int64, device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_fps_wait_test(_ptr(X), X.shape[0], int(n_landmarks), int(n_blocks), int(extra_blocks),
                                            int(poll_limit), _ptr(idx), _stream_ptr(X.device))
    return int(st)


def fp32_peak_probe(device: torch.device, packed: bool, iterations: int) -> float:
    """Enqueue the FP32 FMA throughput kernel on the current stream; returns its flop count."""
    flops = C.c_double(0.0)
    with torch.cuda.device(device):
        st = _lib.get().flood_fp32_peak_probe(int(bool(packed)), int(iterations), C.byref(flops),
                                              _stream_ptr(device))
    _lib.check(st, "flood_fp32_peak_probe")
    return float(flops.value)


class Grid:
    """Library-owned uniform cell grid over X (flood_build_grid)."""

    def __init__(self, handle: C.c_void_p, device: torch.device):
        self._h = handle
        self.device = device

    @property
    def handle(self) -> C.c_void_p:
        if not self._h:
            raise ValueError("grid already destroyed")
        return self._h

    def info(self) -> dict:
        inf = _lib.GridInfo()
        _lib.check(_lib.get().flood_grid_get_info(self.handle, C.byref(inf)), "flood_grid_get_info")
        return {"n_points": inf.n_points, "n_cells": inf.n_cells, "dims": tuple(inf.dims),
                "cell_size": inf.cell_size, "origin": tuple(inf.origin), "bbox_lo": tuple(inf.bbox_lo),
                "bbox_hi": tuple(inf.bbox_hi), "device_bytes": inf.device_bytes}

    def close(self) -> None:
        if self._h:
            _lib.get().flood_grid_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_grid(X: torch.Tensor, cell_size: float = 0.0, sync: bool = True) -> Grid:
    """Uniform cell grid over X (flood_build_grid); sync=False: asynchronous, see fps()."""
    X = _points(X, "X")
    h = C.c_void_p(0)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_build_grid(_ptr(X), X.shape[0], float(cell_size), C.byref(h), _stream_ptr(X.device))
    _lib.check(st, "flood_build_grid")
    grid = Grid(h, X.device)
    if sync:
        check(X.device)
    return grid


@dataclass
class DeviceComplex:
    """Simplex lists of Del(L) on the device (int32, layout of complex.SimplexLists)."""
    n_vertices: int
    simplices: list   # k -> (n_k, k+1) int32 CUDA tensor
    facets: list      # k -> (n_k, k+1) int32 CUDA tensor

    @property
    def counts(self) -> list:
        return [int(s.shape[0]) for s in self.simplices]

    def arrays(self):
        s = P4(*[C.c_void_p(t.data_ptr() if t.numel() else 0) for t in self.simplices[:4]] +
               [C.c_void_p(0)] * (4 - len(self.simplices)))
        f = P4(*[C.c_void_p(t.data_ptr() if t.numel() else 0) for t in self.facets[:4]] +
               [C.c_void_p(0)] * (4 - len(self.facets)))
        n = I64x4(*(self.counts + [0] * (4 - len(self.simplices))))
        return s, f, n


def to_device(cx, device) -> DeviceComplex:
    sims = [torch.from_numpy(np.ascontiguousarray(s, dtype=np.int32)).to(device) for s in cx.simplices]
    facs = [torch.from_numpy(np.ascontiguousarray(f, dtype=np.int32)).to(device) for f in cx.facets]
    return DeviceComplex(int(cx.n_vertices), sims, facs)


def filtration_masked(grid: Grid, L: torch.Tensor, cx: DeviceComplex, m: int):
    """The paper's masked full-grid evaluation (§4.2, App. A.1), for comparison.

    Returns (values[k] float32, pairs evaluated). Values equal filtration()'s
    up to FP32 rounding.
    """
    L = _points(L, "L")
    s, _, n = cx.arrays()
    vals = [torch.empty(c, dtype=torch.float32, device=L.device) for c in cx.counts]
    vp = P4(*[_ptr(v) if v.numel() else C.c_void_p(0) for v in vals] + [C.c_void_p(0)] * (4 - len(vals)))
    pairs = C.c_int64(0)
    with torch.cuda.device(L.device):
        st = _lib.get().flood_filtration_masked(grid.handle, _ptr(L), L.shape[0], s, n, int(m), vp, C.byref(pairs),
                                                _stream_ptr(L.device))
    _lib.check(st, "flood_filtration_masked")
    return vals, int(pairs.value)


def masking_ball_counts(grid: Grid, L: torch.Tensor, cx: DeviceComplex) -> list:
    """Per dimension, the number of (simplex, point) incidences with the point in the simplex's
    Lemma 2 masking ball (§4.2): sum over k-simplices of |X ∩ B(c, sqrt(2) r)|."""
    L = _points(L, "L")
    s, _, n = cx.arrays()
    out = I64x4(0, 0, 0, 0)
    with torch.cuda.device(L.device):
        st = _lib.get().flood_masking_ball_counts(grid.handle, _ptr(L), L.shape[0], s, n, out,
                                                  _stream_ptr(L.device))
    _lib.check(st, "flood_masking_ball_counts")
    return [int(v) for v in out]


def complex_faces(tets: torch.Tensor, n_vertices: int) -> DeviceComplex:
    """Faces and facet incidence of the tetrahedra on the device (flood_complex_faces).

    tets: int32 CUDA (n, 4) with ascending vertex ids. Rows of the lower
    dimensions follow their first producing (parent, j), not lexicographic order.
    """
    if not isinstance(tets, torch.Tensor) or not tets.is_cuda or tets.dtype != torch.int32 or tets.dim() != 2 \
            or tets.shape[1] != 4:
        raise ValueError("tets must be an int32 CUDA tensor of shape (n, 4)")
    tets = tets.contiguous()
    dev, n3 = tets.device, tets.shape[0]
    tri = torch.empty((4 * n3, 3), dtype=torch.int32, device=dev)
    edg = torch.empty((6 * n3, 2), dtype=torch.int32, device=dev)
    f3 = torch.empty((n3, 4), dtype=torch.int32, device=dev)
    f2 = torch.empty((4 * n3, 3), dtype=torch.int32, device=dev)
    f1 = torch.empty((6 * n3, 2), dtype=torch.int32, device=dev)
    n2, n1 = C.c_int64(0), C.c_int64(0)
    with torch.cuda.device(dev):
        st = _lib.get().flood_complex_faces(_ptr(tets), n3, int(n_vertices), _ptr(tri), _ptr(edg), _ptr(f3),
                                            _ptr(f2), _ptr(f1), C.byref(n2), C.byref(n1), _stream_ptr(dev))
    _lib.check(st, "flood_complex_faces")
    verts = torch.arange(int(n_vertices), dtype=torch.int32, device=dev)[:, None]
    return DeviceComplex(int(n_vertices), [verts, edg[:n1.value], tri[:n2.value], tets],
                         [torch.zeros_like(verts), f1[:n1.value], f2[:n2.value], f3])


def filtration(grid: Grid, L: torch.Tensor, cx: DeviceComplex, m: int, want_src: bool = True, sync: bool = True):
    """Flood values of every simplex (§4.1). Returns (values[k] float32, src[k] int32 (n_k,2) or None).

    sync=False: asynchronous, see fps()."""
    L = _points(L, "L")
    s, f, n = cx.arrays()
    vals = [torch.empty(c, dtype=torch.float32, device=L.device) for c in cx.counts]
    srcs = [torch.empty((c, 2), dtype=torch.int32, device=L.device) for c in cx.counts] if want_src else None
    vp = P4(*[_ptr(v) if v.numel() else C.c_void_p(0) for v in vals] + [C.c_void_p(0)] * (4 - len(vals)))
    sp = P4(*([_ptr(t) if t.numel() else C.c_void_p(0) for t in srcs] + [C.c_void_p(0)] * (4 - len(srcs)))
            if want_src else [C.c_void_p(0)] * 4)
    with torch.cuda.device(L.device):
        st = _lib.get().flood_filtration(grid.handle, _ptr(L), L.shape[0], s, f, n, int(m), vp, sp,
                                         _stream_ptr(L.device))
    _finish(st, "flood_filtration", L.device, sync)
    return vals, srcs


def filtration_batch(jobs, want_src: bool = False, sync: bool = True):
    """Flood values of several clouds in one batched call.

    jobs: list of (grid, L, DeviceComplex, m). Returns a list of (values, src).
    Each cloud's results equal those of filtration() on it alone, bit for bit.
    """
    if not jobs:
        return []
    dev = jobs[0][1].device
    arr = (_lib.FiltrationJob * len(jobs))()
    outs, keep = [], []
    for i, (grid, L, cx, m) in enumerate(jobs):
        L = _points(L, "L")
        keep.append(L)
        s, f, n = cx.arrays()
        vals = [torch.empty(c, dtype=torch.float32, device=dev) for c in cx.counts]
        srcs = [torch.empty((c, 2), dtype=torch.int32, device=dev) for c in cx.counts] if want_src else None
        j = arr[i]
        j.grid = grid.handle
        j.L = L.data_ptr()
        j.n_landmarks = L.shape[0]
        j.m = int(m)
        for k in range(4):
            j.simplices[k] = s[k]
            j.facets[k] = f[k]
            j.n_simplices[k] = n[k]
            j.values[k] = vals[k].data_ptr() if k < len(vals) and vals[k].numel() else 0
            j.src[k] = srcs[k].data_ptr() if want_src and k < len(srcs) and srcs[k].numel() else 0
        outs.append((vals, srcs))
    with torch.cuda.device(dev):
        st = _lib.get().flood_filtration_batch(arr, len(jobs), _stream_ptr(dev))
    _finish(st, "flood_filtration_batch", dev, sync)
    return outs


def last_filtration_stats() -> dict:
    st = _lib.FiltrationStats()
    _lib.check(_lib.get().flood_last_filtration_stats(C.byref(st)), "flood_last_filtration_stats")
    return {k: list(getattr(st, k)) for k in ("simplices", "samples", "pairs", "work_items", "active_samples",
                                               "shells", "tiles", "flood_kernel_ms")}


def persistence(cx: DeviceComplex, values) -> dict:
    """Persistence pairs of the flood filtration on the device (flood_persistence, §2).

    values: float32 CUDA tensors per dimension (the flood values of cx).
    Returns {"pairs": [k -> int32 (n, 2) CUDA tensor of (birth row of dim k,
    death row of dim k+1)] for k = 0..2, "essential": [k -> int32 rows] for
    k = 0..3, "rounds": [parallel reduction rounds per dimension]}.
    """
    dev = values[0].device
    counts = cx.counts + [0] * (4 - len(cx.counts))
    s, f, n = cx.arrays()
    vals = [v.to(torch.float32).contiguous() for v in values] + [None] * (4 - len(values))
    vp = P4(*[_ptr(v) if v is not None and v.numel() else C.c_void_p(0) for v in vals])
    pairs = [torch.empty((max(counts[k + 1], 1), 2), dtype=torch.int32, device=dev) for k in range(3)]
    ess = [torch.empty(max(counts[k], 1), dtype=torch.int32, device=dev) for k in range(4)]
    pp = (C.c_void_p * 3)(*[_ptr(t) for t in pairs])
    ep = P4(*[_ptr(t) for t in ess])
    n_pairs, n_ess, rounds = (C.c_int64 * 3)(), I64x4(), I64x4()
    with torch.cuda.device(dev):
        st = _lib.get().flood_persistence(s, f, n, vp, pp, n_pairs, ep, n_ess, rounds, _stream_ptr(dev))
    _lib.check(st, "flood_persistence")
    return {"pairs": [pairs[k][:n_pairs[k]] for k in range(3)], "essential": [ess[k][:n_ess[k]] for k in range(4)],
            "rounds": [int(r) for r in rounds]}


def diagrams_from_pairs(ph: dict, values, max_dim: int = 2) -> list:
    """dgm_0..dgm_max_dim (host float64 (n, 2), death inf for essential classes) from persistence()."""
    v = [np.asarray(x.cpu().numpy() if isinstance(x, torch.Tensor) else x, dtype=np.float64) for x in values]
    out = []
    for k in range(max_dim + 1):
        pr = ph["pairs"][k].cpu().numpy()
        b, d = v[k][pr[:, 0]], v[k + 1][pr[:, 1]]
        keep = d > b
        e = v[k][ph["essential"][k].cpu().numpy()]
        pts = np.concatenate([np.stack([b[keep], d[keep]], 1), np.stack([e, np.full(e.shape, np.inf)], 1)])
        out.append(pts[np.lexsort((pts[:, 1], pts[:, 0]))].reshape(-1, 2))
    return out


def kernel_launches() -> int:
    """Kernels libflood has launched in this process so far."""
    return int(_lib.get().flood_kernel_launches())


def filtration_backward(grid: Grid, L: torch.Tensor, cx: DeviceComplex, m: int, src, grads, n_points: int):
    """(grad_X (N,3), grad_L (n_L,3)) of sum_sigma grads[k][sigma] * f(sigma)."""
    L = _points(L, "L")
    s, _, n = cx.arrays()
    gX = torch.zeros((n_points, 3), dtype=torch.float32, device=L.device)
    gL = torch.zeros_like(L)
    srcp = P4(*[_ptr(t) if t is not None and t.numel() else C.c_void_p(0) for t in src] +
              [C.c_void_p(0)] * (4 - len(src)))
    gs = [None if g is None else g.to(torch.float32).contiguous() for g in grads]
    gp = P4(*[_ptr(g) if g is not None and g.numel() else C.c_void_p(0) for g in gs] +
            [C.c_void_p(0)] * (4 - len(gs)))
    with torch.cuda.device(L.device):
        st = _lib.get().flood_filtration_backward(grid.handle, _ptr(L), L.shape[0], s, n, int(m), srcp, gp,
                                                  _ptr(gX), _ptr(gL), _stream_ptr(L.device))
    _lib.check(st, "flood_filtration_backward")
    return gX, gL


class FloodFunction(torch.autograd.Function):
    """Differentiable flood values: forward(X, L, grid, cx, m) -> values of dims 0..3 (concatenated).

    X and L are independent inputs; the grid must have been built from X.
    """

    @staticmethod
    def forward(ctx, X, L, grid, cx, m):
        vals, srcs = filtration(grid, L, cx, m, want_src=True)
        ctx.grid, ctx.cx, ctx.m, ctx.srcs, ctx.n_points = grid, cx, m, srcs, X.shape[0]
        ctx.counts = cx.counts
        ctx.save_for_backward(L)
        return torch.cat(vals)

    @staticmethod
    def backward(ctx, g):
        (L,) = ctx.saved_tensors
        parts = list(torch.split(g.contiguous(), ctx.counts))
        gX, gL = filtration_backward(ctx.grid, L, ctx.cx, ctx.m, ctx.srcs, parts, ctx.n_points)
        return gX, gL, None, None, None


def flood_values(X: torch.Tensor, L: torch.Tensor, grid: Grid, cx: DeviceComplex, m: int):
    """Differentiable flood values split per dimension."""
    out = FloodFunction.apply(X, L, grid, cx, m)
    return list(torch.split(out, cx.counts))


def _weights(weights, cx: DeviceComplex, device):
    """Check given sets: weights[k] float32 CUDA (n_k, S_k, k+1) for k >= 1 (weights[0] unused)."""
    ws, ptrs, counts = [None], [C.c_void_p(0)], [0]
    for k in range(1, 4):
        n_k = cx.counts[k] if k < len(cx.counts) else 0
        w = weights[k] if k < len(weights) else None
        if w is None:
            if n_k:
                raise ValueError(f"weights[{k}] is required for {n_k} simplices")
            ws.append(None)
            ptrs.append(C.c_void_p(0))
            counts.append(0)
            continue
        if not isinstance(w, torch.Tensor) or not w.is_cuda or w.device != device or w.dtype != torch.float32:
            raise ValueError(f"weights[{k}] must be a float32 CUDA tensor on {device}")
        if w.dim() != 3 or w.shape[0] != n_k or w.shape[2] != k + 1:
            raise ValueError(f"weights[{k}] must have shape ({n_k}, S, {k + 1})")
        w = w.contiguous()
        ws.append(w)
        ptrs.append(_ptr(w) if w.numel() else C.c_void_p(0))
        counts.append(int(w.shape[1]))
    return ws, P4(*ptrs), I32x4(*counts)


def filtration_given(grid: Grid, L: torch.Tensor, cx: DeviceComplex, weights, want_src: bool = True,
                     sync: bool = True):
    """Flood values for given point sets P_sigma (§4.1; random draws, Lemma 4).

    weights[k]: float32 CUDA (n_k, S_k, k+1) barycentric coordinates of each
    simplex's own points (lambda_0 implied). Returns (values[k], src[k] or None).
    """
    L = _points(L, "L")
    ws, wp, ns = _weights(weights, cx, L.device)
    s, f, n = cx.arrays()
    vals = [torch.empty(c, dtype=torch.float32, device=L.device) for c in cx.counts]
    srcs = [torch.empty((c, 2), dtype=torch.int32, device=L.device) for c in cx.counts] if want_src else None
    vp = P4(*[_ptr(v) if v.numel() else C.c_void_p(0) for v in vals] + [C.c_void_p(0)] * (4 - len(vals)))
    sp = P4(*([_ptr(t) if t.numel() else C.c_void_p(0) for t in srcs] + [C.c_void_p(0)] * (4 - len(srcs)))
            if want_src else [C.c_void_p(0)] * 4)
    with torch.cuda.device(L.device):
        st = _lib.get().flood_filtration_given(grid.handle, _ptr(L), L.shape[0], s, f, n, wp, ns, vp, sp,
                                               _stream_ptr(L.device))
    _finish(st, "flood_filtration_given", L.device, sync)
    return vals, srcs


def filtration_given_backward(grid: Grid, L: torch.Tensor, cx: DeviceComplex, weights, src, grads,
                              n_points: int):
    """(grad_X, grad_L) of sum_sigma grads[k][sigma] * f(sigma) for filtration_given's values."""
    L = _points(L, "L")
    ws, wp, ns = _weights(weights, cx, L.device)
    s, _, n = cx.arrays()
    gX = torch.zeros((n_points, 3), dtype=torch.float32, device=L.device)
    gL = torch.zeros_like(L)
    srcp = P4(*[_ptr(t) if t is not None and t.numel() else C.c_void_p(0) for t in src] +
              [C.c_void_p(0)] * (4 - len(src)))
    gs = [None if g is None else g.to(torch.float32).contiguous() for g in grads]
    gp = P4(*[_ptr(g) if g is not None and g.numel() else C.c_void_p(0) for g in gs] +
            [C.c_void_p(0)] * (4 - len(gs)))
    with torch.cuda.device(L.device):
        st = _lib.get().flood_filtration_given_backward(grid.handle, _ptr(L), L.shape[0], s, n, wp, ns, srcp, gp,
                                                        _ptr(gX), _ptr(gL), _stream_ptr(L.device))
    _lib.check(st, "flood_filtration_given_backward")
    return gX, gL


class GivenFloodFunction(torch.autograd.Function):
    """Differentiable flood values over given point sets: forward(X, L, grid, cx, weights)."""

    @staticmethod
    def forward(ctx, X, L, grid, cx, weights):
        vals, srcs = filtration_given(grid, L, cx, weights, want_src=True)
        ctx.grid, ctx.cx, ctx.weights, ctx.srcs, ctx.n_points = grid, cx, weights, srcs, X.shape[0]
        ctx.counts = cx.counts
        ctx.save_for_backward(L)
        return torch.cat(vals)

    @staticmethod
    def backward(ctx, g):
        (L,) = ctx.saved_tensors
        parts = list(torch.split(g.contiguous(), ctx.counts))
        gX, gL = filtration_given_backward(ctx.grid, L, ctx.cx, ctx.weights, ctx.srcs, parts, ctx.n_points)
        return gX, gL, None, None, None


def flood_values_given(X: torch.Tensor, L: torch.Tensor, grid: Grid, cx: DeviceComplex, weights):
    """Differentiable flood values over given point sets, split per dimension."""
    out = GivenFloodFunction.apply(X, L, grid, cx, weights)
    return list(torch.split(out, cx.counts))


# ---------------------------------------------------------------- ambient dimension d = 2..5
def _points_nd(X: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if X.dtype != torch.float32 or X.dim() != 2 or not 2 <= X.shape[1] <= _lib.ND_MAX_DIM:
        raise ValueError(f"{name} must be float32 of shape (n, d), 2 <= d <= {_lib.ND_MAX_DIM}")
    return X.contiguous()


def fps_nd(X: torch.Tensor, n_landmarks: int, start: int = 0, sync: bool = True):
    """Farthest point sampling in R^d (flood_fps_nd). Returns (idx int64[n], key float32[n])."""
    X = _points_nd(X, "X")
    idx = torch.empty(n_landmarks, dtype=torch.int64, device=X.device)
    key = torch.empty(n_landmarks, dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_fps_nd(_ptr(X), X.shape[0], X.shape[1], int(n_landmarks), int(start), _ptr(idx),
                                     _ptr(key), _stream_ptr(X.device))
    _finish(st, "flood_fps_nd", X.device, sync)
    return idx, key


class GridNd:
    """Library-owned cell grid over X in R^d (flood_build_grid_nd)."""

    def __init__(self, handle: C.c_void_p, device: torch.device, dim: int):
        self._h = handle
        self.device = device
        self.dim = dim

    @property
    def handle(self) -> C.c_void_p:
        if not self._h:
            raise ValueError("grid already destroyed")
        return self._h

    def info(self) -> dict:
        inf = _lib.GridNdInfo()
        _lib.check(_lib.get().flood_grid_nd_get_info(self.handle, C.byref(inf)), "flood_grid_nd_get_info")
        d = inf.dim
        return {"n_points": inf.n_points, "n_cells": inf.n_cells, "dim": d, "dims": tuple(inf.dims[:d]),
                "cell_size": inf.cell_size, "bbox_lo": tuple(inf.bbox_lo[:d]), "bbox_hi": tuple(inf.bbox_hi[:d]),
                "device_bytes": inf.device_bytes}

    def close(self) -> None:
        if self._h:
            _lib.get().flood_grid_nd_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_grid_nd(X: torch.Tensor, cell_size: float = 0.0, sync: bool = True) -> GridNd:
    """Cell grid over X in R^d (flood_build_grid_nd)."""
    X = _points_nd(X, "X")
    h = C.c_void_p(0)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_build_grid_nd(_ptr(X), X.shape[0], X.shape[1], float(cell_size), C.byref(h),
                                            _stream_ptr(X.device))
    _lib.check(st, "flood_build_grid_nd")
    grid = GridNd(h, X.device, X.shape[1])
    if sync:
        check(X.device)
    return grid


def filtration_nd(grid: GridNd, L: torch.Tensor, cx: DeviceComplex, m: int, sync: bool = True) -> list:
    """Flood values of every simplex of Del(L) in R^d (flood_filtration_nd): values[k] float32, k = 0..d."""
    L = _points_nd(L, "L")
    if L.shape[1] != grid.dim:
        raise ValueError(f"L has {L.shape[1]} coordinates, the grid {grid.dim}")
    K = _lib.ND_MAX_DIM + 1
    counts = cx.counts + [0] * (K - len(cx.counts))
    counts[0] = L.shape[0]
    s = _lib.P6(*[C.c_void_p(t.data_ptr() if t.numel() else 0) for t in cx.simplices[:K]] +
                [C.c_void_p(0)] * (K - len(cx.simplices)))
    f = _lib.P6(*[C.c_void_p(t.data_ptr() if t.numel() else 0) for t in cx.facets[:K]] +
                [C.c_void_p(0)] * (K - len(cx.facets)))
    n = _lib.I64x6(*counts)
    vals = [torch.empty(counts[k], dtype=torch.float32, device=L.device) for k in range(len(cx.simplices))]
    vp = _lib.P6(*[_ptr(v) if v.numel() else C.c_void_p(0) for v in vals] + [C.c_void_p(0)] * (K - len(vals)))
    with torch.cuda.device(L.device):
        st = _lib.get().flood_filtration_nd(grid.handle, _ptr(L), L.shape[0], s, f, n, int(m), vp,
                                            _stream_ptr(L.device))
    _finish(st, "flood_filtration_nd", L.device, sync)
    return vals


def last_filtration_nd_stats() -> dict:
    st = _lib.NdStats()
    _lib.check(_lib.get().flood_last_filtration_nd_stats(C.byref(st)), "flood_last_filtration_nd_stats")
    d = st.dim
    out = {"dim": d}
    for k in ("items", "pruned", "resolved", "exact", "fallback", "pairs", "pairs_fallback", "cells"):
        out[k] = list(getattr(st, k))[:d + 1]
    return out


def gather_rows(X: torch.Tensor, idx: torch.Tensor, sync: bool = True) -> torch.Tensor:
    """L = X[idx] on the device by flood_gather_rows (the landmark rows of FPS's picks)."""
    if not isinstance(X, torch.Tensor) or not X.is_cuda or X.dtype != torch.float32 or X.dim() != 2:
        raise ValueError("X must be a float32 CUDA tensor of shape (n, d)")
    if not isinstance(idx, torch.Tensor) or idx.device != X.device or idx.dtype != torch.int64 or idx.dim() != 1:
        raise ValueError("idx must be an int64 CUDA tensor of shape (n,) on X's device")
    X, idx = X.contiguous(), idx.contiguous()
    L = torch.empty((idx.shape[0], X.shape[1]), dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.get().flood_gather_rows(_ptr(X), X.shape[0], X.shape[1], _ptr(idx), idx.shape[0], _ptr(L),
                                          _stream_ptr(X.device))
    _finish(st, "flood_gather_rows", X.device, sync)
    return L
