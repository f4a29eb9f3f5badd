"""Landmarks that are not points of X (§3 allows L ⊄ X): parity of the CUDA path
with the FP64 oracle through the C ABI.

Vertex values are d(v, X) > 0, enter every coface through the facet maximum,
and bound the samples by min_j (|p - v_j| + d(v_j, X)). Bars as everywhere:
values within 1e-5 x the bounding-box diagonal of X; the attaining sample's
oracle distance equals the value; gradients against the oracle's subgradient.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _off(X, n_l, amp, seed, frac=1.0):
    """FPS landmarks of X (oracle), a fraction of them moved off X by U[-amp, amp]^3."""
    idx, _ = oracle.fps(X, n_l, 0)
    rng = np.random.default_rng(seed)
    L = X[idx].astype(np.float64)
    moved = rng.random(n_l) < frac
    L[moved] += rng.uniform(-amp, amp, (int(moved.sum()), 3))
    L = np.ascontiguousarray(L, dtype=np.float32)
    return L, delaunay_complex(L), moved


def gpu_values(X, L, cx, m, want_src=True):
    ops = _ops()
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    grid = ops.build_grid(Xd)
    vals, src = ops.filtration(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device), m, want_src=want_src)
    grid.close()
    return [v.cpu().numpy() for v in vals], ([s.cpu().numpy() for s in src] if want_src else None)


def assert_close(vals, ref, X, what):
    tol = TOL * _diam(X)
    for k in range(len(vals)):
        if vals[k].size:
            err = np.max(np.abs(vals[k].astype(np.float64) - ref[k]))
            assert err <= tol, f"{what} dim {k}: {err:.3e} > {tol:.3e}"


def check_src(X, L, cx, m, vals, src):
    ind = oracle.flood.KDIndex(X, "kdtree")
    tol = TOL * _diam(X)
    for k in (1, 2, 3):
        d = src[k][:, 0] >> 28
        rows = src[k][:, 0] & ((1 << 28) - 1)
        for dim in range(0, k + 1):
            t = np.nonzero(d == dim)[0]
            if t.size == 0:
                continue
            if dim == 0:
                P = L[rows[t]].astype(np.float64)
            else:
                comps = oracle.interior_compositions(m, dim)[src[k][t, 1]]
                P = np.einsum("nj,njd->nd", comps / m, L[cx.simplices[dim][rows[t]]].astype(np.float64))
            dist, _ = ind.query(P)
            assert np.max(np.abs(dist - vals[k][t])) <= tol, (k, dim)


def test_all_landmarks_off_X_sphere_10k():
    X = data.sphere_cloud()
    L, cx, _ = _off(X, 128, 0.02, seed=1)
    ref = oracle.flood_values(X, L, cx.simplices, 6, method="brute")
    vals, src = gpu_values(X, L, cx, 6)
    assert_close(vals, ref.values, X, "off X")
    assert np.all(vals[0] > 0)
    check_src(X, L, cx, 6, vals, src)
    assert np.any((src[1][:, 0] >> 28) == 0)          # some edges take a vertex's value


@pytest.mark.parametrize("m", [1, 4, 10])
def test_half_the_landmarks_off_X(m):
    X = data.torus_cloud(20000, seed=11)
    L, cx, moved = _off(X, 60, 0.03, seed=12, frac=0.5)
    ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
    vals, src = gpu_values(X, L, cx, m)
    assert_close(vals, ref.values, X, f"half off, m={m}")
    assert np.all(vals[0][~moved] == 0) and np.all(vals[0][moved] > 0)
    check_src(X, L, cx, m, vals, src)


def test_landmarks_far_outside_the_cloud():
    """Some landmarks far beyond X's bounding box: the nearest-point search widens
    its box until it holds a point, and every cull box is clamped to the grid."""
    X = data.shape_mix_cloud(20000, n_shapes=3, seed=21)
    idx, _ = oracle.fps(X, 40, 0)
    L = X[idx].astype(np.float64)
    L[:5] += np.array([0.0, 0.0, 12.0])
    L = np.ascontiguousarray(L, dtype=np.float32)
    cx = delaunay_complex(L)
    ref = oracle.flood_values(X, L, cx.simplices, 4, method="kdtree")
    vals, _ = gpu_values(X, L, cx, 4, want_src=False)
    assert_close(vals, ref.values, X, "far")


def test_given_sets_with_landmarks_off_X():
    ops = _ops()
    X = data.torus_cloud(20000, seed=31)
    L, cx, _ = _off(X, 50, 0.03, seed=32)
    w = [None] + [data.random_barycentric(cx.counts[k], (7, 15, 30)[k - 1], k, seed=33) for k in (1, 2, 3)]
    ref = oracle.flood_values_random(X, L, cx.simplices, w, method="kdtree")
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd)
    vals, _ = ops.filtration_given(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device),
                                   [None] + [torch.from_numpy(x).cuda() for x in w[1:]])
    grid.close()
    assert_close([v.cpu().numpy() for v in vals], ref.values, X, "given, off X")


def test_backward_with_landmarks_off_X():
    ops = _ops()
    X = data.jitter(data.torus_cloud(3000, seed=41), amp=1e-6, seed=42)
    L, cx, _ = _off(X, 30, 0.03, seed=43)
    m = 6
    gamma = data.upstream_gradients(cx.counts, seed=44)
    res = oracle.flood_values(X, L, cx.simplices, m, method="brute")
    dX_ref, dL_ref = oracle.analytic_gradient(X, L, cx.simplices, m, gamma, result=res)
    Xd = torch.from_numpy(X).cuda().requires_grad_(True)
    Ld = torch.from_numpy(L).cuda().requires_grad_(True)
    grid = ops.build_grid(Xd.detach())
    vals = ops.flood_values(Xd, Ld, grid, ops.to_device(cx, Xd.device), m)
    sum((v * torch.from_numpy(g).cuda()).sum() for v, g in zip(vals, gamma)).backward()
    grid.close()
    gX, gL = Xd.grad.cpu().numpy(), Ld.grad.cpu().numpy()
    scale = max(1.0, np.abs(dX_ref).max(), np.abs(dL_ref).max())
    assert np.max(np.abs(gX - dX_ref)) <= 1e-3 * scale
    assert np.max(np.abs(gL - dL_ref)) <= 1e-3 * scale
    assert np.array_equal(np.abs(gX).sum(1) > 0, np.abs(dX_ref).sum(1) > 0)
