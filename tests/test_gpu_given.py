"""Parity of flood_filtration_given (caller-given point sets P_sigma, e.g. the
uniform random draws of Lemma 4) with the FP64 oracle, through the C ABI.

Bars: values within 1e-5 x the diagonal of X's bounding box; the attaining
(dim, row, sample) names a point whose oracle distance is the value; with the
interior grid as the given sets, values and src bit for bit those of the grid
path. Landmarks come from the oracle's FPS, weights from the seeded generator.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.random_flood import lambdas
from paper_2509_22432_b300 import complex_from_simplices, data, delaunay_complex
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _dev():
    return torch.device("cuda:0")


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _weights(cx, S, seed):
    return [None] + [data.random_barycentric(cx.counts[k], S[k - 1], k, seed=seed) for k in (1, 2, 3)]


def _dw(w):
    return [None] + [torch.from_numpy(np.ascontiguousarray(x)).to(_dev()) for x in w[1:]]


def gpu_given(X, L, cx, w, cell_size=0.0, want_src=True):
    ops = _ops()
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(_dev())
    grid = ops.build_grid(Xd, cell_size)
    Ld = torch.from_numpy(np.ascontiguousarray(L)).to(_dev())
    vals, src = ops.filtration_given(grid, Ld, ops.to_device(cx, _dev()), _dw(w), want_src=want_src)
    out = [v.cpu().numpy() for v in vals], ([s.cpu().numpy() for s in src] if want_src else None)
    grid.close()
    return out


def _landmarks(X, n_l):
    idx, key = oracle.fps(X, n_l, 0)
    L = X[idx]
    return L, delaunay_complex(L), key


def assert_close(vals, ref, X, what=""):
    tol = TOL * _diam(X)
    for k in range(len(vals)):
        got = np.asarray(vals[k], np.float64)
        assert got.shape == ref[k].shape, (what, k)
        if got.size:
            err = np.max(np.abs(got - ref[k]))
            assert err <= tol, f"{what} dim {k}: max |gpu - oracle| = {err:.3e} > {tol:.3e}"


def check_src(X, L, cx, w, vals, src, index=None, rows_per_dim=None):
    """src[k][i] = (dim << 28 | row, s) must name a point of that simplex's set whose
    oracle distance to X is the value (or a vertex, value 0)."""
    ind = index or oracle.flood.KDIndex(X, "kdtree")
    tol = TOL * _diam(X)
    for k in (1, 2, 3):
        sel = np.arange(cx.counts[k]) if rows_per_dim is None else rows_per_dim[k]
        d = src[k][sel, 0] >> 28
        rows = src[k][sel, 0] & ((1 << 28) - 1)
        s = src[k][sel, 1]
        assert np.all(d <= k)
        v0 = d == 0
        assert np.all(vals[k][sel][v0] == 0.0)
        for dim in range(1, k + 1):
            t = np.nonzero(d == dim)[0]
            if t.size == 0:
                continue
            assert np.all(s[t] >= 0) and np.all(s[t] < w[dim].shape[1])
            lam = lambdas(w[dim][rows[t], s[t]])
            P = np.einsum("nj,njd->nd", lam, L[cx.simplices[dim][rows[t]]].astype(np.float64))
            dist, _ = ind.query(P)
            assert np.max(np.abs(dist - vals[k][sel][t])) <= tol, (k, dim)


def test_given_sphere_10k_random_sets():
    """Unit sphere + noise, 10,000 points, 128 landmarks, uniform random sets of 9 / 20 / 35 points."""
    X = data.sphere_cloud()
    L, cx, _ = _landmarks(X, 128)
    w = _weights(cx, (9, 20, 35), seed=11)
    ref = oracle.flood_values_random(X, L, cx.simplices, w, method="brute")
    vals, src = gpu_given(X, L, cx, w)
    assert_close(vals, ref.values, X, "sphere")
    assert np.all(vals[0] == 0)
    check_src(X, L, cx, w, vals, src)
    for k in range(2, 4):
        assert np.all(vals[k - 1][cx.facets[k]].max(axis=1) <= vals[k])


@pytest.mark.parametrize("S", [(0, 0, 0), (1, 1, 1), (0, 5, 0), (3, 0, 7), (257, 100, 50), (31, 33, 65)])
def test_given_sample_counts(S):
    X = data.torus_cloud(6000, seed=21)
    L, cx, _ = _landmarks(X, 40)
    w = _weights(cx, S, seed=22)
    ref = oracle.flood_values_random(X, L, cx.simplices, w, method="kdtree")
    vals, src = gpu_given(X, L, cx, w)
    assert_close(vals, ref.values, X, f"S={S}")
    check_src(X, L, cx, w, vals, src)


@pytest.mark.parametrize("m", [4, 10])
def test_given_interior_grid_is_the_grid_path_bitwise(m):
    """lambda_j = fl32(c_j / m) over the interior compositions: bit for bit flood_filtration(m)."""
    ops = _ops()
    X = data.torus_cloud(20000, seed=31)
    L, cx, _ = _landmarks(X, 60)
    w = [None]
    for k in (1, 2, 3):
        lam = (oracle.interior_compositions(m, k).astype(np.float32) / np.float32(m)).astype(np.float32)
        w.append(np.ascontiguousarray(np.broadcast_to(lam, (cx.counts[k],) + lam.shape)))
    Xd = torch.from_numpy(X).to(_dev())
    grid = ops.build_grid(Xd)
    Ld = torch.from_numpy(L).to(_dev())
    dcx = ops.to_device(cx, _dev())
    gv, gs = ops.filtration(grid, Ld, dcx, m)
    rv, rs = ops.filtration_given(grid, Ld, dcx, _dw(w))
    grid.close()
    for k in range(4):
        assert np.array_equal(gv[k].cpu().numpy().view(np.uint32), rv[k].cpu().numpy().view(np.uint32)), k
        assert np.array_equal(gs[k].cpu().numpy(), rs[k].cpu().numpy()), k


@pytest.mark.parametrize("n", [4, 5, 9, 17, 63])
def test_given_tiny_ragged_clouds(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, 3)).astype(np.float32)
    L, cx, _ = _landmarks(X, min(n, 6))
    w = _weights(cx, (3, 4, 5), seed=n)
    ref = oracle.flood_values_random(X, L, cx.simplices, w, method="brute")
    vals, _ = gpu_given(X, L, cx, w)
    assert_close(vals, ref.values, X, f"n={n}")


def test_given_large_sets_span_many_groups():
    """5,000 points per edge and 2,000 per triangle: one simplex spreads over many sample groups."""
    X = data.sphere_cloud(3000, seed=51)
    L, cx, _ = _landmarks(X, 16)
    w = _weights(cx, (5000, 2000, 300), seed=52)
    ref = oracle.flood_values_random(X, L, cx.simplices, w, method="kdtree")
    vals, src = gpu_given(X, L, cx, w)
    assert_close(vals, ref.values, X, "large sets")
    check_src(X, L, cx, w, vals, src)


def test_given_values_bitwise_invariant_to_cell_size():
    X = data.torus_cloud(30000, seed=61)
    L, cx, key = _landmarks(X, 80)
    w = _weights(cx, (7, 15, 30), seed=62)
    h = float(np.sqrt(key[-1]))
    base, bsrc = gpu_given(X, L, cx, w, cell_size=0.5 * h)
    for c in (0.2 * h, 1.7 * h, 0.0):
        v, s = gpu_given(X, L, cx, w, cell_size=c)
        for k in range(4):
            assert np.array_equal(v[k].view(np.uint32), base[k].view(np.uint32)), (c, k)
            assert np.array_equal(s[k], bsrc[k]), (c, k)


def test_given_invalid_inputs_raise():
    ops = _ops()
    X = data.sphere_cloud(2000, seed=71)
    L, cx, _ = _landmarks(X, 20)
    Xd = torch.from_numpy(X).to(_dev())
    grid = ops.build_grid(Xd)
    Ld = torch.from_numpy(L).to(_dev())
    dcx = ops.to_device(cx, _dev())
    w = _dw(_weights(cx, (3, 3, 3), seed=72))
    bad = [None] + [t.clone() for t in w[1:]]
    bad[2][1, 2, 1] = float("nan")
    with pytest.raises(FloodError) as e:
        ops.filtration_given(grid, Ld, dcx, bad)
    assert e.value.name == "FLOOD_EINVAL"
    big = [None, torch.full((cx.counts[1], 65537, 2), 0.5, device=_dev()), w[2], w[3]]
    with pytest.raises(FloodError) as e:
        ops.filtration_given(grid, Ld, dcx, big)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(ValueError):
        ops.filtration_given(grid, Ld, dcx, [None, w[1], w[2][:, :, :2].contiguous(), w[3]])
    with pytest.raises(ValueError):
        ops.filtration_given(grid, Ld, dcx, [None, w[1], None, w[3]])
    # the library still works after the rejected calls
    vals, _ = ops.filtration_given(grid, Ld, dcx, w)
    assert torch.isfinite(vals[3]).all()
    grid.close()


def test_given_edges_only():
    X = data.sphere_cloud(3000, seed=81)
    idx, _ = oracle.fps(X, 10, 0)
    L = X[idx]
    edges_only = complex_from_simplices([delaunay_complex(L).simplices[1]], 10)
    w = [None, data.random_barycentric(edges_only.counts[1], 6, 1, seed=82),
         np.zeros((0, 0, 3), np.float32), np.zeros((0, 0, 4), np.float32)]
    ref = oracle.flood_values_random(X, L, edges_only.simplices, w, method="brute")
    vals, _ = gpu_given(X, L, edges_only, w)
    assert_close(vals, ref.values, X, "edges only")


def test_given_backward_matches_oracle_gradient():
    ops = _ops()
    X = data.jitter(data.torus_cloud(3000, seed=91), amp=1e-6, seed=92)
    L, cx, _ = _landmarks(X, 30)
    L = L.copy()
    w = _weights(cx, (5, 8, 12), seed=93)
    gamma = data.upstream_gradients(cx.counts, seed=94)
    res = oracle.flood_values_random(X, L, cx.simplices, w, method="brute")
    dX_ref, dL_ref = oracle.analytic_gradient_random(X, L, cx.simplices, w, gamma, res)
    dev = _dev()
    Xd = torch.from_numpy(X).to(dev).requires_grad_(True)
    Ld = torch.from_numpy(L).to(dev).requires_grad_(True)
    grid = ops.build_grid(Xd.detach())
    vals = ops.flood_values_given(Xd, Ld, grid, ops.to_device(cx, dev), _dw(w))
    sum((v * torch.from_numpy(g).to(dev)).sum() for v, g in zip(vals, gamma)).backward()
    grid.close()
    gX, gL = Xd.grad.cpu().numpy(), Ld.grad.cpu().numpy()
    scale = max(1.0, np.abs(dX_ref).max(), np.abs(dL_ref).max())
    assert np.max(np.abs(gX - dX_ref)) <= 1e-3 * scale
    assert np.max(np.abs(gL - dL_ref)) <= 1e-3 * scale
    assert np.array_equal(np.abs(gX).sum(1) > 0, np.abs(dX_ref).sum(1) > 0)


@pytest.mark.slow
def test_given_torus_1m_every_simplex():
    """1,000,000-point torus, 2,000 landmarks, uniform random sets of 9 / 36 / 84 points per
    edge / triangle / tetrahedron (the interior counts of m = 10): every simplex."""
    X = data.torus_cloud()
    L, cx, key = _landmarks(X, 2000)
    w = _weights(cx, (9, 36, 84), seed=7)
    ind = oracle.flood.KDIndex(X, "kdtree")
    ref = oracle.flood_values_random(X, L, cx.simplices, w, index=ind)
    vals, src = gpu_given(X, L, cx, w, cell_size=0.5 * float(np.sqrt(key[-1])))
    assert_close(vals, ref.values, X, "torus 1M")
    rng = np.random.default_rng(3)
    rows = [None] + [rng.choice(cx.counts[k], min(cx.counts[k], 2000), replace=False) for k in (1, 2, 3)]
    check_src(X, L, cx, w, vals, src, index=ind, rows_per_dim=rows)
