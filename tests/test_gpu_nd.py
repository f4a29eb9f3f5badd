"""Parity of the general-dimension path (flood_fps_nd, flood_build_grid_nd,
flood_filtration_nd) with the FP64 oracle in ambient dimensions 2..5 (§3; §5.3, Fig. 4c).

Bars: FPS picks and keys bit-exact; flood values within 1e-5 x the diagonal of
X's bounding box; values bitwise independent of the cell size (every skip and
stop of the search is exact); the three-dimensional path and the general one
agree on the same cloud within the same tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import complex_from_simplices, data, delaunay_complex
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _gpu_values(X, L, cx, m, cell=0.0):
    ops = _ops()
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    grid = ops.build_grid_nd(Xd, cell)
    vals = ops.filtration_nd(grid, torch.from_numpy(np.ascontiguousarray(L, np.float32)).cuda(),
                             ops.to_device(cx, Xd.device), m)
    info = grid.info()
    grid.close()
    return [v.cpu().numpy() for v in vals], info


def _assert_close(got, ref, X, what=""):
    tol = TOL * _diam(X)
    for k, (g, r) in enumerate(zip(got, ref)):
        assert g.shape == r.shape, (what, k)
        if g.size:
            err = float(np.max(np.abs(g.astype(np.float64) - r)))
            assert err <= tol, f"{what} dim {k}: max |gpu - oracle| = {err:.3e} > {tol:.3e}"


# ---------------------------------------------------------------- FPS
@pytest.mark.parametrize("d,n,n_l,start,seed", [(2, 3000, 50, 0, 1), (3, 5001, 64, 17, 2), (4, 20_000, 100, 3, 3),
                                                (5, 40_000, 200, 0, 4), (5, 777, 777, 5, 5), (4, 1, 1, 0, 6)])
def test_fps_nd_bit_exact(d, n, n_l, start, seed):
    X = data.swisscheese_cloud(n, seed=seed, dim=d) if n > 1 else np.zeros((1, d), np.float32)
    idx, key = _ops().fps_nd(torch.from_numpy(X).cuda(), n_l, start)
    ref_i, ref_k = oracle.fps(X, n_l, start)
    assert np.array_equal(idx.cpu().numpy(), ref_i)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), ref_k.astype(np.float32).view(np.uint32))


def test_fps_nd_points_beyond_the_register_resident_ones():
    """3M points in R^5: more than the threads keep in registers and the blocks in shared memory;
    the rest are read from memory at every pick (all three tiers in use)."""
    rng = np.random.default_rng(81)
    X = rng.uniform(-1, 1, (3_000_000, 5)).astype(np.float32)
    idx, key = _ops().fps_nd(torch.from_numpy(X).cuda(), 60, 11)
    ref_i, ref_k = oracle.fps(X, 60, 11)
    assert np.array_equal(idx.cpu().numpy(), ref_i)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), ref_k.astype(np.float32).view(np.uint32))


def test_fps_nd_ties_duplicates_and_errors():
    ops = _ops()
    # the 4-cube's vertices, each twice: ties everywhere, lowest index wins
    V = np.array([[(i >> b) & 1 for b in (3, 2, 1, 0)] for i in range(16)], dtype=np.float32)
    X = np.concatenate([V, V])
    idx, key = ops.fps_nd(torch.from_numpy(X).cuda(), 16, 0)
    ref_i, ref_k = oracle.fps(X, 16, 0)
    assert np.array_equal(idx.cpu().numpy(), ref_i) and np.array_equal(key.cpu().numpy(), ref_k)
    with pytest.raises(FloodError) as e:
        ops.fps_nd(torch.from_numpy(X).cuda(), 17, 0)          # only 16 distinct points
    assert e.value.name == "FLOOD_EDEGENERATE"
    bad = X.copy()
    bad[5, 2] = np.inf
    with pytest.raises(FloodError) as e:
        ops.fps_nd(torch.from_numpy(bad).cuda(), 4, 0)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError) as e:
        ops.fps_nd(torch.from_numpy(X).cuda(), 4, 32)         # start out of range
    assert e.value.name == "FLOOD_EINVAL"
    idx, _ = ops.fps_nd(torch.from_numpy(X).cuda(), 4, 0)       # the stream still works
    assert np.array_equal(idx.cpu().numpy(), ref_i[:4])


def test_fps_nd_two_coordinates_through_the_three_dimensional_kernel():
    """d = 2 runs the 3-D FPS on the points at z = 0: ties, duplicates, one pick, one point,
    running out of distinct points, non-finite input and a cloud over many blocks, against the
    oracle's two-dimensional picks."""
    ops = _ops()
    # a 5 x 5 lattice, each point twice: many-way exact ties, lowest index wins
    g = np.array([[i, j] for i in range(5) for j in range(5)], dtype=np.float32)
    X = np.concatenate([g, g])
    idx, key = ops.fps_nd(torch.from_numpy(X).cuda(), 25, 3)
    ref_i, ref_k = oracle.fps(X, 25, 3)
    assert np.array_equal(idx.cpu().numpy(), ref_i) and np.array_equal(key.cpu().numpy(), ref_k)
    idx, key = ops.fps_nd(torch.from_numpy(X).cuda(), 1, 7)     # the start alone
    assert idx.cpu().numpy().tolist() == [7] and np.isinf(key.cpu().numpy()[0])
    one = np.array([[0.25, -1.5]], dtype=np.float32)             # a single point
    idx, _ = ops.fps_nd(torch.from_numpy(one).cuda(), 1, 0)
    assert idx.cpu().numpy().tolist() == [0]
    with pytest.raises(FloodError) as e:
        ops.fps_nd(torch.from_numpy(X).cuda(), 26, 0)           # only 25 distinct points
    assert e.value.name == "FLOOD_EDEGENERATE"
    bad = X.copy()
    bad[11, 1] = np.nan
    with pytest.raises(FloodError) as e:
        ops.fps_nd(torch.from_numpy(bad).cuda(), 4, 0)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError) as e:
        ops.fps_nd(torch.from_numpy(X).cuda(), 4, 50)          # start out of range
    assert e.value.name == "FLOOD_EINVAL"
    # many blocks (points on chip across the grid-wide exchange)
    Y = data.swisscheese_cloud(200_000, seed=31, dim=2)
    idx, key = ops.fps_nd(torch.from_numpy(Y).cuda(), 500, 9)
    ref_i, ref_k = oracle.fps(Y, 500, 9)
    assert np.array_equal(idx.cpu().numpy(), ref_i)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), ref_k.astype(np.float32).view(np.uint32))


# ---------------------------------------------------------------- flood values
def _case(d, n, n_l, seed):
    X = data.swisscheese_cloud(n, seed=seed, dim=d)
    L = X[oracle.fps(X, n_l, 0)[0]]
    return X, L, delaunay_complex(L)


@pytest.mark.parametrize("d,n,n_l,m,seed", [(4, 20_000, 40, 6, 11), (5, 20_000, 30, 6, 12), (4, 30_000, 60, 10, 13),
                                            (5, 50_000, 45, 12, 14), (2, 10_000, 80, 8, 15), (3, 10_000, 60, 8, 16)])
def test_filtration_nd_matches_oracle(d, n, n_l, m, seed):
    X, L, cx = _case(d, n, n_l, seed)
    got, info = _gpu_values(X, L, cx, m)
    assert info["dim"] == d and info["n_points"] == n
    ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree").values
    _assert_close(got, ref, X, f"d={d} m={m}")
    assert np.all(got[0] == 0.0)                               # landmarks are points of X


@pytest.mark.parametrize("d", [4, 5])
def test_filtration_nd_is_bitwise_independent_of_the_cell_size(d):
    X, L, cx = _case(d, 30_000, 50, 21 + d)
    base, info = _gpu_values(X, L, cx, 8)
    for cell in (0.25 * info["cell_size"], 3.0 * info["cell_size"], 100.0):
        got, inf2 = _gpu_values(X, L, cx, 8, cell)
        for k in range(d + 1):
            assert np.array_equal(got[k].view(np.uint32), base[k].view(np.uint32)), (cell, k)
    assert inf2["n_cells"] == 1                                # an edge above the extent: one cell


def test_filtration_nd_landmarks_off_the_cloud():
    """L not a subset of X (§3): vertex values d(v, X) > 0 and every bound uses them."""
    rng = np.random.default_rng(31)
    X, L, _ = _case(5, 20_000, 35, 31)
    L = (L + rng.normal(0, 0.05, L.shape)).astype(np.float32)
    cx = delaunay_complex(L)
    got, _ = _gpu_values(X, L, cx, 6)
    ref = oracle.flood_values(X, L, cx.simplices, 6, method="kdtree").values
    _assert_close(got, ref, X, "L off X")
    assert np.all(got[0] > 0)


def test_three_dimensional_cloud_in_five_dimensions_matches_the_3d_path():
    """A 3-D cloud embedded in R^5 (two zero coordinates): the general path gives the 3-D path's values."""
    ops = _ops()
    X3 = data.torus_cloud(40_000, seed=41)
    idx, key = oracle.fps(X3, 150, 0)
    L3 = X3[idx]
    cx = delaunay_complex(L3)
    Xd = torch.from_numpy(X3).cuda()
    g3 = ops.build_grid(Xd, 0.0)
    v3, _ = ops.filtration(g3, torch.from_numpy(L3).cuda(), ops.to_device(cx, Xd.device), 8, want_src=False)
    g3.close()
    X5 = np.zeros((X3.shape[0], 5), np.float32)
    X5[:, :3] = X3
    got, info = _gpu_values(X5, X5[idx], cx, 8)
    assert info["dims"][3] == 1 and info["dims"][4] == 1       # flat axes get one cell
    _assert_close(got[:4], [v.cpu().numpy().astype(np.float64) for v in v3], X3, "3-D in 5-D")


def test_filtration_nd_regular_simplex_closed_form():
    d = 5
    E = np.eye(d + 1) - 1.0 / (d + 1)
    Q, _ = np.linalg.qr(E.T)
    V = (E @ Q[:, :d]).astype(np.float32)
    V *= np.float32(2.0 / np.linalg.norm(V[0] - V[1]))
    cx = complex_from_simplices([np.arange(d + 1)[None]], d + 1)
    got, _ = _gpu_values(V, V, cx, 12)
    Vf = V.astype(np.float64)
    R = np.linalg.norm(Vf - Vf.mean(0), axis=1).min()
    assert abs(got[d][0] - R) <= 1e-6 * R + TOL * _diam(V)
    assert np.allclose(got[1], np.linalg.norm(Vf[0] - Vf[1]) / 2, rtol=2e-6)


def test_filtration_nd_small_m_and_empty_dimensions():
    X, L, cx = _case(4, 8000, 25, 51)
    for m in (1, 2, 3, 4):                                     # m < k + 1: no interior samples in dimension k
        got, _ = _gpu_values(X, L, cx, m)
        ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree").values
        _assert_close(got, ref, X, f"m={m}")
    # a complex whose top dimensions are empty (edges and triangles only)
    tris = cx.simplices[2][:50]
    cx2 = complex_from_simplices([tris], L.shape[0], top_dim=2)
    got, _ = _gpu_values(X, L, cx2, 6)
    ref = oracle.flood_values(X, L, cx2.simplices, 6, method="kdtree").values
    _assert_close(got, ref, X, "edges and triangles")


@pytest.mark.parametrize("d,n", [(5, 7), (5, 12), (4, 9), (4, 40), (2, 4)])
def test_filtration_nd_tiny_clouds(d, n):
    """Every point a landmark (L = X): a handful of points, one or a few cells."""
    rng = np.random.default_rng(100 + n + d)
    X = rng.uniform(-1, 1, (n, d)).astype(np.float32)
    cx = delaunay_complex(X)
    got, _ = _gpu_values(X, X, cx, 6)
    ref = oracle.flood_values(X, X, cx.simplices, 6).values
    _assert_close(got, ref, X, f"tiny d={d} n={n}")


def test_filtration_nd_large_m_and_duplicates():
    """m = 19 (20 points per edge, §5.3) in R^4, on a cloud where every point appears three times."""
    rng = np.random.default_rng(121)
    base = data.swisscheese_cloud(4000, seed=122, dim=4)
    X = np.concatenate([base, base, base])
    L = base[oracle.fps(base, 25, 0)[0]]
    cx = delaunay_complex(L)
    got, _ = _gpu_values(X, L, cx, 19)
    ref = oracle.flood_values(X, L, cx.simplices, 19, method="kdtree").values
    _assert_close(got, ref, X, "m=19 duplicates")


def test_filtration_nd_rejects_bad_input():
    ops = _ops()
    X, L, cx = _case(5, 5000, 20, 61)
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid_nd(Xd)
    dcx = ops.to_device(cx, Xd.device)
    Ld = torch.from_numpy(L).cuda()
    with pytest.raises(ValueError):
        ops.filtration_nd(grid, Ld[:, :4].contiguous(), dcx, 6)
    with pytest.raises(FloodError) as e:
        ops.filtration_nd(grid, Ld, dcx, 65)
    assert e.value.name == "FLOOD_EINVAL"
    bad = [s.clone() for s in dcx.simplices]
    bad[3][7, 1] = 10_000
    with pytest.raises(FloodError) as e:
        ops.filtration_nd(grid, Ld, ops.DeviceComplex(dcx.n_vertices, bad, dcx.facets), 6)
    assert e.value.name == "FLOOD_EINVAL"
    Lb = Ld.clone()
    Lb[3, 0] = float("nan")
    with pytest.raises(FloodError) as e:
        ops.filtration_nd(grid, Lb, dcx, 6)
    assert e.value.name == "FLOOD_EINVAL"
    got = ops.filtration_nd(grid, Ld, dcx, 6)                  # and the next call works
    ref = oracle.flood_values(X, L, cx.simplices, 6, method="kdtree").values
    _assert_close([v.cpu().numpy() for v in got], ref, X, "after errors")
    grid.close()


def test_filtration_nd_stats_account_for_every_item():
    ops = _ops()
    X, L, cx = _case(5, 30_000, 40, 71)
    _gpu_values(X, L, cx, 8)
    st = ops.last_filtration_nd_stats()
    assert st["dim"] == 5
    from math import comb
    for k in range(6):
        n_items = (L.shape[0] if k == 0 else cx.counts[k] * comb(7, k))
        assert st["items"][k] == n_items
        assert st["pruned"][k] + st["resolved"][k] + st["exact"][k] + st["fallback"][k] == n_items
    assert st["pruned"][0] == 0 and st["resolved"][0] == L.shape[0]   # every landmark finds itself


def _golden(name):
    import importlib.util
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_fps_golden", os.path.join(here, "golden", "make_fps_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod, mod.read(name)


@pytest.mark.slow
@pytest.mark.parametrize("d", [4, 5])
def test_fps_nd_full_size_equals_stored_oracle_picks(d):
    """|X| = 1M, |L| = 1k in R^d (Fig. 4c's workload): every pick equals the oracle's stored pick."""
    mod, g = _golden(f"swisscheese{d}d-1M")
    X = data.swisscheese_cloud(1_000_000, seed=6, dim=d)
    assert mod.cloud_sha256(X) == g["x_sha256"]
    idx, key = _ops().fps_nd(torch.from_numpy(X).cuda(), 1000, 0)
    assert np.array_equal(idx.cpu().numpy(), g["idx"])
    assert key.cpu().numpy()[-1].view(np.uint32) == np.uint32(int(g["last_key_hex"], 16))


@pytest.mark.slow
def test_filtration_nd_swisscheese_5d_1m_sampled():
    """The scaling workload of Fig. 4c at d = 5: |X| = 1M, |L| = 1k, m = 10; sampled values against the oracle."""
    mod, g = _golden("swisscheese5d-1M")
    X = data.swisscheese_cloud(1_000_000, seed=6, dim=5)
    assert mod.cloud_sha256(X) == g["x_sha256"]
    ref_i = g["idx"]
    L = X[ref_i]
    cx = delaunay_complex(L)
    got, _ = _gpu_values(X, L, cx, 10)
    rng = np.random.default_rng(91)
    subset = [None] + [rng.choice(cx.counts[k], min(60, cx.counts[k]), replace=False) for k in range(1, 6)]
    subset[0] = np.arange(0)
    ref = oracle.flood_values(X, L, cx.simplices, 10, method="kdtree", subset=subset)
    for k in range(1, 6):
        err = np.max(np.abs(got[k][subset[k]].astype(np.float64) - ref.values[k]))
        assert err <= TOL * _diam(X), (k, err)
