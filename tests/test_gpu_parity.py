"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: FPS landmark indices bit-exact; flood values within 1e-5 x the diagonal
of X's bounding box (the tolerance the benchmark spec fixes); integer outputs exact.
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


def _dev():
    return torch.device("cuda:0")


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def gpu_flood(X, L, cx, m, cell_size=0.0, want_src=True):
    ops = _ops()
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(_dev())
    grid = ops.build_grid(Xd, cell_size)
    Ld = torch.from_numpy(np.ascontiguousarray(L)).to(_dev())
    vals, src = ops.filtration(grid, Ld, ops.to_device(cx, _dev()), m, want_src=want_src)
    stats = ops.last_filtration_stats()
    out = [v.cpu().numpy() for v in vals], ([s.cpu().numpy() for s in src] if want_src else None), stats
    grid.close()
    return out


def assert_close(vals, ref, X, what=""):
    tol = TOL * _diam(X)
    for k in range(len(vals)):
        got = np.asarray(vals[k], np.float64)
        assert got.shape == ref[k].shape, (what, k)
        if got.size:
            err = np.max(np.abs(got - ref[k]))
            assert err <= tol, f"{what} dim {k}: max |gpu - oracle| = {err:.3e} > {tol:.3e}"


# ----------------------------------------------------------------------------- FPS

@pytest.mark.parametrize("n,n_l,start,seed", [(1, 1, 0, 0), (7, 7, 3, 1), (1000, 64, 0, 2), (4099, 300, 17, 3),
                                               (10_000, 128, 0, 1)])
def test_fps_bit_exact_small(n, n_l, start, seed):
    X = data.sphere_cloud(n, seed=seed)
    idx, key = _ops().fps(torch.from_numpy(X).to(_dev()), n_l, start)
    ri, rk = oracle.fps(X, n_l, start)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), rk.view(np.uint32))


def test_fps_ties_and_duplicates():
    # a lattice has many exactly equal keys; ties must go to the lowest index
    g = np.stack(np.meshgrid(np.arange(12), np.arange(12), np.arange(12), indexing="ij"), -1).reshape(-1, 3)
    X = np.concatenate([g, g[:100]]).astype(np.float32)          # duplicated points too
    idx, _ = _ops().fps(torch.from_numpy(X).to(_dev()), 200, 5)
    ri, _ = oracle.fps(X, 200, 5)
    assert np.array_equal(idx.cpu().numpy(), ri)


# Every launch shape of the persistent FPS kernel gives the same picks: one
# block holding its points on chip (n <= 7,168), several such blocks, one
# block streaming chunks from memory, several streaming blocks; and runs to
# the last point, where rounds make many picks at small, close keys.
@pytest.mark.parametrize("n,n_l,blocks,seed", [
    (5_000, 200, 0, 11), (5_000, 200, 3, 12),
    (30_000, 300, 0, 13), (30_000, 300, 4, 14), (30_000, 300, 1, 15), (30_000, 300, 5, 24),
    (100_000, 500, 0, 16), (100_000, 500, 1, 17), (100_000, 500, 5, 18),
    (3_000, 3_000, 0, 21), (3_000, 3_000, 2, 22), (20_000, 4_000, 2, 23)])
def test_fps_launch_shapes_bit_exact(n, n_l, blocks, seed):
    X = data.shape_mix_cloud(n, seed=seed)
    idx, key = _ops().fps(torch.from_numpy(X).to(_dev()), n_l, 0, n_blocks=blocks)
    ri, rk = oracle.fps(X, n_l, 0)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), rk.view(np.uint32))


def test_fps_ties_in_spatial_order():
    # A shuffled 40^3 integer lattice (plus duplicates): keys are small
    # integers, so nearly every pick is a many-way exact tie that must go to
    # the lowest original row although points are processed in Morton order.
    g = np.stack(np.meshgrid(np.arange(40), np.arange(40), np.arange(40), indexing="ij"), -1).reshape(-1, 3)
    g = g[np.random.default_rng(21).permutation(g.shape[0])]
    X = np.concatenate([g, g[:500]]).astype(np.float32)
    ri, rk = oracle.fps(X, 400, 7)
    for blocks in (0, 1, 3, 9):
        idx, key = _ops().fps(torch.from_numpy(X).to(_dev()), 400, 7, n_blocks=blocks)
        assert np.array_equal(idx.cpu().numpy(), ri), blocks
        assert np.array_equal(key.cpu().numpy(), rk), blocks


def test_fps_rejects_nonfinite_in_sorted_path_and_bad_width():
    ops = _ops()
    Y = data.sphere_cloud(20_000)
    Y[12_345, 2] = np.inf
    with pytest.raises(FloodError) as e:
        ops.fps(torch.from_numpy(Y).to(_dev()), 5, 0)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError) as e:
        ops.fps(torch.from_numpy(data.sphere_cloud(100)).to(_dev()), 5, 0, n_blocks=-1)
    assert e.value.name == "FLOOD_EINVAL"


@pytest.mark.slow
def test_fps_one_block_enlarged_chunks():
    """1.3M points on one block: chunks grow to 320 points so their metadata fits shared memory."""
    X = data.torus_cloud(1_300_000, seed=19)
    idx, key = _ops().fps(torch.from_numpy(X).to(_dev()), 64, 0, n_blocks=1)
    ri, rk = oracle.fps(X, 64, 0)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(key.cpu().numpy(), rk)


def test_fps_degenerate_and_invalid():
    ops = _ops()
    X = np.zeros((10, 3), np.float32)
    X[1] = 1.0
    with pytest.raises(FloodError) as e:
        ops.fps(torch.from_numpy(X).to(_dev()), 3, 0)
    assert e.value.name == "FLOOD_EDEGENERATE"
    Y = data.sphere_cloud(100)
    Y[5, 1] = np.nan
    with pytest.raises(FloodError) as e:
        ops.fps(torch.from_numpy(Y).to(_dev()), 5, 0)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError):
        ops.fps(torch.from_numpy(data.sphere_cloud(100)).to(_dev()), 101, 0)


@pytest.mark.slow
def test_fps_bit_exact_torus_1m():
    """1M-point torus, 2000 landmarks (register-resident variant at full size)."""
    X = data.torus_cloud()
    idx, key = _ops().fps(torch.from_numpy(X).to(_dev()), 2000, 0)
    ri, rk = oracle.fps(X, 2000, 0)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(key.cpu().numpy(), rk)


# ----------------------------------------------------------------------------- flood values

def _case(X, n_l, m, method="brute"):
    idx, _ = oracle.fps(X, n_l, 0)
    L = X[idx]
    cx = delaunay_complex(L)
    ref = oracle.flood_values(X, L, cx.simplices, m, method=method)
    return L, cx, ref


def test_flood_sphere_10k_m6_all_simplices():
    """Unit sphere + noise, 10,000 points, 128 FPS landmarks, m=6: every simplex vs brute force."""
    X = data.sphere_cloud()
    L, cx, ref = _case(X, 128, 6, method="brute")
    vals, src, stats = gpu_flood(X, L, cx, 6)
    assert_close(vals, ref.values, X, "sphere")
    assert np.all(vals[0] == 0)
    assert stats["pairs"][3] > 0


@pytest.mark.parametrize("m", [1, 2, 3, 5, 12, 19])
def test_flood_resolutions(m):
    X = data.torus_cloud(6000, seed=7)
    L, cx, ref = _case(X, 40, m, method="kdtree")
    vals, _, _ = gpu_flood(X, L, cx, m)
    assert_close(vals, ref.values, X, f"m={m}")


def test_sample_counts_match_the_grid_printed_in_the_paper():
    """§5.3 prints 210 points per triangle and 1540 per tetrahedron at 20 points per edge
    (m = 19); the CUDA path evaluates the interior samples of every face once, so on one
    tetrahedron its per-dimension sample counts plus the vertices add up to those totals."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "grid_counts_sec5_3.txt")
    per_edge, per_tri, per_tet = [tuple(int(v) for v in l.split()) for l in open(path)
                                  if l.strip() and not l.startswith("#")][0]
    m = per_edge - 1
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float32)
    cx = complex_from_simplices([np.array([[0, 1, 2, 3]])], 4)
    _, _, stats = gpu_flood(V, V, cx, m)
    s = stats["samples"]
    assert s[1] == 6 * (per_edge - 2)
    assert 3 + 3 * s[1] // 6 + s[2] // 4 == per_tri
    assert 4 + s[1] + s[2] + s[3] == per_tet


@pytest.mark.parametrize("m", [24, 30])
def test_flood_many_samples_per_simplex(m):
    """Many samples per simplex (hundreds to thousands) through the bucketed sample groups."""
    X = data.sphere_cloud(20_000, seed=9)
    L, cx, ref = _case(X, 24, m, method="kdtree")
    vals, _, stats = gpu_flood(X, L, cx, m)
    assert_close(vals, ref.values, X, f"m={m}")
    assert 0 < stats["active_samples"][3] <= stats["samples"][3]


@pytest.mark.parametrize("n", [4, 5, 9, 17, 63])
def test_flood_tiny_ragged_clouds(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, 3)).astype(np.float32)
    n_l = min(n, 6)
    L, cx, ref = _case(X, n_l, 4)
    vals, _, _ = gpu_flood(X, L, cx, 4)
    assert_close(vals, ref.values, X, f"n={n}")


def test_flood_closed_forms_on_gpu():
    # regular tetrahedron with X = its vertices: f = a sqrt(6)/4 exactly at 4 | m
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float32)
    cx = complex_from_simplices([np.array([[0, 1, 2, 3]])], 4)
    vals, src, _ = gpu_flood(V, V, cx, 8)
    a = 2 * np.sqrt(2)
    assert abs(vals[3][0] - a * np.sqrt(6) / 4) <= 1e-6
    assert np.allclose(vals[1], a / 2, atol=1e-6)         # edges between their two points
    assert (src[3][0, 0] >> 28) == 3                       # attained by the tetrahedron's own interior


def test_flood_flat_and_duplicate_points():
    rng = np.random.default_rng(3)
    X = np.concatenate([rng.uniform(-1, 1, (3000, 2)), np.zeros((3000, 1))], 1)
    X[:, 2] += rng.normal(0, 1e-3, 3000)
    X = np.concatenate([X, X[:500]]).astype(np.float32)
    L, cx, ref = _case(X, 30, 6, method="kdtree")
    vals, _, _ = gpu_flood(X, L, cx, 6)
    assert_close(vals, ref.values, X, "flat")


def test_values_bitwise_invariant_to_cell_size():
    """Each value depends only on (simplex, sample, point) arithmetic: tiling must not change a bit."""
    X = data.shape_mix_cloud(40_000, seed=31)
    idx, _ = oracle.fps(X, 80, 0)
    L = X[idx]
    cx = delaunay_complex(L)
    runs = [gpu_flood(X, L, cx, 8, cell_size=h, want_src=True) for h in (0.0, 0.05, 0.2, 1.0, 3.0)]
    ref = oracle.flood_values(X, L, cx.simplices, 8, method="kdtree")
    assert_close(runs[0][0], ref.values, X, "default cell size")
    for v, s, _ in runs[1:]:
        for k in range(4):
            assert np.array_equal(v[k].view(np.uint32), runs[0][0][k].view(np.uint32))
            assert np.array_equal(s[k], runs[0][1][k])


def test_voids_heavy_groups_and_empty_shells():
    """A swisscheese-like cloud (§5.3 synthetic data: uniform points minus balls) at several cell
    sizes: samples inside the voids are far from every point, so they run in the heavy-group kernel,
    many are dropped by the nearest-landmark bound and scans start past empty shells. Values must
    match the oracle and stay bitwise identical across cell sizes."""
    X = data.swisscheese_cloud(30_000, n_holes=6, seed=17)
    idx, _ = oracle.fps(X, 150, 0)
    L = X[idx]
    cx = delaunay_complex(L)
    ref = oracle.flood_values(X, L, cx.simplices, 8, method="kdtree")
    runs = [gpu_flood(X, L, cx, 8, cell_size=h, want_src=True) for h in (0.0, 0.02, 0.08, 0.5)]
    for v, _, _ in runs:
        assert_close(v, ref.values, X, "voids")
    for v, s, _ in runs[1:]:
        for k in range(4):
            assert np.array_equal(v[k].view(np.uint32), runs[0][0][k].view(np.uint32))
            assert np.array_equal(s[k], runs[0][1][k])


def test_batched_filtration_equals_each_cloud_alone():
    """Clouds sharing one batched flood launch get exactly their alone results."""
    ops = _ops()
    dev = _dev()
    jobs, alone = [], []
    for i, (gen, n, n_l, m) in enumerate([(data.torus_cloud, 30_000, 60, 8), (data.sphere_cloud, 5_000, 40, 6),
                                          (data.shape_mix_cloud, 50_000, 120, 8), (data.sphere_cloud, 800, 12, 5)]):
        X = gen(n, seed=100 + i)
        idx, _ = oracle.fps(X, n_l, 0)
        L = X[idx]
        cx = delaunay_complex(L)
        Xd = torch.from_numpy(X).to(dev)
        grid = ops.build_grid(Xd)
        dcx = ops.to_device(cx, dev)
        Ld = torch.from_numpy(L).to(dev)
        v, s = ops.filtration(grid, Ld, dcx, m)
        alone.append(([a.cpu().numpy() for a in v], [b.cpu().numpy() for b in s]))
        jobs.append((grid, Ld, dcx, m))
        if i == 0:
            ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
            assert_close(alone[0][0], ref.values, X, "batch member")
    outs = ops.filtration_batch(jobs, want_src=True)
    for (v, s), (va, sa) in zip(outs, alone):
        for k in range(4):
            assert np.array_equal(v[k].cpu().numpy().view(np.uint32), va[k].view(np.uint32))
            assert np.array_equal(s[k].cpu().numpy(), sa[k])


def test_src_points_at_attaining_sample():
    X = data.torus_cloud(8000, seed=5)
    m = 6
    L, cx, ref = _case(X, 40, m, method="kdtree")
    vals, src, _ = gpu_flood(X, L, cx, m)
    ind = oracle.flood.KDIndex(X)
    for k in (1, 2, 3):
        d = src[k][:, 0] >> 28
        rows = src[k][:, 0] & ((1 << 28) - 1)
        ok = d >= 1
        assert np.all(d <= k)
        for dim in range(1, k + 1):
            sel = np.nonzero(ok & (d == dim))[0]
            if sel.size == 0:
                continue
            comps = oracle.interior_compositions(m, dim)[src[k][sel, 1]]
            V = L[cx.simplices[dim][rows[sel]]].astype(np.float64)
            P = np.einsum("nj,njd->nd", comps / m, V)
            dist, _ = ind.query(P)
            assert np.max(np.abs(dist - vals[k][sel])) <= TOL * _diam(X)


def test_invalid_inputs_raise():
    ops = _ops()
    X = data.sphere_cloud(2000, seed=2)
    idx, _ = oracle.fps(X, 20, 0)
    L = X[idx].copy()
    cx = delaunay_complex(L)
    Xd = torch.from_numpy(X).to(_dev())
    grid = ops.build_grid(Xd)
    dcx = ops.to_device(cx, _dev())
    Lnan = L.copy()
    Lnan[2, 1] = np.nan
    with pytest.raises(FloodError) as e:
        ops.filtration(grid, torch.from_numpy(Lnan).to(_dev()), dcx, 6)
    assert e.value.name == "FLOOD_EINVAL"
    bad = ops.to_device(cx, _dev())
    bad.simplices[2][0, 1] = 10_000
    with pytest.raises(FloodError) as e:
        ops.filtration(grid, torch.from_numpy(L).to(_dev()), bad, 6)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError):
        ops.filtration(grid, torch.from_numpy(L).to(_dev()), dcx, 0)
    Y = X.copy()
    Y[3, 0] = np.inf
    with pytest.raises(FloodError):
        ops.build_grid(torch.from_numpy(Y).to(_dev()))
    grid.close()


def test_empty_dimensions():
    X = data.sphere_cloud(3000, seed=4)
    idx, _ = oracle.fps(X, 10, 0)
    L = X[idx]
    full = delaunay_complex(L)
    edges_only = complex_from_simplices([full.simplices[1]], 10)
    ref = oracle.flood_values(X, L, edges_only.simplices, 6)
    vals, _, _ = gpu_flood(X, L, edges_only, 6)
    assert_close(vals, ref.values, X, "edges only")


# ----------------------------------------------------------------------------- backward

def test_backward_matches_oracle_gradient():
    ops = _ops()
    X = data.jitter(data.torus_cloud(3000, seed=81), amp=1e-6, seed=82)
    m = 6
    idx, _ = oracle.fps(X, 30, 0)
    L = X[idx].copy()
    cx = delaunay_complex(L)
    gamma = data.upstream_gradients(cx.counts, seed=83)
    res = oracle.flood_values(X, L, cx.simplices, m, method="brute")
    dX_ref, dL_ref = oracle.analytic_gradient(X, L, cx.simplices, m, gamma, result=res)
    dev = _dev()
    Xd = torch.from_numpy(X).to(dev).requires_grad_(True)
    Ld = torch.from_numpy(L).to(dev).requires_grad_(True)
    grid = ops.build_grid(Xd.detach())
    vals = ops.flood_values(Xd, Ld, grid, ops.to_device(cx, dev), m)
    loss = sum((v * torch.from_numpy(g).to(dev)).sum() for v, g in zip(vals, gamma))
    loss.backward()
    gX, gL = Xd.grad.cpu().numpy(), Ld.grad.cpu().numpy()
    scale = max(1.0, np.abs(dX_ref).max(), np.abs(dL_ref).max())
    assert np.max(np.abs(gX - dX_ref)) <= 1e-3 * scale
    assert np.max(np.abs(gL - dL_ref)) <= 1e-3 * scale
    assert np.array_equal(np.abs(gX).sum(1) > 0, np.abs(dX_ref).sum(1) > 0)


def test_backward_matches_central_differences():
    ops = _ops()
    X = data.jitter(data.torus_cloud(2000, seed=91), amp=1e-6, seed=92)
    m = 5
    idx, _ = oracle.fps(X, 20, 0)
    L = X[idx].copy()
    cx = delaunay_complex(L)
    gamma = data.upstream_gradients(cx.counts, seed=93)
    dev = _dev()
    Xd = torch.from_numpy(X).to(dev).requires_grad_(True)
    Ld = torch.from_numpy(L).to(dev).requires_grad_(True)
    grid = ops.build_grid(Xd.detach())
    vals = ops.flood_values(Xd, Ld, grid, ops.to_device(cx, dev), m)
    sum((v * torch.from_numpy(g).to(dev)).sum() for v, g in zip(vals, gamma)).backward()
    gX, gL = Xd.grad.cpu().numpy(), Ld.grad.cpu().numpy()
    rng = np.random.default_rng(0)
    nz = np.argwhere(np.abs(gX) > 0)
    probes = [("X", int(a), int(b)) for a, b in nz[rng.choice(len(nz), 30, replace=False)]]
    probes += [("L", int(a), int(rng.integers(3))) for a in rng.choice(L.shape[0], 15, replace=False)]
    fd, kink, _ = oracle.finite_difference(X, L, cx.simplices, m, gamma, probes, h=1e-4, method="brute")
    an = np.array([gX[r, c] if w == "X" else gL[r, c] for (w, r, c) in probes])
    ok = ~kink
    assert ok.sum() >= 25
    assert np.allclose(an[ok], fd[ok], rtol=1e-2, atol=1e-3)
