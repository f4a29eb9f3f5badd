"""Parity at the full workload sizes (B300; slow).

* 5,000,000-point union of 8 surfaces, 10,000 FPS landmarks, m = 12: FPS
  checked by properties that hold at any size (every key equals the exact
  binary32 minimum over earlier landmarks, keys never increase, and no
  sampled point beats a pick or ties it with a lower index); flood values of
  sampled simplices, over 10,000 seeded random landmarks, against the FP64
  k-d tree oracle.
* 1,000,000-point jittered torus, 2,000 landmarks, m = 10, upstream
  gradients ~ N(0,1): backward against the oracle's analytic subgradient and
  central differences (h = 1e-5) on 1,000 coordinates.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def check_fps_properties(X, idx, key, n_sample=2000, seed=0):
    """Sampled verification of FPS picks (binary32 keys, lowest-index ties)."""
    n_l = idx.shape[0]
    assert len(set(idx.tolist())) == n_l
    L = X[idx]
    # key[j] = min_{l < j} kappa(x_{idx[j]}, l), exactly
    for j in range(1, n_l):
        k = oracle.fps_key(L[:j], L[j]).min()
        assert k == key[j], j
    assert np.all(np.diff(key[1:]) <= 0)
    # sampled points never beat (or tie with a lower index) the pick of any iteration
    rng = np.random.default_rng(seed)
    sample = rng.choice(X.shape[0], n_sample, replace=False)
    d = np.full(n_sample, np.inf, np.float32)
    for j in range(1, n_l):
        d = np.minimum(d, oracle.fps_key(X[sample], L[j - 1]))
        assert np.all(d <= key[j]), j
        tie = d == key[j]
        assert np.all(sample[tie] >= idx[j]), j


@pytest.fixture(scope="module")
def shapes5m():
    X = data.shape_mix_cloud()
    Xd = torch.from_numpy(X).cuda()
    idx, key = _ops().fps(Xd, 10_000, 0)
    return X, Xd, idx.cpu().numpy(), key.cpu().numpy()


def test_fps_5m_properties(shapes5m):
    X, _, idx, key = shapes5m
    assert idx[0] == 0
    check_fps_properties(X, idx, key)


def test_flood_5m_sampled_simplices(shapes5m):
    """Landmarks: 10,000 seeded random rows of X (oracle inputs never come from the CUDA path;
    the CUDA FPS picks are checked by properties above)."""
    X, Xd, _, key = shapes5m
    ops = _ops()
    m = 12
    idx = np.sort(np.random.default_rng(12).choice(X.shape[0], 10_000, replace=False))
    L = X[idx]
    cx = delaunay_complex(L)
    grid = ops.build_grid(Xd, 0.5 * float(np.sqrt(key[-1])))
    vals, src = ops.filtration(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device), m)
    vals = [v.cpu().numpy() for v in vals]
    grid.close()
    rng = np.random.default_rng(1)
    subset = [None] + [rng.choice(cx.counts[k], min(cx.counts[k], 1500), replace=False) for k in (1, 2, 3)]
    subset[0] = np.arange(L.shape[0])
    ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree", subset=subset)
    tol = TOL * _diam(X)
    for k in range(4):
        err = np.max(np.abs(vals[k][ref.simplex_ids[k]].astype(np.float64) - ref.values[k]))
        assert err <= tol, (k, err, tol)
    # monotone filtration over the whole complex
    for k in range(1, 4):
        assert np.all(vals[k - 1][cx.facets[k]].max(axis=1) <= vals[k])


@pytest.fixture(scope="module")
def torus_grad():
    X = data.jitter(data.torus_cloud(), amp=1e-6, seed=5)
    ops = _ops()
    Xd = torch.from_numpy(X).cuda()
    idx, key = oracle.fps(X, 2000, 0)          # the oracle's picks: its inputs never come from CUDA
    L = X[idx].copy()
    cx = delaunay_complex(L)
    gamma = data.upstream_gradients(cx.counts, seed=5)
    m = 10
    Xg = Xd.clone().requires_grad_(True)
    Lg = torch.from_numpy(L).cuda().requires_grad_(True)
    grid = ops.build_grid(Xd, 0.5 * float(np.sqrt(key[-1])))
    vals = ops.flood_values(Xg, Lg, grid, ops.to_device(cx, Xd.device), m)
    loss = sum((v * torch.from_numpy(g).cuda()).sum() for v, g in zip(vals, gamma))
    loss.backward()
    grid.close()
    return X, L, cx, gamma, m, Xg.grad.cpu().numpy(), Lg.grad.cpu().numpy()


def test_backward_1m_matches_analytic_subgradient(torus_grad):
    X, L, cx, gamma, m, gX, gL = torus_grad
    res = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
    dX, dL = oracle.analytic_gradient(X, L, cx.simplices, m, gamma, result=res)
    scale = max(1.0, np.abs(dX).max(), np.abs(dL).max())
    # a few attaining pairs may differ by FP32 near-ties; they must stay rare
    bad_X = np.any(np.abs(gX - dX) > 1e-3 * scale, axis=1)
    bad_L = np.any(np.abs(gL - dL) > 1e-3 * scale, axis=1)
    assert bad_X.sum() <= 0.001 * max(1, np.count_nonzero(np.abs(dX).sum(1)))
    assert bad_L.sum() <= 0.01 * L.shape[0]


def test_backward_1m_central_differences(torus_grad):
    X, L, cx, gamma, m, gX, gL = torus_grad
    rng = np.random.default_rng(5)
    nzX = np.argwhere(np.abs(gX) > 0)
    probes = [("X", int(a), int(b)) for a, b in nzX[rng.choice(len(nzX), 500, replace=False)]]
    probes += [("L", int(a), int(rng.integers(3))) for a in rng.choice(L.shape[0], 250, replace=False)]
    probes += [("X", int(a), int(rng.integers(3))) for a in rng.choice(X.shape[0], 250, replace=False)]
    # h = 1e-5: the central-difference error of f = |p* - x*| is O((h / f)^2),
    # and flood values here go down to ~5e-3 (1.5 point spacings)
    fd, kink, _ = oracle.finite_difference(X, L, cx.simplices, m, gamma, probes, h=1e-5, method="kdtree")
    an = np.array([gX[r, c] if w == "X" else gL[r, c] for (w, r, c) in probes])
    ok = ~kink
    # probes whose attaining (sample, point) pair changes within +-h are kinks:
    # counted, not compared
    assert ok.sum() >= 800, ok.sum()
    close = np.isclose(an[ok], fd[ok], rtol=1e-2, atol=1e-3)
    assert close.mean() >= 0.99, (close.mean(), ok.sum())
