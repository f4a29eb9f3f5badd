"""Parity at the full workload sizes (B300; slow).

* 5,000,000-point union of 8 surfaces, 10,000 FPS landmarks, m = 12: the CUDA
  picks equal the oracle's picks (stored by tests/golden/make_fps_golden.py,
  which runs only the oracle), index for index, and the keys bit for bit;
  flood values of the complex of those landmarks (the workload's own
  complex) on thousands of sampled simplices per dimension against the FP64
  k-d tree oracle.
* 1,000,000-point noisy torus, 2,000 landmarks: the same check of the picks.
* 1,000,000-point jittered torus, 2,000 landmarks, m = 10, upstream
  gradients ~ N(0,1): backward against the oracle's analytic subgradient and
  central differences (h = 1e-5) on 1,000 coordinates.
"""
import hashlib
import importlib.util
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5
HERE = os.path.dirname(os.path.abspath(__file__))


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _golden(workload, X):
    """The oracle's stored picks for this workload; the cloud must be the one they were computed on."""
    spec = importlib.util.spec_from_file_location("make_fps_golden", os.path.join(HERE, "golden",
                                                                                 "make_fps_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    g = mod.read(workload)
    assert mod.cloud_sha256(X) == g["x_sha256"], "the seeded generator drew a different cloud on this host"
    return g


def _check_picks(X, n_l, workload):
    g = _golden(workload, X)
    idx, key = _ops().fps(torch.from_numpy(X).cuda(), n_l, 0)
    idx, key = idx.cpu().numpy(), key.cpu().numpy()
    assert np.array_equal(idx, g["idx"]), int(np.argmax(idx != g["idx"]))
    assert hashlib.sha256(np.ascontiguousarray(key, np.float32).tobytes()).hexdigest() == g["key_sha256"]
    return g


@pytest.fixture(scope="module")
def shapes5m():
    X = data.shape_mix_cloud()
    g = _check_picks(X, 10_000, "shapes-5M")
    return X, g["idx"], np.uint32(int(g["last_key_hex"], 16)).view(np.float32)


def test_fps_5m_equals_the_oracle_picks(shapes5m):
    X, idx, _ = shapes5m
    assert idx[0] == 0 and len(set(idx.tolist())) == 10_000


def test_fps_1m_torus_equals_the_oracle_picks():
    _check_picks(data.torus_cloud(1_000_000, seed=2), 2000, "torus-1M")


def test_flood_5m_on_the_fps_complex(shapes5m):
    """The workload's own complex: Delaunay of the 10,000 oracle (= CUDA) FPS landmarks, m = 12."""
    X, idx, last_key = shapes5m
    ops = _ops()
    m = 12
    L = X[idx]
    cx = delaunay_complex(L)
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd, 0.5 * float(np.sqrt(last_key)))
    vals, src = ops.filtration(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device), m)
    vals = [v.cpu().numpy() for v in vals]
    grid.close()
    rng = np.random.default_rng(1)
    subset = [np.arange(L.shape[0])] + [rng.choice(cx.counts[k], min(cx.counts[k], 4000), replace=False)
                                        for k in (1, 2, 3)]
    ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree", subset=subset)
    tol = TOL * _diam(X)
    for k in range(4):
        err = np.max(np.abs(vals[k][ref.simplex_ids[k]].astype(np.float64) - ref.values[k]))
        assert err <= tol, (k, err, tol)
    # monotone filtration over the whole complex
    for k in range(1, 4):
        lower = vals[0][cx.simplices[1]] if k == 1 else vals[k - 1][cx.facets[k]]
        assert np.all(lower.max(axis=1) <= vals[k])


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
    # A few attaining (sample, point) pairs may differ where FP32 and FP64 see a
    # near-tie; measured on this workload: 6 of 20,192 non-zero rows of dX and
    # 7 of 2,000 rows of dL. The bars allow about twice that and no more.
    bad_X = np.any(np.abs(gX - dX) > 1e-3 * scale, axis=1)
    bad_L = np.any(np.abs(gL - dL) > 1e-3 * scale, axis=1)
    n_rows = np.count_nonzero(np.abs(dX).sum(1))
    assert bad_X.sum() <= 0.0006 * max(1, n_rows), (int(bad_X.sum()), n_rows)
    assert bad_L.sum() <= 0.008 * L.shape[0], int(bad_L.sum())


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
    # counted, not compared (measured: 57 of 1,000); every other probe agreed
    assert ok.sum() >= 900, ok.sum()
    close = np.isclose(an[ok], fd[ok], rtol=1e-2, atol=1e-3)
    assert close.mean() >= 0.995, (close.mean(), ok.sum(), int((~close).sum()))
