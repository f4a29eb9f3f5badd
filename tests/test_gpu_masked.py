"""The paper's masked full-grid evaluation (flood_filtration_masked, §4.2 / App. A.1)
against the FP64 oracle and against the pruned path: same values within 1e-5 x
the bounding-box diagonal of X; far more pairs evaluated."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _setup(X, n_l):
    idx, key = oracle.fps(X, n_l, 0)
    L = X[idx]
    return L, delaunay_complex(L), key


def test_masked_equals_oracle_sphere_10k():
    ops = _ops()
    X = data.sphere_cloud()
    L, cx, _ = _setup(X, 128)
    ref = oracle.flood_values(X, L, cx.simplices, 6, method="brute")
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd)
    vals, pairs = ops.filtration_masked(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device), 6)
    grid.close()
    tol = TOL * _diam(X)
    for k in range(4):
        err = np.max(np.abs(vals[k].cpu().numpy().astype(np.float64) - ref.values[k]))
        assert err <= tol, (k, err)
    assert pairs > 0


@pytest.mark.parametrize("m", [3, 10])
def test_masked_equals_pruned_path(m):
    ops = _ops()
    X = data.torus_cloud(40000, seed=3)
    L, cx, key = _setup(X, 80)
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd, 0.5 * float(np.sqrt(key[-1])))
    Ld = torch.from_numpy(L).cuda()
    dcx = ops.to_device(cx, Xd.device)
    pv, _ = ops.filtration(grid, Ld, dcx, m, want_src=False)
    pruned_pairs = sum(ops.last_filtration_stats()["pairs"])
    mv, pairs = ops.filtration_masked(grid, Ld, dcx, m)
    grid.close()
    tol = TOL * _diam(X)
    for k in range(4):
        err = float((pv[k].double() - mv[k].double()).abs().max()) if pv[k].numel() else 0.0
        assert err <= tol, (m, k, err)
    assert pairs > pruned_pairs


def test_masked_rejects_landmarks_off_X_and_large_grids():
    ops = _ops()
    X = data.sphere_cloud(3000, seed=5)
    L, cx, _ = _setup(X, 20)
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd)
    dcx = ops.to_device(cx, Xd.device)
    with pytest.raises(FloodError) as e:
        ops.filtration_masked(grid, torch.from_numpy(L + np.float32(1e-3)).cuda(), dcx, 4)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError) as e:
        ops.filtration_masked(grid, torch.from_numpy(L).cuda(), dcx, 19)   # C(22, 3) = 1540 samples
    assert e.value.name == "FLOOD_EINVAL"
    vals, _ = ops.filtration_masked(grid, torch.from_numpy(L).cuda(), dcx, 4)
    assert torch.isfinite(vals[3]).all()
    grid.close()
