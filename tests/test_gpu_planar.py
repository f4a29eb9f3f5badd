"""Ambient dimension 2 (the paper varies d; the circle example of App. C.3 is planar):
a planar cloud embedded at z = 0 runs through the same kernels. Every z difference
is exactly 0 in FP32, so keys, samples and distances are those of the plane."""
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


def test_planar_annulus_fps_values_and_gradient():
    ops = _ops()
    X = data.jitter(data.annulus_cloud(20000, seed=9), amp=1e-6, seed=10)
    X[:, 2] = 0.0
    Xd = torch.from_numpy(X).cuda()
    n_l, m = 200, 8
    idx, _ = ops.fps(Xd, n_l, 0)
    idx_o, _ = oracle.fps(X, n_l, 0)
    assert np.array_equal(idx.cpu().numpy(), idx_o)
    L = X[idx_o]
    cx = delaunay_complex(L, dim=2)
    ref = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
    grid = ops.build_grid(Xd)
    Xg = Xd.clone().requires_grad_(True)
    Lg = torch.from_numpy(L).cuda().requires_grad_(True)
    vals = ops.flood_values(Xg, Lg, grid, ops.to_device(cx, Xd.device), m)
    diam = float(np.linalg.norm(X.max(0).astype(np.float64) - X.min(0)))
    for k in range(3):
        err = np.max(np.abs(vals[k].detach().cpu().numpy().astype(np.float64) - ref.values[k]))
        assert err <= TOL * diam, (k, err)
    gamma = data.upstream_gradients(cx.counts, seed=11)
    sum((v * torch.from_numpy(g).cuda()).sum() for v, g in zip(vals, gamma)).backward()
    grid.close()
    dX, dL = oracle.analytic_gradient(X, L, cx.simplices, m, gamma, result=ref)
    gX, gL = Xg.grad.cpu().numpy(), Lg.grad.cpu().numpy()
    assert np.all(gX[:, 2] == 0) and np.all(gL[:, 2] == 0)       # no motion out of the plane
    scale = max(1.0, np.abs(dX).max(), np.abs(dL).max())
    bad = np.any(np.abs(gX - dX) > 1e-3 * scale, axis=1)
    assert bad.sum() <= 0.001 * max(1, np.count_nonzero(np.abs(dX).sum(1)))
