"""Persistence diagrams end to end: GPU flood values against oracle flood values (§2).

The flood filtration exists to be reduced to persistence diagrams (§2, §4.1),
so a value error that is tiny per simplex but reorders the filtration would
show here and nowhere else. For each workload both valued complexes are
reduced by the oracle's Z/2 column reduction (host, FP64):

* if the two filtration orders (value, dimension, lexicographic vertex ids)
  are identical, the pairings must be identical, simplex for simplex, and
  every diagram point then moves by at most max |f_gpu - f_oracle|;
* otherwise the bottleneck distance between the diagrams of each dimension
  must be at most max |f_gpu - f_oracle| (the stability of persistence
  diagrams under perturbations of the filtration function, §2).

Both values must also meet the usual bar, 1e-5 x the bounding-box diagonal.
Landmarks are the oracle's FPS picks (never the CUDA path's).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.persistence import filtration_order
from paper_2509_22432_b300 import data, delaunay_complex

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _diam(X):
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _gpu_values(X, L, cx, m, cell):
    from paper_2509_22432_b300 import ops
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    grid = ops.build_grid(Xd, cell)
    vals, _ = ops.filtration(grid, torch.from_numpy(np.ascontiguousarray(L)).cuda(), ops.to_device(cx, Xd.device),
                             m, want_src=False)
    out = [v.cpu().numpy().astype(np.float64) for v in vals]
    grid.close()
    return out


def compare_diagrams(cx, v_gpu, v_orc, max_dim=2):
    """Returns 'same order' or 'bottleneck' (which rule decided) after asserting it."""
    dmax = max(float(np.max(np.abs(a - b), initial=0.0)) for a, b in zip(v_gpu, v_orc))
    o_gpu, _ = filtration_order(cx.simplices, v_gpu)
    o_orc, _ = filtration_order(cx.simplices, v_orc)
    if o_gpu == o_orc:
        p_gpu, e_gpu = oracle.persistence_pairs(cx.simplices, cx.facets, v_gpu)
        p_orc, e_orc = oracle.persistence_pairs(cx.simplices, cx.facets, v_orc)
        assert p_gpu == p_orc
        assert e_gpu == e_orc
        for b, d in p_gpu:
            assert abs(v_gpu[b[0]][b[1]] - v_orc[b[0]][b[1]]) <= dmax
            assert abs(v_gpu[d[0]][d[1]] - v_orc[d[0]][d[1]]) <= dmax
        return "same order"
    d_gpu = oracle.diagrams(cx.simplices, cx.facets, v_gpu, max_dim=max_dim)
    d_orc = oracle.diagrams(cx.simplices, cx.facets, v_orc, max_dim=max_dim)
    for k in range(max_dim + 1):
        assert oracle.bottleneck_within(d_gpu[k], d_orc[k], dmax * (1 + 1e-9) + 1e-15), k
    return "bottleneck"


def _case(X, n_l, m, cell_factor=0.5):
    idx, key = oracle.fps(X, n_l, 0)
    L = X[idx]
    cx = delaunay_complex(L)
    v_gpu = _gpu_values(X, L, cx, m, cell_factor * float(np.sqrt(key[-1])))
    v_orc = oracle.flood_values(X, L, cx.simplices, m, method="kdtree").values
    tol = TOL * _diam(X)
    for k in range(4):
        assert np.max(np.abs(v_gpu[k] - v_orc[k]), initial=0.0) <= tol, k
    return cx, v_gpu, v_orc


def test_diagrams_sphere_10k_every_simplex():
    """10,000 points on a noisy sphere, 128 landmarks, m = 6: dgm_0..dgm_2 of the whole complex."""
    X = data.sphere_cloud(10_000, seed=1)
    cx, v_gpu, v_orc = _case(X, 128, 6)
    compare_diagrams(cx, v_gpu, v_orc)
    # the sphere's H2 class is present in both (one long-lived dgm_2 point)
    d = oracle.diagrams(cx.simplices, cx.facets, v_gpu)
    assert np.max(d[2][:, 1] - d[2][:, 0], initial=0.0) > 0.5


@pytest.mark.slow
def test_diagrams_shape_mix_300k_m12():
    """300,000 points of the 8-surface mix, 1,000 landmarks, m = 12."""
    X = data.shape_mix_cloud(300_000, seed=33)
    cx, v_gpu, v_orc = _case(X, 1000, 12)
    compare_diagrams(cx, v_gpu, v_orc)


def _golden(workload):
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_fps_golden.py")
    spec = importlib.util.spec_from_file_location("make_fps_golden", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod, mod.read(workload)


@pytest.mark.slow
def test_diagrams_torus_1m_bench_workload():
    """The benchmark workload: 1,000,000-point torus, the oracle's 2,000 FPS picks (stored), m = 10."""
    mod, g = _golden("torus-1M")
    X = data.torus_cloud(1_000_000, seed=2)
    assert mod.cloud_sha256(X) == g["x_sha256"], "the generator drew a different cloud on this host"
    L = X[g["idx"]]
    cx = delaunay_complex(L)
    last = oracle.fps_key(L[:-1], L[-1]).min()
    v_gpu = _gpu_values(X, L, cx, 10, 0.5 * float(np.sqrt(last)))
    v_orc = oracle.flood_values(X, L, cx.simplices, 10, method="kdtree").values
    tol = TOL * _diam(X)
    for k in range(4):
        assert np.max(np.abs(v_gpu[k] - v_orc[k]), initial=0.0) <= tol, k
    compare_diagrams(cx, v_gpu, v_orc)
