"""Persistence pairs on the device (flood_persistence) against the oracle's host reduction (§2).

Both sides reduce the same filtration: the GPU flood values of the same
complex, ordered by (value, dimension, lexicographic vertex ids). The pairing
of a filtration does not depend on how the reduction is carried out, so the
device's pairs and essential classes must equal the oracle's exactly
(integers: bit-exact), and so must the diagrams built from them. Cases: the
noisy sphere (every simplex), the 8-surface mix at m = 12, the benchmark
torus with its stored oracle landmarks, and a complex whose faces were built
on the device (rows not in lexicographic order).
"""
import importlib.util
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _gpu_values(Xd, L, dcx, m, cell):
    from paper_2509_22432_b300 import ops
    grid = ops.build_grid(Xd, cell)
    vals, _ = ops.filtration(grid, L, dcx, m, want_src=False)
    grid.close()
    return vals


def _host_cx(dcx):
    """Host simplex lists and facets of a device complex (for the oracle)."""
    class H:
        pass
    h = H()
    h.simplices = [t.cpu().numpy() for t in dcx.simplices]
    h.facets = [t.cpu().numpy() for t in dcx.facets]
    h.counts = dcx.counts
    return h


def assert_same_pairing(cx_host, dcx, vals):
    from paper_2509_22432_b300 import ops
    ph = ops.persistence(dcx, vals)
    v = [x.cpu().numpy().astype(np.float64) for x in vals]
    pairs, essential = oracle.persistence_pairs(cx_host.simplices, cx_host.facets, v)
    for k in range(3):
        want = np.array(sorted((b[1], d[1]) for b, d in pairs if b[0] == k), dtype=np.int64).reshape(-1, 2)
        got = ph["pairs"][k].cpu().numpy().astype(np.int64)
        got = got[np.lexsort((got[:, 1], got[:, 0]))]
        assert np.array_equal(got, want), k
    for k in range(4):
        want = np.array(sorted(e[1] for e in essential if e[0] == k), dtype=np.int64)
        assert np.array_equal(np.sort(ph["essential"][k].cpu().numpy()), want), k
    dg = ops.diagrams_from_pairs(ph, vals)
    ref = oracle.diagrams(cx_host.simplices, cx_host.facets, v, max_dim=2)
    for k in range(3):
        assert np.array_equal(dg[k], ref[k]), k
    return ph


def _case(X, n_l, m):
    from paper_2509_22432_b300 import ops
    idx, key = oracle.fps(X, n_l, 0)
    L = X[idx]
    cx = delaunay_complex(L)
    Xd = torch.from_numpy(X).cuda()
    dcx = ops.to_device(cx, Xd.device)
    vals = _gpu_values(Xd, torch.from_numpy(L).cuda(), dcx, m, 0.5 * float(np.sqrt(key[-1])))
    return cx, dcx, vals, L


def test_device_pairing_sphere_10k():
    cx, dcx, vals, _ = _case(data.sphere_cloud(10_000, seed=1), 128, 6)
    ph = assert_same_pairing(cx, dcx, vals)
    assert ph["essential"][0].numel() == 1 and all(ph["essential"][k].numel() == 0 for k in (1, 2, 3))


def test_device_pairing_with_device_built_faces():
    """Faces from flood_complex_faces: rows in the device's order, not lexicographic."""
    from paper_2509_22432_b300 import ops
    X = data.shape_mix_cloud(40_000, seed=63)
    idx, key = oracle.fps(X, 400, 0)
    L = X[idx]
    tets = torch.from_numpy(np.ascontiguousarray(delaunay_complex(L).simplices[3], dtype=np.int32)).cuda()
    dcx = ops.complex_faces(tets, L.shape[0])
    vals = _gpu_values(torch.from_numpy(X).cuda(), torch.from_numpy(L).cuda(), dcx, 8, 0.5 * float(np.sqrt(key[-1])))
    assert_same_pairing(_host_cx(dcx), dcx, vals)


@pytest.mark.slow
def test_device_pairing_shape_mix_300k_m12():
    cx, dcx, vals, _ = _case(data.shape_mix_cloud(300_000, seed=33), 1000, 12)
    assert_same_pairing(cx, dcx, vals)


@pytest.mark.slow
def test_device_pairing_torus_1m_bench_workload():
    from paper_2509_22432_b300 import ops
    spec = importlib.util.spec_from_file_location("make_fps_golden", os.path.join(HERE, "golden",
                                                                                 "make_fps_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    g = mod.read("torus-1M")
    X = data.torus_cloud(1_000_000, seed=2)
    assert mod.cloud_sha256(X) == g["x_sha256"]
    L = X[g["idx"]]
    cx = delaunay_complex(L)
    Xd = torch.from_numpy(X).cuda()
    dcx = ops.to_device(cx, Xd.device)
    last = np.uint32(int(g["last_key_hex"], 16)).view(np.float32)
    vals = _gpu_values(Xd, torch.from_numpy(L).cuda(), dcx, 10, 0.5 * float(np.sqrt(last)))
    ph = assert_same_pairing(cx, dcx, vals)
    # the whole Delaunay complex triangulates a ball: one component is the only class that never dies
    assert [ph["essential"][k].numel() for k in range(4)] == [1, 0, 0, 0]
    # the torus's two loops and its void are long-lived points of dgm_1 and dgm_2
    dg = ops.diagrams_from_pairs(ph, vals)
    assert np.sum(dg[1][:, 1] - dg[1][:, 0] > 0.1) >= 2 and np.sum(dg[2][:, 1] - dg[2][:, 0] > 0.1) >= 1


def test_device_pairing_rejects_bad_input():
    from paper_2509_22432_b300 import ops
    from paper_2509_22432_b300._lib import FloodError
    cx, dcx, vals, _ = _case(data.sphere_cloud(2000, seed=64), 40, 4)
    bad = [v.clone() for v in vals]
    bad[2][3] = float("nan")
    with pytest.raises(FloodError) as e:
        ops.persistence(dcx, bad)
    assert e.value.name == "FLOOD_EINVAL"
