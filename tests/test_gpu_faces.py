"""Device face enumeration (flood_complex_faces) against the definition, and the
flood values over the device-built complex against those over the host-built one.

Rows of the device complex are in first-producer order, so they are compared
as sets (unique), and the incidence is checked row by row (valid)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu


def _ops():
    from paper_2509_22432_b300 import ops
    return ops


def _tets(n_points, seed):
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((n_points, 3))
    return np.ascontiguousarray(np.sort(Delaunay(P).simplices, axis=1).astype(np.int32)), n_points


def _device(tets, nv):
    return _ops().complex_faces(torch.from_numpy(tets).cuda(), nv)


def check_complex(dcx, tets):
    tri_ref, edg_ref = oracle.faces_by_definition(tets)
    s = [t.cpu().numpy() for t in dcx.simplices]
    f = [t.cpu().numpy() for t in dcx.facets]
    assert np.array_equal(s[3], tets)
    for k, ref in ((2, tri_ref), (1, edg_ref)):
        assert s[k].shape == ref.shape, k
        assert np.all(np.diff(s[k], axis=1) > 0)                          # ascending ids
        assert sorted(map(tuple, s[k].tolist())) == list(map(tuple, ref.tolist()))   # each face once
    for k in (2, 3):
        assert np.array_equal(f[k], oracle.facet_rows(s[k], s[k - 1])), k
    assert np.array_equal(f[1], s[1][:, ::-1])


@pytest.mark.parametrize("n,seed", [(5, 1), (40, 2), (2000, 3), (30000, 4)])
def test_faces_match_the_definition(n, seed):
    tets, nv = _tets(n, seed)
    check_complex(_device(tets, nv), tets)


def test_faces_are_deterministic_and_handle_shared_and_duplicate_rows():
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4], [0, 1, 2, 3], [5, 6, 7, 8]], dtype=np.int32)
    a, b = _device(tets, 9), _device(tets, 9)
    for x, y in zip(a.simplices + a.facets, b.simplices + b.facets):
        assert torch.equal(x, y)
    check_complex(a, tets)
    assert a.counts == [9, 15, 11, 4]


def test_faces_empty_and_invalid():
    ops = _ops()
    e = ops.complex_faces(torch.zeros((0, 4), dtype=torch.int32, device="cuda"), 3)
    assert e.counts == [3, 0, 0, 0]
    for bad in ([[0, 2, 1, 3]], [[0, 1, 2, 9]], [[-1, 0, 1, 2]], [[0, 1, 1, 2]]):
        with pytest.raises(FloodError) as err:
            ops.complex_faces(torch.tensor(bad, dtype=torch.int32, device="cuda"), 5)
        assert err.value.name == "FLOOD_EINVAL"
    ok = ops.complex_faces(torch.tensor([[0, 1, 2, 3]], dtype=torch.int32, device="cuda"), 4)
    assert ok.counts == [4, 6, 4, 1]


def test_flood_values_over_the_device_complex_equal_the_host_complex():
    """Values depend only on (simplex, sample, point): bit for bit equal per simplex."""
    ops = _ops()
    X = data.torus_cloud(100_000, seed=5)
    idx, _ = oracle.fps(X, 300, 0)
    L = X[idx]
    host = delaunay_complex(L)
    dev = ops.complex_faces(torch.from_numpy(np.ascontiguousarray(host.simplices[3], dtype=np.int32)).cuda(),
                            L.shape[0])
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd)
    Ld = torch.from_numpy(L).cuda()
    hv, _ = ops.filtration(grid, Ld, ops.to_device(host, Xd.device), 8)
    dv, _ = ops.filtration(grid, Ld, dev, 8)
    grid.close()
    for k in (1, 2, 3):
        hmap = {tuple(r): v for r, v in zip(host.simplices[k].tolist(), hv[k].cpu().numpy().view(np.uint32))}
        rows = dev.simplices[k].cpu().numpy().tolist()
        got = dv[k].cpu().numpy().view(np.uint32)
        assert len(rows) == len(hmap)
        assert all(hmap[tuple(r)] == g for r, g in zip(rows, got)), k
