"""Serving loop (flood_serve_*): continuous batching, admission, failure isolation.

The GPU tests check that every cloud's result from the batched server equals
the one-cloud path on that cloud alone, bit for bit (values and landmarks),
that a request whose triangulation fails fails alone, and that admission
respects the device-memory budget. The CPU tests cover configuration and
capacity checks, which need no GPU.
"""
import numpy as np
import pytest

from paper_2509_22432_b300 import data, delaunay_complex
from paper_2509_22432_b300._lib import FloodError


def _clouds(n_clouds=12, seed=7):
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(2000), np.log(60000), n_clouds)).astype(int)
    return [data.shape_mix_cloud(int(n), n_shapes=1 + i % 3, seed=1000 + i) for i, n in enumerate(sizes)]


def _alone(X, n_l, m, cell_factor=0.5):
    import torch
    from paper_2509_22432_b300 import ops
    Xd = torch.from_numpy(X).cuda()
    idx, key = ops.fps(Xd, n_l, 0)
    idx_h = idx.cpu().numpy()
    L = X[idx_h]
    cx = delaunay_complex(L)
    grid = ops.build_grid(Xd, cell_factor * float(np.sqrt(key[-1].item())))
    vals, _ = ops.filtration(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device), m, want_src=False)
    grid.close()
    return idx_h, [v.cpu().numpy() for v in vals]


@pytest.mark.gpu
def test_batched_server_results_equal_one_cloud_path():
    from paper_2509_22432_b300.serve import Server
    clouds = _clouds()
    m = 8
    with Server(max_inflight=6, max_batch=8, gpu_workers=3, triangulation_workers=3, device_faces=False) as srv:
        tickets = [srv.submit(X, 0, m) for X in clouds]
        results = [srv.result(t, timeout_ms=120_000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(clouds) and st["failed"] == 0
    assert st["batches"] >= 1
    for X, res in zip(clouds, results):
        assert res["status"] == 0
        n_l = max(4, int(round(0.02 * X.shape[0])))
        idx, vals = _alone(X, n_l, m)
        assert np.array_equal(res["landmarks"], idx)
        for k in range(4):
            assert np.array_equal(res["values"][k].view(np.uint32), vals[k].view(np.uint32)), k


@pytest.mark.gpu
def test_device_faces_server_equals_one_cloud_path_per_simplex():
    """Tetrahedra-only callbacks: faces built on the device; each simplex's value is
    bit for bit the one-cloud path's (rows matched by their vertex ids)."""
    from paper_2509_22432_b300.serve import Server
    clouds = _clouds(8, seed=9)
    m = 8
    with Server(max_inflight=6, max_batch=8, gpu_workers=3, triangulation_workers=3, device_faces=True) as srv:
        results = [srv.result(t, timeout_ms=120_000) for t in [srv.submit(X, 0, m) for X in clouds]]
        st = srv.stats()
    assert st["completed"] == len(clouds) and st["failed"] == 0
    for X, res in zip(clouds, results):
        assert res["status"] == 0
        n_l = max(4, int(round(0.02 * X.shape[0])))
        idx, vals = _alone(X, n_l, m)
        assert np.array_equal(res["landmarks"], idx)
        host = delaunay_complex(X[idx])
        assert np.array_equal(res["values"][0].view(np.uint32), vals[0].view(np.uint32))
        for k in (1, 2, 3):
            rows = res["simplices"][k]
            assert rows.shape == host.simplices[k].shape, k
            ref = {tuple(r): v for r, v in zip(host.simplices[k].tolist(), vals[k].view(np.uint32))}
            got = res["values"][k].view(np.uint32)
            assert all(ref[tuple(r)] == g for r, g in zip(rows.tolist(), got)), k


@pytest.mark.gpu
def test_precomputed_tetrahedra_give_the_same_results_without_qhull():
    """tets_cache (the bench's no-Delaunay arm): the landmarks' tetrahedra looked up by their bytes;
    every cloud hits the cache and its values are bit for bit those of the Qhull run."""
    import torch
    from paper_2509_22432_b300 import ops
    from paper_2509_22432_b300.serve import Server, delaunay_tets
    clouds = _clouds(6, seed=11)
    m = 8
    cache = {}
    for X in clouds:
        n_l = max(4, int(np.floor(float(np.float32(0.02)) * X.shape[0] + 0.5)))  # the server's rounding
        idx, _ = ops.fps(torch.from_numpy(X).cuda(), n_l, 0)
        L = np.ascontiguousarray(X[idx.cpu().numpy()], dtype=np.float32)
        cache[L.tobytes()] = delaunay_tets(L)
    out = []
    for tc in (None, cache):
        with Server(max_inflight=4, max_batch=4, gpu_workers=2, triangulation_workers=2, device_faces=True,
                    tets_cache=tc) as srv:
            out.append([srv.result(t, timeout_ms=120_000) for t in [srv.submit(X, 0, m) for X in clouds]])
            if tc is not None:
                assert srv.cache_misses == 0
    for a, b in zip(*out):
        assert a["status"] == 0 and b["status"] == 0
        assert np.array_equal(a["landmarks"], b["landmarks"])
        for k in range(4):
            assert np.array_equal(a["values"][k].view(np.uint32), b["values"][k].view(np.uint32)), k


@pytest.mark.gpu
def test_failed_triangulation_fails_only_its_request():
    from paper_2509_22432_b300.serve import Server

    def tri(L):
        if L.shape[0] == 77:
            raise RuntimeError("triangulation failed")
        return delaunay_complex(L)

    clouds = [data.sphere_cloud(5000, seed=s) for s in range(5)]
    with Server(max_inflight=4, max_batch=4, triangulate=tri) as srv:
        t = [srv.submit(X, 77 if i == 2 else 60, 6) for i, X in enumerate(clouds)]
        res = [srv.result(x, timeout_ms=60_000) for x in t]
        st = srv.stats()
    assert [r["status"] != 0 for r in res] == [False, False, True, False, False]
    assert st["failed"] == 1 and st["completed"] == 4


@pytest.mark.gpu
def test_admission_respects_device_budget():
    from paper_2509_22432_b300.serve import Server
    clouds = [data.torus_cloud(40000, seed=s) for s in range(6)]
    budget = 3 * (64 * 40000 + 20000 * 800 + (8 << 20))   # about three clouds at once
    with Server(device_budget_bytes=budget, max_inflight=16, max_batch=16) as srv:
        t = [srv.submit(X, 0, 8) for X in clouds]
        res = [srv.result(x, timeout_ms=60_000) for x in t]
        st = srv.stats()
        with pytest.raises(FloodError) as e:
            srv.submit(data.torus_cloud(2_000_000, seed=9), 0, 8)
        assert e.value.name == "FLOOD_ECAPACITY"
    assert all(r["status"] == 0 for r in res)
    assert 0 < st["device_bytes_peak"] <= budget


def test_server_rejects_invalid_configuration():
    from paper_2509_22432_b300.serve import Server
    with pytest.raises(FloodError) as e:
        Server(max_batch=0)
    assert e.value.name == "FLOOD_EINVAL"
    with pytest.raises(FloodError):
        Server(device_budget_bytes=0)
    with pytest.raises(FloodError):
        Server(cell_factor=-1.0)


def test_oversized_cloud_is_rejected_at_submit():
    """Admission capacity is checked on the host before any device work."""
    from paper_2509_22432_b300.serve import Server
    srv = Server(device_budget_bytes=64 << 20, max_inflight=2, max_batch=2)
    try:
        with pytest.raises(FloodError) as e:
            srv.submit(np.zeros((2_000_000, 3), np.float32), 0, 8)
        assert e.value.name == "FLOOD_ECAPACITY"
        with pytest.raises(FloodError):
            srv.submit(np.zeros((3, 3), np.float32), 0, 8)     # too few points
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()
