"""flood_fps_noalloc: the scratch-free FPS entry point for callers that cannot allocate.

Some callers cannot let a library allocate device memory (their own pool owns
the device, their loop forbids allocator calls after start-up, or their host
framework forbids it). flood_fps_noalloc serves them from a fixed array
compiled into the library. These tests call it through the C ABI twice in a
row, on different inputs, and require the same picks as flood_fps (indices
are integers, so the bar is exact equality). This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2509_22432_b300 import data
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu


def test_noalloc_fps_matches_fps_on_two_calls_in_a_row():
    from paper_2509_22432_b300 import ops

    dev = torch.device("cuda:0")
    cases = [(data.torus_cloud(1_000_000, seed=2), 300, 0), (data.sphere_cloud(70_001, seed=13), 257, 11)]
    for X, n_l, start in cases:
        Xd = torch.from_numpy(X).to(dev)
        idx_ref, key_ref = ops.fps(Xd, n_l, start)
        idx, key = ops.fps_noalloc(Xd, n_l, start)
        assert torch.equal(idx, idx_ref)
        assert np.array_equal(key.cpu().numpy().view(np.uint32), key_ref.cpu().numpy().view(np.uint32))


def test_noalloc_fps_at_its_maximum_size_against_fps_and_the_oracle():
    """Exactly 2^20 points, the documented maximum; the picks are also checked against the
    oracle (integers: exact equality). The library checks on every call that the pieces it
    carved from the fixed array add up to flood_fps_scratch_bytes, whose worst case over the
    launch widths (points streamed from memory) a CPU test compares with the array's size."""
    from paper_2509_22432_b300 import ops
    import oracle

    X = data.shape_mix_cloud(1 << 20, seed=21)
    Xd = torch.from_numpy(X).cuda()
    for _ in range(2):                                  # two calls in a row share the array
        idx, key = ops.fps_noalloc(Xd, 200, 0)
        idx_ref, key_ref = ops.fps(Xd, 200, 0)
        assert torch.equal(idx, idx_ref)
        assert np.array_equal(key.cpu().numpy().view(np.uint32), key_ref.cpu().numpy().view(np.uint32))
    ri, rk = oracle.fps(X, 200, 0)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), rk.view(np.uint32))


def test_noalloc_fps_rejects_more_points_than_its_fixed_maximum():
    from paper_2509_22432_b300 import ops

    X = torch.zeros(((1 << 20) + 1, 3), dtype=torch.float32, device="cuda:0")
    with pytest.raises(FloodError) as e:
        ops.fps_noalloc(X, 4, 0)
    assert e.value.name == "FLOOD_ECAPACITY"
