"""The asynchronous boundary: FPS, grid build and filtration enqueue and return.

* A whole step (FPS -> grid -> filtration) is enqueued while the stream is
  still busy with earlier work: the host calls return before that work ends,
  so none of them waits on the device.
* Device-side errors of asynchronous calls come back through flood_check, or
  through the next call on the same stream once the status has arrived; the
  error is reported once, and the calls after it work.
* Results of the asynchronous path are bitwise those of the synchronous one,
  and flood_grid_get_info waits for the device-built geometry.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data, delaunay_complex
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu


def _workload():
    from paper_2509_22432_b300 import ops
    X = data.torus_cloud(200_000, seed=61)
    Xd = torch.from_numpy(X).cuda()
    idx, key = ops.fps(Xd, 600, 0)
    cx = ops.to_device(delaunay_complex(X[idx.cpu().numpy()]), Xd.device)
    return X, Xd, idx, key, cx


def test_a_step_is_enqueued_without_waiting_on_the_device():
    from paper_2509_22432_b300 import ops
    X, Xd, idx0, key0, cx = _workload()
    cell = 0.5 * float(np.sqrt(key0[-1].item()))
    ref, _ = ops.filtration(ops.build_grid(Xd, cell), Xd[idx0], cx, 8, want_src=False)
    torch.cuda.synchronize()
    torch.cuda._sleep(int(4e8))                       # about 0.2 s of device time ahead of the step
    t0 = time.perf_counter()
    idx, key = ops.fps(Xd, 600, 0, sync=False)
    grid = ops.build_grid(Xd, cell, sync=False)
    vals, _ = ops.filtration(grid, Xd[idx], cx, 8, want_src=False, sync=False)
    host_s = time.perf_counter() - t0
    busy = torch.cuda.current_stream().query() is False
    ops.check()
    assert busy, "the stream finished before the calls returned: something waited on the device"
    assert host_s < 0.15, host_s
    assert torch.equal(idx, idx0)
    for a, b in zip(vals, ref):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    info = grid.info()
    assert info["n_cells"] == info["dims"][0] * info["dims"][1] * info["dims"][2]
    assert np.allclose(info["bbox_lo"], X.min(0)) and np.allclose(info["bbox_hi"], X.max(0))
    grid.close()


def test_device_errors_come_back_through_check_or_the_next_call():
    from paper_2509_22432_b300 import ops
    X = data.sphere_cloud(5000, seed=62)
    bad = X.copy()
    bad[77, 1] = np.nan
    Xd, Bd = torch.from_numpy(X).cuda(), torch.from_numpy(bad).cuda()
    # through flood_check
    ops.fps(Bd, 16, 0, sync=False)                    # arguments are fine: returns OK
    with pytest.raises(FloodError) as e:
        ops.check()
    assert e.value.name == "FLOOD_EINVAL"
    ops.check()                                       # reported once
    # through the next call, once the status has arrived
    g = ops.build_grid(Bd, 0.0, sync=False)
    torch.cuda.synchronize()
    with pytest.raises(FloodError) as e:
        ops.fps(Xd, 16, 0, sync=False)
    assert e.value.name == "FLOOD_EINVAL"
    g.close()
    idx, _ = ops.fps(Xd, 16, 0)                       # and the calls after it work
    assert np.array_equal(idx.cpu().numpy(), oracle.fps(X, 16, 0)[0])
