"""A device-side wait that runs out returns a status and leaves the context usable.

Every wait in libflood's kernels is bounded: a wait that gives up raises a
timeout flag, the kernel returns, and the call reports FLOOD_ETIMEOUT instead
of trapping or hanging. flood_fps_wait_test makes the FPS grid exchange wait
for one block that is never launched (nothing ever writes its slot), with a
short poll limit, so the wait of the first round runs out after about a
millisecond. The next ordinary calls in the same process must still be
correct (checked against the oracle).
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2509_22432_b300 import data

pytestmark = pytest.mark.gpu


def test_fps_exchange_wait_runs_out_cleanly_and_the_context_stays_usable():
    from paper_2509_22432_b300 import ops

    X = data.torus_cloud(20_000, seed=31)
    Xd = torch.from_numpy(X).cuda()
    for n_blocks in (2, 4):          # resident kernel: 4 x 7,168 points hold the cloud; 2 blocks stream it
        t0 = time.perf_counter()
        st = ops.fps_wait_test(Xd, 64, n_blocks=n_blocks, extra_blocks=1, poll_limit=2000)
        dt = time.perf_counter() - t0
        assert st == -4, st                          # FLOOD_ETIMEOUT
        assert dt < 5.0, dt                          # the bounded wait, not the default bound of seconds
    # the same process keeps working: ordinary FPS and a filtration-sized call afterwards
    idx, key = ops.fps(Xd, 64, 0)
    ri, rk = oracle.fps(X, 64, 0)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(key.cpu().numpy().view(np.uint32), rk.view(np.uint32))
    idx2, _ = ops.fps(Xd, 64, 0, n_blocks=4)
    assert np.array_equal(idx2.cpu().numpy(), ri)
    torch.cuda.synchronize()


def test_wait_test_rejects_shapes_without_an_exchange():
    from paper_2509_22432_b300 import ops

    Xd = torch.from_numpy(data.sphere_cloud(1000, seed=3)).cuda()
    assert ops.fps_wait_test(Xd, 8, n_blocks=1, extra_blocks=1, poll_limit=10) == -1     # one block: no exchange
    assert ops.fps_wait_test(Xd, 8, n_blocks=2, extra_blocks=200, poll_limit=10) == -1   # beyond the slot table
