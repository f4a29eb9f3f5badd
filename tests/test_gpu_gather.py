"""flood_gather_rows: L = X[idx] bit for bit (the landmark rows of FPS's picks, §3)."""
import numpy as np
import pytest
import torch

from paper_2509_22432_b300 import data
from paper_2509_22432_b300._lib import FloodError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,n,n_idx", [(3, 100_000, 2000), (5, 7, 7), (2, 1, 3), (4, 50_000, 0)])
def test_gather_rows_is_bitwise_indexing(d, n, n_idx):
    from paper_2509_22432_b300 import ops
    rng = np.random.default_rng(n + d)
    X = rng.standard_normal((n, d)).astype(np.float32)
    idx = rng.integers(0, n, n_idx).astype(np.int64)
    L = ops.gather_rows(torch.from_numpy(X).cuda(), torch.from_numpy(idx).cuda())
    assert L.shape == (n_idx, d)
    assert np.array_equal(L.cpu().numpy().view(np.uint32), X[idx].view(np.uint32))


def test_gather_rows_of_fps_picks_and_bad_index():
    from paper_2509_22432_b300 import ops
    X = data.sphere_cloud(5000, seed=91)
    Xd = torch.from_numpy(X).cuda()
    idx, _ = ops.fps(Xd, 64, 0)
    assert torch.equal(ops.gather_rows(Xd, idx), Xd[idx])
    bad = idx.clone()
    bad[5] = 5000
    ops.gather_rows(Xd, bad, sync=False)
    with pytest.raises(FloodError) as e:
        ops.check()
    assert e.value.name == "FLOOD_EINVAL"
    assert torch.equal(ops.gather_rows(Xd, idx), Xd[idx])   # and the stream still works
