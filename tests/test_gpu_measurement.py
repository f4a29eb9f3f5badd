"""The measurement helpers the benchmark reports with.

* flood_masking_ball_counts: the size of the paper's masked candidate sets
  (Lemma 2 ball of every simplex), against the oracle's FP64 ball (§4.2);
  the FP32 ball test may classify points within rounding of the sphere
  either way (an edge's endpoints lie on it), so the count must lie between
  the oracle's counts for the ball shrunk and grown by 1e-5 relative.
* flood_fp32_peak_probe: a pure-FMA kernel; its rate must be a plausible
  FP32 rate for this GPU (the benchmark divides by it).
* flood_last_fps_stats: exchange rounds of the last FPS call (at most one
  round per pick, at least one per 32 picks).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.flood import ritter_ball
from paper_2509_22432_b300 import data, delaunay_complex

pytestmark = pytest.mark.gpu


def _oracle_ball_counts(X, L, simplices, rel):
    """Points strictly inside the ball shrunk by (1 - rel), and inside it grown by (1 + rel):
    an edge's own endpoints lie exactly on its ball, so rounding decides them either way."""
    X64 = np.asarray(X, np.float64)
    lo, hi = [0, 0, 0, 0], [0, 0, 0, 0]
    for k in (1, 2, 3):
        for row in np.asarray(simplices[k]):
            c, _, rho = ritter_ball(np.asarray(L, np.float64)[row])
            d2 = ((X64 - c) ** 2).sum(axis=1)
            lo[k] += int(np.count_nonzero(d2 < (rho * (1 - rel)) ** 2))
            hi[k] += int(np.count_nonzero(d2 <= (rho * (1 + rel)) ** 2))
    return lo, hi


def test_masking_ball_counts_match_the_oracle_ball():
    from paper_2509_22432_b300 import ops

    X = data.sphere_cloud(10_000, seed=1)
    idx, _ = oracle.fps(X, 128, 0)
    L = X[idx]
    cx = delaunay_complex(L)
    Xd = torch.from_numpy(X).cuda()
    grid = ops.build_grid(Xd, 0.0)
    got = ops.masking_ball_counts(grid, torch.from_numpy(L).cuda(), ops.to_device(cx, Xd.device))
    grid.close()
    lo, hi = _oracle_ball_counts(X, L, cx.simplices, 1e-5)
    assert got[0] == 0
    for k in (1, 2, 3):
        assert lo[k] > 0
        assert lo[k] <= got[k] <= hi[k], (k, lo[k], got[k], hi[k])


@pytest.mark.parametrize("packed", [False, True])
def test_fp32_peak_probe_rate_is_plausible(packed):
    from paper_2509_22432_b300 import ops

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ops.fp32_peak_probe(dev, packed, 1000)                      # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    flops = ops.fp32_peak_probe(dev, packed, 20_000)
    b.record(stream)
    b.synchronize()
    tflops = flops / (a.elapsed_time(b) * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal = sms * 128 * 2 * 2.032e9 / 1e12                    # FP32 lanes x 2 flops x top clock
    assert 0.2 * nominal < tflops < 2.2 * nominal, (tflops, nominal)


def test_fps_stats_count_exchange_rounds():
    from paper_2509_22432_b300 import ops

    X = data.torus_cloud(200_000, seed=9)
    ops.fps(torch.from_numpy(X).cuda(), 500, 0)
    st = ops.fps_stats()
    assert st["picks"] == 500
    assert (499 + 31) // 32 <= st["rounds"] <= 499
    assert st["blocks"] >= 1
