"""Host-side pieces of bench.py, on the CPU: the step statistics and the
Listing-1 host timing (its product equals the naive oracle's)."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_step_stats_median_min_and_t_interval():
    import bench
    st = bench.step_stats([1.0, 1.1, 0.9, 1.05, 0.95])
    assert st["median_ms"] == 1.0 and st["min_ms"] == 0.9
    assert math.isclose(st["mean_ms"], 1.0)
    sd = np.std([1.0, 1.1, 0.9, 1.05, 0.95], ddof=1)
    half = 2.776 * sd / math.sqrt(5)     # Student t, 4 degrees of freedom
    assert np.allclose(st["ci95_ms"], [1.0 - half, 1.0 + half])
    assert "ci95_ms" not in bench.step_stats([3.0])


def test_listing1_sample_times_the_tiled_product():
    import torch
    import bench
    rng = np.random.default_rng(1)
    A = torch.tensor(rng.uniform(-1, 1, (300, 64)))
    B = torch.tensor(rng.uniform(-1, 1, (64, 200)))
    fl, dt, r, used, a, b = bench.listing1_sample(A, B, 0.01)
    assert (a, b) == (180, 181)         # FindSeqSchedule at S = 32768
    assert r == 200 and used >= 1 and dt > 0
    assert math.isclose(fl, 2.0 * r * r * 64 / dt)


def test_host_info_fields():
    import bench
    h = bench.host_info()
    assert h["nproc"] == os.cpu_count() and h["machine"]
