"""Host-side pieces of bench.py, on the CPU: the step statistics, the tiled
host timing, the I/O report's Theorem-1 figures and the reference arm's line."""
import math
import os
import sys

import numpy as np
import pytest

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


def test_tiled_sample_times_the_tiled_product():
    import torch
    import bench
    rng = np.random.default_rng(1)
    A = torch.tensor(rng.uniform(-1, 1, (300, 64)))
    B = torch.tensor(rng.uniform(-1, 1, (64, 200)))
    fl, dt, r, used, a, b = bench.tiled_sample(A, B, 0.01)
    assert (a, b) == (180, 181)         # FindSeqSchedule at S = 32768
    assert r == 200 and used >= 1 and dt > 0
    assert math.isclose(fl, 2.0 * r * r * 64 / dt)


def test_host_info_fields():
    import bench
    h = bench.host_info()
    assert h["nproc"] == os.cpu_count() and h["machine"]


def test_io_report_bounds_follow_theorem1():
    """The bench's I/O block: Theorem 1 at the chip's fast memory (L2 + every SM's
    shared and tensor memory, in input words) and the compulsory bytes, for the
    plain and the emulated dtypes, against the oracle's closed form."""
    import types
    import bench
    from oracle import bounds
    m = n = k = 4096
    plan = types.SimpleNamespace(fast_words=123904.0, io_words=1.0e9,
                                 bound_words=bounds.thm1(m, n, k, 123904.0))
    l2, sms, smem = 126 * 2 ** 20, 152, 233472
    for dt, w_in, w_out, passes in [("bf16", 2, 4, 1), ("f64", 8, 8, 1),
                                    ("f64_emu_bf16", 2, 8, 21), ("f32_emu_tf32", 4, 4, 2)]:
        out = bench.io_report(m, n, k, dt, plan, 5e9, l2, sms, smem)
        s_chip = (l2 + sms * (smem + 262144)) / w_in
        assert out["S_chip_words"] == s_chip
        thm1 = passes * 2.0 * m * n * k / math.sqrt(s_chip) + m * n
        assert out["theorem1_bytes_at_S_chip"] == pytest.approx(thm1 * w_in)
        assert out["operand_passes_per_call"] == passes
        assert out["ratio_dram_vs_theorem1_chip"] == pytest.approx(5e9 / (thm1 * w_in))
        slices = 6 if dt == "f64_emu_bf16" else (2 if dt == "f32_emu_tf32" else 1)
        assert out["compulsory_bytes"] == w_in * slices * (m * k + k * n) + w_out * m * n


def test_reference_arm_line(monkeypatch, capsys):
    """`bench.py --impl reference`: one JSON line with the oracle's own timing as
    value, cpu_baseline and e2e (no host-device bytes); non-zero ranks print
    nothing."""
    import json
    import types
    import bench
    monkeypatch.setattr(bench, "oracle_sample", lambda m, n, k, t, **kw: (2.0e9, 0.5, 64))
    args = types.SimpleNamespace(workload="512", dtype="f64", steps=2, warmup=1, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["unit"] == "TFLOP/s"
    assert line["value"] == pytest.approx(2.0e-3)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["higher_is_better"] is True and line["metric"] == bench.METRIC
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_grouped_oracle_sample_counts_the_problems_it_ran():
    # a short budget covers the first problems; their flop are 2 m n k each (or
    # the 64 x 64 corner of a problem above 3e8 multiply-adds)
    import bench
    import cosma_inputs as ci
    dims = ci.grouped_dims(512, seed=1)
    flop, dt, count = bench.grouped_oracle_sample(dims, 0.3)
    assert 1 <= count <= len(dims) and dt > 0
    want = 0.0
    for m, n, k in dims[:count]:
        m, n, k = int(m), int(n), int(k)
        want += 2.0 * (64 * 64 if m * n * k > 3e8 else m * n) * k
    assert flop == want
    assert bench.grouped_oracle_sample(dims[:2], 60.0)[2] == 2


def test_reference_arm_grouped_workload(monkeypatch, capsys):
    import json
    import types
    import bench
    monkeypatch.setattr(bench, "grouped_oracle_sample", lambda dims, t: (3.0e9, 1.5, 40))
    args = types.SimpleNamespace(workload="grouped512", dtype="bf16", steps=2, warmup=1, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["value"] == pytest.approx(2.0e-3)
    assert line["ms_per_step"] == pytest.approx(1500.0)
    assert line["config"]["workload"].startswith(bench.GROUPED_WORKLOAD)
    assert "first 40 problems" in line["cpu_baseline"]["sample"]
