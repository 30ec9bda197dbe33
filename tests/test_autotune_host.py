"""Host logic of the autotuner (no GPU): the random shape families, the
candidate filter, the resumable record file, the feature rows and the initial
weights of the cost model."""
import json
import math

import numpy as np
import pytest

from oracle import mlp as om


@pytest.fixture(scope="module")
def tune():
    from paper_1908_09606_gb300 import build as b
    b.build()
    from paper_1908_09606_gb300 import autotune, cosma
    cosma.load()
    return autotune


def test_random_shapes_are_log_uniform_capped_and_reproducible(tune):
    cosma = tune.cosma
    shapes = tune.random_shapes(400, seed=7, lo=256, hi=65536, cap_bytes=16e9)
    assert len(shapes) == 400 and shapes == tune.random_shapes(400, seed=7)
    assert shapes != tune.random_shapes(400, seed=8)
    d = np.array(shapes, dtype=np.float64)
    assert d.min() >= 256 and d.max() <= 65536
    win, wout = tune.DTYPE_BYTES[cosma.COSMA_BF16]
    m, n, k = d.T
    assert np.all(np.maximum.reduce([m * k * win, k * n * win, m * n * wout]) <= 16e9)
    # log2 of each dimension is uniform on [8, 16] before the cap removes large
    # shapes: its mean sits a little below 12 and its spread near 8 / sqrt(12)
    lg = np.log2(d)
    assert 10.5 < lg.mean() < 12.2
    assert 1.8 < lg.std() < 2.6
    small = tune.random_shapes(50, seed=7, max_flops=1e12)
    assert all(2.0 * a * b * c <= 1e12 for a, b, c in small)


def test_candidates_respect_the_workspace_cap(tune):
    cosma = tune.cosma
    for shape in [(4096, 4096, 4096), (300, 260, 70), (1024, 1024, 1 << 18)]:
        every = tune.candidates(*shape, cosma.COSMA_BF16, float("inf"))
        assert every and all(0 <= c < cosma.COSMA_MLP_OUT for c, _ in every)
        cap = min(p.workspace_bytes for _, p in every)
        kept = tune.candidates(*shape, cosma.COSMA_BF16, cap)
        assert kept and all(p.workspace_bytes <= cap for _, p in kept)
        assert {c for c, _ in kept} == {c for c, p in every if p.workspace_bytes <= cap}


def test_record_file_resumes_and_skips_blank_lines(tune, tmp_path):
    path = tmp_path / "rows.jsonl"
    assert tune._load_rows(str(path)) == []
    rows = [{"m": 256, "n": 512, "k": 1024, "dtype": 2, "cand": c, "seconds": 1e-4 * (c + 1)}
            for c in range(3)]
    path.write_text(json.dumps(rows[0]) + "\n\n" + json.dumps(rows[1]) + "\n" +
                    json.dumps(rows[2]) + "\n")
    assert tune._load_rows(str(path)) == rows


def test_feature_rows_and_log_time_targets(tune):
    rows = [{"m": 256, "n": 65536, "k": 1000, "dtype": 2, "cand": 4, "seconds": 0.25},
            {"m": 4096, "n": 4096, "k": 4096, "dtype": 2, "cand": 0, "seconds": 3e-3}]
    X, cand, y = tune.features(rows)
    assert X.shape == (2, tune.cosma.COSMA_MLP_IN) and X.dtype == np.float32
    for r, x in zip(rows, X):
        assert np.allclose(x, om.features(r["m"], r["n"], r["k"], r["dtype"]), rtol=1e-6,
                           atol=1e-7)
    assert cand.tolist() == [4, 0]
    assert y[0] == -2.0 and y[1] == pytest.approx(math.log2(3e-3))


def test_initial_weights_he_uniform_zero_biases(tune):
    cosma = tune.cosma
    p = tune.init_params(3)
    assert p.dtype == np.float32 and p.size == cosma.COSMA_MLP_PARAMS
    assert np.array_equal(p, tune.init_params(3)) and not np.array_equal(p, tune.init_params(4))
    W1, b1, W2, b2, W3, b3 = om.unpack(p.astype(np.float64))
    for W, fan_in in [(W1, cosma.COSMA_MLP_IN), (W2, cosma.COSMA_MLP_HIDDEN),
                      (W3, cosma.COSMA_MLP_HIDDEN)]:
        lim = math.sqrt(6.0 / fan_in)
        assert np.abs(W).max() <= lim and np.abs(W).max() > 0.8 * lim
        assert abs(W.mean()) < 0.1 * lim
    assert not b1.any() and not b2.any() and not b3.any()


def test_destandardized_network_predicts_log2_seconds(tune):
    """Folding the target standardisation into the last layer gives the same
    network with outputs sigma * y + mu (checked with the FP64 oracle MLP)."""
    p = tune.init_params(5)
    rng = np.random.default_rng(2)
    p = p + rng.normal(0.0, 0.05, p.size).astype(np.float32)  # nonzero biases too
    X = rng.uniform(0.5, 1.0, (6, tune.cosma.COSMA_MLP_IN))
    mu, sigma = -7.25, 2.5
    q = tune.destandardize(p, mu, sigma)
    Y, _ = om.forward(p.astype(np.float64), X)
    Yq, _ = om.forward(q.astype(np.float64), X)
    assert np.allclose(Yq, sigma * Y + mu, rtol=1e-5, atol=1e-5)
    # hidden layers untouched
    n_hidden = q.size - tune.cosma.COSMA_MLP_OUT * (tune.cosma.COSMA_MLP_HIDDEN + 1)
    assert np.array_equal(q[:n_hidden], p[:n_hidden])


def test_calibration_shapes_are_a_fixed_fifth(tune):
    shapes = tune.random_shapes(2000, seed=11)
    flags = [tune.is_calibration(m, n, k, 2) for m, n, k in shapes]
    assert flags == [tune.is_calibration(m, n, k, 2) for m, n, k in shapes]
    assert 0.15 < np.mean(flags) < 0.25
    assert tune.MARGINS[0] > 0 and math.isinf(tune.MARGINS[-1])
    assert list(tune.MARGINS) == sorted(tune.MARGINS)


def test_parser_modes(tune):
    """Collection, training on stored timings, partial re-collection and
    evaluation of installed weights are separate, explicit modes."""
    ap = tune.parser()
    a = ap.parse_args(["--out", "x"])
    assert not a.no_collect and a.collect_dtypes is None and a.eval_only is None
    a = ap.parse_args(["--out", "x", "--collect-dtypes", "f64_emu_bf16", "--epochs", "10"])
    assert a.collect_dtypes == "f64_emu_bf16" and a.epochs == 10
    a = ap.parse_args(["--out", "x", "--eval-only", "w.npy", "--dtypes", "bf16"])
    assert a.eval_only == "w.npy" and a.dtypes == "bf16"
    assert set(a.dtypes.split(",")) <= set(tune.cosma.DTYPES)
