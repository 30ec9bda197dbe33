"""The shared seeded input generator (host half): known-answer vectors and the
stated value mapping."""
import os

import numpy as np
import pytest

import cosma_inputs as ci

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_philox_known_answers(row):
    out = ci.philox4x32_10(*row[:6])
    assert [int(x) for x in out] == row[6:]


def test_uniform_f64_range_and_grid():
    x = ci.matrix(64, 96, "uniform", "f64", seed=0)
    assert x.shape == (64, 96)
    assert x.min() >= -1.0 and x.max() < 1.0
    # values are multiples of 2^-52
    assert np.all(np.ldexp(x + 1.0, 52) == np.floor(np.ldexp(x + 1.0, 52)))
    assert abs(x.mean()) < 0.05 and abs(x.var() - 1.0 / 3.0) < 0.03


def test_uniform_f32_exact():
    x = ci.matrix(32, 32, "uniform", "f32", seed=3)
    assert x.dtype == np.float32
    assert np.all(np.ldexp(x.astype(np.float64) + 1.0, 23) % 1.0 == 0.0)


def test_integer_range():
    x = ci.matrix(100, 100, "integer", "f64", seed=5)
    assert set(np.unique(x)) <= set(range(-8, 9))
    assert len(np.unique(x)) == 17


def test_loguniform_span():
    x = ci.matrix(200, 200, "loguniform", "f64", seed=7)
    ax = np.abs(x)
    assert ax.min() >= 2.0 ** -27 and ax.max() < 2.0 ** 27
    assert ax.min() < 1e-7 and ax.max() > 1e7
    assert (x < 0).any() and (x > 0).any()


def test_rows_cols_entries_agree_with_matrix():
    m, n = 37, 53
    A = ci.matrix(m, n, "uniform", "f64", seed=11, stream=ci.STREAM_A)
    r = ci.rows([0, 5, 36], n, "uniform", "f64", seed=11, stream=ci.STREAM_A)
    assert np.array_equal(r, A[[0, 5, 36]])
    c = ci.cols([0, 52, 7], m, n, "uniform", "f64", seed=11, stream=ci.STREAM_A)
    assert np.array_equal(c, A[:, [0, 52, 7]].T)
    e = ci.entries([3, 9], [4, 50], n, "uniform", "f64", seed=11, stream=ci.STREAM_A)
    assert np.array_equal(e, A[[3, 9], [4, 50]])


def test_streams_and_seeds_differ():
    a = ci.matrix(8, 8, seed=0, stream=0)
    b = ci.matrix(8, 8, seed=0, stream=1)
    c = ci.matrix(8, 8, seed=1, stream=0)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_bf16_is_rounded_f32():
    torch = pytest.importorskip("torch")
    x32 = ci.matrix(16, 16, "uniform", "f32", seed=2)
    xb = ci.matrix(16, 16, "uniform", "bf16", seed=2)
    assert xb.dtype == torch.bfloat16
    assert torch.equal(xb, torch.from_numpy(x32).to(torch.bfloat16))
