"""Pins for the step-by-step oracle of the emulated-FP64 method (oracle/ozaki.py)."""
import numpy as np
import pytest

from oracle import gemm as og
from oracle import ozaki


def _rand(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, shape)


def test_digits_reassemble_and_stay_balanced():
    for beta, s in [(8, 6), (7, 7), (6, 3)]:
        L = beta * s - 1
        for F in [0, 1, -1, 2 ** L - 1, -(2 ** L - 1), 123456789 % 2 ** L, -(987654321 % 2 ** L)]:
            d = ozaki._digits(F, beta, s)
            assert sum(x << (beta * (s - 1 - q)) for q, x in enumerate(d)) == F
            assert all(-(1 << (beta - 1)) <= x < (1 << (beta - 1)) for x in d[1:])
            assert abs(d[0]) <= (1 << (beta - 1))


def test_integer_inputs_are_exact():
    rng = np.random.default_rng(1)
    A = rng.integers(-8, 9, (7, 11)).astype(float)
    B = rng.integers(-8, 9, (11, 5)).astype(float)
    for beta, s in [(8, 6), (8, 3), (7, 2)]:
        assert np.array_equal(ozaki.gemm(A, B, beta, s), A @ B)


def test_many_bits_give_the_correctly_rounded_product():
    # beta s = 64 bits > 53: truncation is below half an ulp of every entry
    A, B = _rand((6, 9), 2), _rand((9, 4), 3)
    C = ozaki.gemm(A, B, 8, 8)
    ref = og.gemm(A, B, "dot2")  # Dot2: as if computed in twice the precision
    assert np.all(np.abs(C - ref) <= 2.0 ** -52 * np.abs(ref) + 1e-300)


@pytest.mark.parametrize("beta,s", [(8, 3), (7, 2), (8, 6)])
def test_truncation_error_within_bound_and_visible(beta, s):
    A, B = _rand((8, 40), 4), _rand((40, 6), 5)
    C = ozaki.gemm(A, B, beta, s)
    ref = og.gemm(A, B, "dot2")
    bound = ozaki.truncation_bound(A, B, beta, s) + 2.0 ** -53 * np.abs(ref)
    assert np.all(np.abs(C - ref) <= bound)
    if beta * s < 40:  # the truncated triangle really changes the result
        assert np.max(np.abs(C - ref)) > 2.0 ** -(beta * s + 8)


def test_zero_rows_and_columns():
    A, B = _rand((3, 5), 6), _rand((5, 4), 7)
    A[1, :] = 0.0
    B[:, 2] = 0.0
    C = ozaki.gemm(A, B, 8, 4)
    assert not C[1, :].any() and not C[:, 2].any()
