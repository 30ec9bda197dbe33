"""Pins for the oracle GEMM (oracle/gemm.py): closed forms, exact integer
arithmetic, exact rational arithmetic, the classical error bound, Freivalds."""
from fractions import Fraction

import numpy as np
import pytest

import cosma_inputs as ci
from oracle import gemm as og


def _exact_int_product(A, B):
    Ai = [[int(v) for v in row] for row in A]
    Bi = [[int(v) for v in row] for row in B]
    m, k, n = len(Ai), len(Bi), len(Bi[0])
    return np.array([[sum(Ai[i][t] * Bi[t][j] for t in range(k)) for j in range(n)]
                     for i in range(m)], dtype=np.float64)


@pytest.mark.parametrize("method", ["naive", "dot2"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 5, 3), (13, 29, 64), (33, 17, 129)])
def test_integer_inputs_exact(method, shape):
    m, n, k = shape
    A = ci.matrix(m, k, "integer", "f64", seed=1, stream=0)
    B = ci.matrix(k, n, "integer", "f64", seed=1, stream=1)
    C = og.gemm(A, B, method)
    assert np.array_equal(C, _exact_int_product(A, B))


@pytest.mark.parametrize("method", ["naive", "dot2"])
def test_identity(method):
    B = ci.matrix(24, 31, "uniform", "f64", seed=2, stream=1)
    assert np.array_equal(og.gemm(np.eye(24), B, method), B)
    A = ci.matrix(19, 31, "uniform", "f64", seed=2, stream=0)
    assert np.array_equal(og.gemm(A, np.eye(31), method), A)


@pytest.mark.parametrize("method", ["naive", "dot2"])
def test_diagonal_scales_rows(method):
    d = ci.entries(np.arange(20), np.zeros(20), 1, "uniform", "f64", seed=3, stream=0)
    B = ci.matrix(20, 27, "uniform", "f64", seed=3, stream=1)
    C = og.gemm(np.diag(d), B, method)
    assert np.array_equal(C, d[:, None] * B)


@pytest.mark.parametrize("method", ["naive", "dot2"])
def test_rank1(method):
    # A = u 1^T, B = 1 v^T  ->  C = k u v^T (integer u, v: exact)
    m, n, k = 9, 11, 37
    u = ci.entries(np.arange(m), np.zeros(m), 1, "integer", "f64", seed=4, stream=0)
    v = ci.entries(np.arange(n), np.zeros(n), 1, "integer", "f64", seed=4, stream=1)
    A = np.repeat(u[:, None], k, axis=1)
    B = np.repeat(v[None, :], k, axis=0)
    assert np.array_equal(og.gemm(A, B, method), k * np.outer(u, v))


def test_dot2_against_exact_rationals():
    m, n, k = 4, 5, 40
    A = ci.matrix(m, k, "loguniform", "f64", seed=5, stream=0)
    B = ci.matrix(k, n, "loguniform", "f64", seed=5, stream=1)
    C = og.gemm(A, B, "dot2")
    u = 2.0 ** -53
    for i in range(m):
        for j in range(n):
            exact = sum(Fraction(A[i, t]) * Fraction(B[t, j]) for t in range(k))
            absdot = sum(abs(Fraction(A[i, t]) * Fraction(B[t, j])) for t in range(k))
            # Ogita-Rump-Oishi Prop. 5.5: |res - x^T y| <= u|x^T y| + gamma_n^2 |x|^T|y|
            gam = k * u / (1 - k * u)
            bound = u * abs(exact) + Fraction(gam * gam) * absdot
            assert abs(Fraction(C[i, j]) - exact) <= bound


def test_naive_within_gamma_k():
    m, n, k = 6, 7, 200
    A = ci.matrix(m, k, "loguniform", "f64", seed=6, stream=0)
    B = ci.matrix(k, n, "uniform", "f64", seed=6, stream=1)
    C = og.gemm(A, B, "naive")
    u = 2.0 ** -53
    gam = k * u / (1 - k * u)
    for i in range(m):
        for j in range(n):
            exact = sum(Fraction(A[i, t]) * Fraction(B[t, j]) for t in range(k))
            absdot = sum(abs(Fraction(A[i, t]) * Fraction(B[t, j])) for t in range(k))
            assert abs(Fraction(C[i, j]) - exact) <= Fraction(gam) * absdot


def test_naive_matches_order_of_definition():
    # the naive chain in t = 0..k-1 is reproduced exactly by a Python loop
    A = ci.matrix(3, 50, "uniform", "f64", seed=7, stream=0)
    B = ci.matrix(50, 4, "uniform", "f64", seed=7, stream=1)
    C = og.gemm(A, B, "naive")
    for i in range(3):
        for j in range(4):
            c = 0.0
            for t in range(50):
                c = c + float(A[i, t]) * float(B[t, j])
            assert C[i, j] == c


def test_dot2_pairs_match_full():
    m, n, k = 10, 12, 77
    A = ci.matrix(m, k, "uniform", "f64", seed=8, stream=0)
    B = ci.matrix(k, n, "uniform", "f64", seed=8, stream=1)
    C = og.gemm(A, B, "dot2")
    ii = np.array([0, 3, 9, 9])
    jj = np.array([0, 11, 5, 0])
    out = og.dot2_pairs(A[ii], B[:, jj].T)
    assert np.array_equal(out, C[ii, jj])


def test_freivalds_accepts_correct_and_flags_planted_error():
    m, n, k = 40, 30, 50
    A = ci.matrix(m, k, "uniform", "f64", seed=9, stream=0)
    B = ci.matrix(k, n, "uniform", "f64", seed=9, stream=1)
    C = og.gemm(A, B, "dot2")
    x = ci.entries(np.arange(n), np.zeros(n), 1, "uniform", "f64", seed=9, stream=2)
    r, scale = og.freivalds(A, B, C, x)
    assert np.all(np.abs(r) <= 4 * 2.0 ** -53 * scale + 1e-300)
    Cbad = C.copy()
    Cbad[17, 4] += 1e-9
    r2, scale2 = og.freivalds(A, B, Cbad, x)
    assert np.abs(r2[17]) > 1e3 * 2.0 ** -53 * scale2[17]


def test_empty_and_k0():
    assert og.gemm(np.zeros((0, 3)), np.zeros((3, 4))).shape == (0, 4)
    C = og.gemm(np.zeros((3, 0)), np.zeros((0, 4)))
    assert C.shape == (3, 4) and not C.any()


# ---- gemm_ex: alpha op(A) op(B) + beta C0 -------------------------------------

def _int_loops(Astore, Bstore, C0, alpha, beta, ta, tb):
    """Brute force with Python integers, indexing the stored arrays directly."""
    m = len(Astore[0]) if ta else len(Astore)
    k = len(Astore) if ta else len(Astore[0])
    n = len(Bstore) if tb else len(Bstore[0])
    out = [[0] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            acc = 0
            for t in range(k):
                a = Astore[t][i] if ta else Astore[i][t]
                b = Bstore[j][t] if tb else Bstore[t][j]
                acc += int(a) * int(b)
            out[i][j] = alpha * acc + beta * int(C0[i][j])
    return out


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
def test_gemm_ex_integer_all_transposes(ta, tb):
    rng = np.random.default_rng(11)
    m, n, k = 5, 7, 6
    Ast = rng.integers(-8, 9, (k, m) if ta else (m, k))
    Bst = rng.integers(-8, 9, (n, k) if tb else (k, n))
    C0 = rng.integers(-50, 51, (m, n))
    for alpha, beta in [(1, 0), (3, -2), (-1, 1), (0, 5)]:
        got = og.gemm_ex(Ast, Bst, C0, alpha, beta, ta, tb)
        want = np.array(_int_loops(Ast.tolist(), Bst.tolist(), C0.tolist(), alpha, beta, ta, tb),
                        dtype=np.float64)
        assert np.array_equal(got, want), (alpha, beta)


def test_gemm_ex_alpha_zero_and_beta_zero():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((4, 3))
    B = rng.standard_normal((3, 5))
    C0 = rng.standard_normal((4, 5))
    assert np.array_equal(og.gemm_ex(A, B, C0, 0.0, 0.625), 0.625 * C0)
    A[0, 0] = np.nan  # not read when alpha == 0
    assert np.array_equal(og.gemm_ex(A, B, C0, 0.0, 2.0), 2.0 * C0)
    C0[:] = np.nan    # not read when beta == 0
    A[0, 0] = 1.0
    assert np.isfinite(og.gemm_ex(A, B, C0, 1.5, 0.0)).all()


def test_gemm_ex_identity_closed_form():
    rng = np.random.default_rng(13)
    Bst = rng.standard_normal((6, 4))   # stored n x k: op(B) = Bst^T (k = 4, n = 6)
    C0 = rng.standard_normal((4, 6))
    got = og.gemm_ex(np.eye(4), Bst, C0, 2.0, -1.0, False, True)
    assert np.array_equal(got, 2.0 * Bst.T + (-1.0) * C0)


# ---- zgemm: complex alpha op(A) op(B) + beta C0 -----------------------------------

@pytest.mark.parametrize("op_a", [0, 1, 2])
@pytest.mark.parametrize("op_b", [0, 1, 2])
def test_zgemm_gaussian_integers_all_ops(op_a, op_b):
    rng = np.random.default_rng(21)
    m, n, k = 4, 5, 3
    def mk(r, c):
        return rng.integers(-6, 7, (r, c)) + 1j * rng.integers(-6, 7, (r, c))
    Ast = mk(k, m) if op_a else mk(m, k)
    Bst = mk(n, k) if op_b else mk(k, n)
    C0 = mk(m, n)
    alpha, beta = 2 - 1j, -1 + 3j
    got = og.zgemm(Ast, Bst, C0, alpha, beta, op_a, op_b)
    def el(X, o, i, j):  # element (i, j) of op(X) from the stored X
        if o == 0:
            return complex(X[i][j])
        v = complex(X[j][i])
        return v.conjugate() if o == 2 else v
    for i in range(m):
        for j in range(n):
            acc = sum(el(Ast, op_a, i, t) * el(Bst, op_b, t, j) for t in range(k))
            assert got[i, j] == alpha * acc + beta * complex(C0[i][j])


def test_zgemm_alpha_zero_beta_zero():
    rng = np.random.default_rng(22)
    A = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    B = rng.standard_normal((4, 2)) + 1j * rng.standard_normal((4, 2))
    C0 = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    assert np.array_equal(og.zgemm(A, B, C0, 0, 1j), 1j * C0)
    C0[:] = np.nan
    assert np.isfinite(og.zgemm(A, B, C0, 1, 0)).all()


@pytest.mark.parametrize("shape,ab", [((37, 53, 29), (8, 8)), ((100, 64, 300), (17, 33)),
                                      ((5, 7, 1), (2, 3)), ((64, 96, 0), (16, 16))])
def test_tiled_equals_naive_bit_for_bit(shape, ab):
    """The tiled schedule of Sec. 5.2 forms every entry by the same chain
    t = 0..k-1 as the naive loop, so the two agree exactly, ragged tiles included."""
    m, n, k = shape
    rng = np.random.default_rng(7)
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    C, used = og.tiled(A, B, *ab)
    assert used >= 1
    assert np.array_equal(C, og.gemm(A, B, "naive"))
    C1, used1 = og.tiled(A, B, *ab, threads=1)
    assert used1 == 1 and np.array_equal(C1, C)
