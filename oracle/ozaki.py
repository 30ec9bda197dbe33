"""Oracle of the emulated-FP64 method, step by step (test infrastructure only).

The emulation is not in the paper: it is the precision pattern the build adds
(FP64-accuracy products from small-integer slices on tensor cores), following
the error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
transformations of matrix multiplication by using fast routines of matrix
multiplication and its applications", Numer. Algorithms 59, 2012), in the form
this library documents:

  1. row scales: sigma_i is the exponent with 2^(sigma_i - 1) <= max_t |A_it|
     < 2^sigma_i (tau_j likewise for the columns of B); a zero row has no scale;
  2. each entry becomes the integer F = round(|x| 2^(L - sigma)), ties away
     from zero, with x's sign, L = beta s - 1;
  3. F is written as s balanced base-2^beta digits d_1 .. d_s (most significant
     first, d_q in [-2^(beta-1), 2^(beta-1)) for q >= 2);
  4. the level sums L_l = sum_{q + r = l} D^A_q D^B_r for l = 2 .. s + 1 (the
     truncated triangle q + r <= s + 1) are exact integers;
  5. C_ij = 2^(sigma_i + tau_j - 2L) sum_l 2^(beta (2s - l)) L_l[i, j], formed
     exactly and rounded once to FP64.

Everything is exact integer / rational arithmetic in Python (tiny sizes only),
so this is the method's own result with no rounding but the last.  Pins
(tests/test_oracle_ozaki.py): integer inputs give the exact product; with
beta s far beyond 53 bits the result is the correctly rounded exact product;
the truncation error obeys the bound derived from steps 2 and 4.
"""

from fractions import Fraction
import math

import numpy as np


def _scale_exponent(vals):
    mx = max((abs(float(v)) for v in vals), default=0.0)
    if mx == 0.0 or not math.isfinite(mx):
        return None
    return math.frexp(mx)[1]  # mx = f 2^e, 1/2 <= f < 1: 2^(e-1) <= mx < 2^e


def _scaled_integer(x, sigma, L):
    if sigma is None or x == 0.0:
        return 0
    y = abs(Fraction(float(x))) * Fraction(2) ** (L - sigma)
    F = math.floor(y + Fraction(1, 2))  # nearest, ties away from zero (y >= 0)
    return -F if x < 0 else F


def _digits(F, beta, s):
    base, half = 1 << beta, 1 << (beta - 1)
    d = [0] * s
    for q in range(s - 1, 0, -1):
        r = F % base  # Python: 0 <= r < base
        if r >= half:
            r -= base
        d[q] = r
        F = (F - r) >> beta
    d[0] = F
    return d


def slices(X, by_rows, beta, s):
    """Scale exponents and the s digit matrices of X, scaled per row (A) or per
    column (B)."""
    X = np.asarray(X, dtype=np.float64)
    L = beta * s - 1
    rows, cols = X.shape
    if by_rows:
        sig = [_scale_exponent(X[i, :]) for i in range(rows)]
    else:
        sig = [_scale_exponent(X[:, j]) for j in range(cols)]
    D = np.zeros((s, rows, cols), dtype=np.int64)
    for i in range(rows):
        for j in range(cols):
            e = sig[i] if by_rows else sig[j]
            D[:, i, j] = _digits(_scaled_integer(X[i, j], e, L), beta, s)
    return sig, D


def gemm(A, B, beta=8, s=6):
    """C = A B by the emulation's steps 1-5 above (FP64 result)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    n = B.shape[1]
    L = beta * s - 1
    sa, DA = slices(A, True, beta, s)
    sb, DB = slices(B, False, beta, s)
    levels = {}
    for l in range(2, s + 2):
        acc = np.zeros((m, n), dtype=object)
        for q in range(1, l):
            r = l - q
            if q > s or r > s:
                continue
            acc = acc + (DA[q - 1].astype(object) @ DB[r - 1].astype(object))
        levels[l] = acc
    C = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        for j in range(n):
            if sa[i] is None or sb[j] is None:
                continue
            tot = sum(int(levels[l][i, j]) << (beta * (2 * s - l)) for l in levels)
            C[i, j] = float(Fraction(tot) * Fraction(2) ** (sa[i] + sb[j] - 2 * L))
    return C


def truncation_bound(A, B, beta=8, s=6):
    """|C_emu - A B| entrywise bound from steps 2 and 4: every product term is off
    by at most 2^(sigma_i + tau_j) (2 + s(s-1)/2) 2^(-beta s) (rounding of both
    factors to L bits, and the s(s-1)/2 dropped digit pairs), plus the final
    rounding of C."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    k = A.shape[1]
    sa = [_scale_exponent(A[i, :]) for i in range(A.shape[0])]
    sb = [_scale_exponent(B[:, j]) for j in range(B.shape[1])]
    per = (2 + s * (s - 1) / 2) * 2.0 ** (-beta * s)
    out = np.zeros((A.shape[0], B.shape[1]))
    for i, e in enumerate(sa):
        for j, f in enumerate(sb):
            if e is not None and f is not None:
                out[i, j] = k * math.ldexp(per, e + f)
    return out
