"""Host (numpy) half of the shared input generator; see the package docstring."""

import numpy as np

KINDS = ("uniform", "integer", "loguniform")

# A and B of one problem are drawn from two streams of the same seed.
STREAM_A = 0
STREAM_B = 1

# Philox4x32 round multipliers and Weyl key increments (Salmon et al. 2011, Sec. 4).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32 with 10 rounds.

    All arguments are broadcastable integer arrays holding 32-bit values.
    Returns four uint32 arrays (the output words x0..x3).
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def _words(e, seed, stream):
    e = np.asarray(e, dtype=np.uint64)
    seed = int(seed)
    w0, w1, _, _ = philox4x32_10(
        e & _MASK, e >> _S32, np.uint64(stream), np.uint64(0),
        np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    return w0.astype(np.uint64), w1.astype(np.uint64)


def _values(e, kind, dtype, seed, stream):
    w0, w1 = _words(e, seed, stream)
    if kind == "uniform":
        if dtype == "f64":
            r53 = (w1 << np.uint64(21)) | (w0 >> np.uint64(11))
            return np.ldexp(r53.astype(np.float64), -52) - 1.0
        r24 = (w0 >> np.uint64(8)).astype(np.float64)
        x = (np.ldexp(r24, -23) - 1.0).astype(np.float32)  # exact in f32
        return x
    if kind == "integer":
        v = (w0 % np.uint64(17)).astype(np.int64) - 8
        return v.astype(np.float64 if dtype == "f64" else np.float32)
    if kind == "loguniform":
        e2 = ((w0 >> np.uint64(1)) % np.uint64(54)).astype(np.int64) - 27
        mant = 1.0 + np.ldexp((w1 >> np.uint64(9)).astype(np.float64), -23)
        mag = np.ldexp(mant, e2)
        sign = np.where((w0 & np.uint64(1)) == 1, -1.0, 1.0)
        x = sign * mag
        return x if dtype == "f64" else x.astype(np.float32)
    raise ValueError(f"unknown kind {kind!r}")


def _finish(x, dtype):
    if dtype == "bf16":
        import torch  # host-side rounding to bf16 is round-to-nearest-even
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return x


def matrix(rows_, cols_, kind="uniform", dtype="f64", seed=0, stream=STREAM_A):
    """Full rows_ x cols_ matrix (row-major numpy array; torch bf16 tensor for bf16)."""
    e = np.arange(rows_ * cols_, dtype=np.uint64)
    return _finish(_values(e, kind, dtype, seed, stream).reshape(rows_, cols_), dtype)


def entries(r, c, cols_total, kind="uniform", dtype="f64", seed=0, stream=STREAM_A):
    """Elements (r[i], c[i]) of a matrix with cols_total columns."""
    r = np.asarray(r, dtype=np.uint64)
    c = np.asarray(c, dtype=np.uint64)
    e = r * np.uint64(cols_total) + c
    return _finish(_values(e, kind, dtype, seed, stream), dtype)


def rows(row_idx, cols_total, kind="uniform", dtype="f64", seed=0, stream=STREAM_A):
    """Full rows row_idx (len(row_idx) x cols_total)."""
    r = np.asarray(row_idx, dtype=np.uint64)[:, None]
    c = np.arange(cols_total, dtype=np.uint64)[None, :]
    return entries(r, c, cols_total, kind, dtype, seed, stream)


def cols(col_idx, rows_total, cols_total, kind="uniform", dtype="f64", seed=0, stream=STREAM_B):
    """Full columns col_idx, returned transposed (len(col_idx) x rows_total)."""
    c = np.asarray(col_idx, dtype=np.uint64)[:, None]
    r = np.arange(rows_total, dtype=np.uint64)[None, :]
    return entries(r, c, cols_total, kind, dtype, seed, stream)


def grouped_dims(count, seed=1, lo=64, hi=4096, stream=7):
    """Sizes of a grouped workload: m, n, k of each problem are round(lo (hi/lo)^u),
    u uniform in [0, 1) from this generator (seed, stream) -- log-uniform in [lo, hi]."""
    u = (entries(np.arange(3 * count), np.zeros(3 * count), 1, "uniform", "f64", seed, stream)
         + 1.0) / 2.0
    return np.round(lo * (hi / lo) ** u).astype(np.int64).reshape(count, 3)
