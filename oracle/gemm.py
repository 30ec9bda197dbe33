"""Oracle GEMM: C = A B by its definition (Sec. 2.4; CDAG of Sec. 5.1).

Test infrastructure only (see the package docstring).  The arithmetic lives in
gemm_oracle.c; this module compiles it with gcc (no fused multiply-add
contraction, no fast-math) and calls it through ctypes.

tiled (libtiled_cpu.so, OpenMP) runs the same chain under the tiled
sequential schedule of Sec. 5.2 on the host cores for the benchmark's CPU timing; it is
pinned by bit-equality with the naive loop.

Pins (tests/test_oracle_gemm.py): exact integer products against Python
integers, identity / diagonal / rank-1 closed forms, exact rational arithmetic
(fractions) on tiny inputs for Dot2, the classical bound |C_naive - C| <= gamma_k
|A||B| for the naive loop, and Freivalds catching a planted error; for gemm_ex,
integer alpha op(A) op(B) + beta C0 against Python integer loops in all four
transpose cases, alpha = 0 giving exactly beta C0, and NaN in C0 ignored when
beta = 0; for zgemm, Gaussian-integer products against Python complex loops for
all nine op cases.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gemm_oracle.c")
_SRC_L1 = os.path.join(_HERE, "tiled_cpu.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgemm_oracle.so")
_LIB_L1 = os.path.join(_BUILD, "libtiled_cpu.so")
_lock = threading.Lock()
_lib = None
_lib_l1 = None


def _compile(src, out, flags):
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc"] + flags + ["-ffp-contract=off", "-fno-fast-math", "-fPIC",
                                             "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build():
    """Compile the C oracle and the host tiled loop (idempotent; rebuilds
    when a source is newer)."""
    os.makedirs(_BUILD, exist_ok=True)
    _compile(_SRC, _LIB, ["-O2"])
    try:
        _compile(_SRC_L1, _LIB_L1, ["-O3", "-fopenmp"])
    except subprocess.CalledProcessError:  # no OpenMP: one thread
        _compile(_SRC_L1, _LIB_L1, ["-O3"])
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            for name in ("oracle_gemm_naive", "oracle_gemm_dot2"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, i64, d, i64, d, i64, d, i64]
                f.restype = None
            lib.oracle_dot2_pairs.argtypes = [i64, i64, d, d, d]
            lib.oracle_dot2_pairs.restype = None
            lib.oracle_freivalds.argtypes = [i64, i64, i64, d, i64, d, i64, d, i64, d, d, d, d, d]
            lib.oracle_freivalds.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gemm(A, B, method="dot2"):
    """C = A B in FP64.  method: 'naive' (partial-sum chain t=0..k-1) or 'dot2'."""
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.zeros((m, n), dtype=np.float64)
    if m and n:
        fn = {"naive": _load().oracle_gemm_naive, "dot2": _load().oracle_gemm_dot2}[method]
        fn(m, n, k, _ptr(A), max(k, 1), _ptr(B), max(n, 1), _ptr(C), max(n, 1))
    return C


def tiled(A, B, a, b, threads=0):
    """C = A B by the sequential schedule of Sec. 5.2 on the host cores: a x b
    blocks of C resident while k streams past them, blocks spread over OpenMP
    threads (threads = 0: all).  Every entry is the chain t = 0..k-1, so the result
    equals gemm(A, B, 'naive') bit for bit.  Returns (C, threads used)."""
    global _lib_l1
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    with _lock:
        if _lib_l1 is None:
            build()
            lib = ctypes.CDLL(_LIB_L1)
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.tiled_gemm.argtypes = [i64, i64, i64, d, i64, d, i64, d, i64, i64, i64,
                                          ctypes.c_int]
            lib.tiled_gemm.restype = ctypes.c_int
            _lib_l1 = lib
    C = np.zeros((m, n), dtype=np.float64)
    used = 0
    if m and n:
        used = _lib_l1.tiled_gemm(m, n, k, _ptr(A), max(k, 1), _ptr(B), max(n, 1), _ptr(C),
                                     max(n, 1), int(a), int(b), int(threads))
        if used < 1:
            raise MemoryError("tiled: block buffer allocation failed")
    return C, used


def gemm_ex(A, B, C0, alpha, beta, trans_a=False, trans_b=False, method="dot2"):
    """C = alpha op(A) op(B) + beta C0 in FP64: the BLAS GEMM definition that the
    ScaLAPACK interface of the paper's implementation follows.  op(X) is X, or the
    transpose of the stored X when its flag is set (A stored k x m, B n x k).  As
    in BLAS, beta == 0 does not read C0 and alpha == 0 or k == 0 does not read A, B."""
    A, B = _f64(A), _f64(B)
    opA = A.T if trans_a else A
    opB = B.T if trans_b else B
    m, k = opA.shape
    k2, n = opB.shape
    assert k == k2
    out = np.zeros((m, n), dtype=np.float64)
    if alpha != 0.0 and k > 0:
        out = alpha * gemm(opA, opB, method)
    if beta != 0.0:
        out = out + beta * _f64(C0)
    return out


def zgemm(A, B, C0, alpha, beta, op_a=0, op_b=0):
    """Complex C = alpha op(A) op(B) + beta C0 in complex128 (BLAS ZGEMM definition);
    op 0: X, 1: transpose of the stored X, 2: conjugate transpose.  The product is
    numpy's complex matmul (a library primitive).  beta == 0 does not read C0;
    alpha == 0 or k == 0 does not read A, B."""
    def op(X, o):
        X = np.asarray(X, dtype=np.complex128)
        return X if o == 0 else (X.T if o == 1 else X.conj().T)
    opA, opB = op(A, op_a), op(B, op_b)
    m, k = opA.shape
    assert opB.shape[0] == k
    out = np.zeros((m, opB.shape[1]), dtype=np.complex128)
    if alpha != 0 and k > 0:
        out = alpha * np.matmul(opA, opB)
    if beta != 0:
        out = out + beta * np.asarray(C0, dtype=np.complex128)
    return out


def dot2_pairs(arows, bcols):
    """out[p] = sum_t arows[p,t] * bcols[p,t], compensated (Dot2)."""
    arows, bcols = _f64(arows), _f64(bcols)
    count, k = arows.shape
    assert bcols.shape == (count, k)
    out = np.zeros(count, dtype=np.float64)
    if count:
        _load().oracle_dot2_pairs(count, k, _ptr(arows), _ptr(bcols), _ptr(out))
    return out


def freivalds(A, B, C, x):
    """Return (r, scale): r = C x - A (B x) and scale = |A|(|B||x|), in Dot2."""
    A, B, C, x = _f64(A), _f64(B), _f64(C), _f64(x)
    m, k = A.shape
    n = B.shape[1]
    bx = np.zeros(k)
    absbx = np.zeros(k)
    r = np.zeros(m)
    scale = np.zeros(m)
    _load().oracle_freivalds(m, n, k, _ptr(A), max(k, 1), _ptr(B), max(n, 1), _ptr(C), max(n, 1),
                             _ptr(x), _ptr(bx), _ptr(absbx), _ptr(r), _ptr(scale))
    return r, scale


def normwise_rel_error(C_hat, C_ref):
    """||C_hat - C_ref||_F / ||C_ref||_F over the entries given (flattened)."""
    C_hat = np.asarray(C_hat, dtype=np.float64).ravel()
    C_ref = np.asarray(C_ref, dtype=np.float64).ravel()
    den = np.linalg.norm(C_ref)
    num = np.linalg.norm(C_hat - C_ref)
    return 0.0 if num == 0.0 else (num / den if den else np.inf)
