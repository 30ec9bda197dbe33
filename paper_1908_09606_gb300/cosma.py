"""Thin ctypes binding of include/cosma.h (argument marshalling only).

Every compute step runs in the CUDA library; this module only converts Python
ints / torch tensors into the C call's pointers, sizes and stream.  If the
shared library is missing it raises -- there is no CPU fallback.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcosma_gb300.so")

(COSMA_F64, COSMA_F32, COSMA_BF16, COSMA_F64_EMU_BF16, COSMA_F64_EMU_INT8,
 COSMA_F32_EMU_TF32) = range(6)
DTYPES = {"f64": COSMA_F64, "f32": COSMA_F32, "bf16": COSMA_BF16,
          "f64_emu_bf16": COSMA_F64_EMU_BF16, "f64_emu_int8": COSMA_F64_EMU_INT8,
          "f32_emu_tf32": COSMA_F32_EMU_TF32}
COSMA_OK = 0
COSMA_ERR_INVALID_ARG = -1
COSMA_ERR_UNSUPPORTED = -2
COSMA_ERR_CUDA = -3
COSMA_ERR_TIMEOUT = -4
COSMA_ERR_NONFINITE = -5
COSMA_ERR_NO_WORKSPACE = -6
COSMA_SELECT_ANALYTIC, COSMA_SELECT_LEARNED = 0, 1
KERNELS = {0: "simt_f64", 1: "simt_f32", 2: "tc_bf16", 3: "emu_bf16", 4: "tf32x3"}


class cosma_config(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("selector", ctypes.c_int),
                ("emu_slices", ctypes.c_int), ("emu_slice_bits", ctypes.c_int),
                ("wait_limit", ctypes.c_longlong), ("grouped_tile", ctypes.c_int)]


class cosma_plan(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_m", ctypes.c_int), ("tile_n", ctypes.c_int),
                ("k_block", ctypes.c_int), ("stages", ctypes.c_int), ("pm", ctypes.c_int),
                ("pn", ctypes.c_int), ("pk", ctypes.c_int), ("order", ctypes.c_int),
                ("ctas", ctypes.c_int), ("sms", ctypes.c_int),
                ("workspace_bytes", ctypes.c_longlong), ("fast_words", ctypes.c_double),
                ("io_words", ctypes.c_double), ("bound_words", ctypes.c_double),
                ("est_seconds", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class cosma_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class CosmaError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


_lib = None

# (name, restype, argtypes) of every entry point in include/cosma.h
_I64, _VP, _INT, _LL, _D = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
SIGNATURES = [
    ("cosma_init", _INT, [ctypes.POINTER(cosma_config)]),
    ("cosma_get_config", _INT, [ctypes.POINTER(cosma_config)]),
    ("cosma_set_workspace", _INT, [_VP, ctypes.c_size_t]),
    ("cosma_finalize", None, []),
    ("cosma_gemm", _INT, [_I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _INT, _VP]),
    ("cosma_gemm_planned", _INT, [_I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _INT,
                                  ctypes.POINTER(cosma_plan), _VP]),
    ("cosma_gemm_ex", _INT, [_INT, _INT, _I64, _I64, _I64, _D, _VP, _I64, _VP, _I64, _D, _VP,
                             _I64, _INT, _VP]),
    ("cosma_zgemm", _INT, [_INT, _INT, _I64, _I64, _I64, ctypes.POINTER(_D), _VP, _I64, _VP,
                           _I64, ctypes.POINTER(_D), _VP, _I64, _INT, _VP]),
    ("cosma_cgemm", _INT, [_INT, _INT, _I64, _I64, _I64, ctypes.POINTER(ctypes.c_float), _VP,
                           _I64, _VP, _I64, ctypes.POINTER(ctypes.c_float), _VP, _I64, _INT,
                           _VP]),
    ("cosma_gemm_grouped", _INT, [_INT, ctypes.POINTER(cosma_problem), _INT, _VP]),
    ("cosma_gemm_host", _INT, [_I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _INT, _VP]),
    ("cosma_plan_query", _INT, [_I64, _I64, _I64, _INT, _INT, ctypes.POINTER(cosma_plan)]),
    ("cosma_plan_units", _LL, [_I64, _I64, _I64, ctypes.POINTER(cosma_plan),
                               ctypes.POINTER(ctypes.c_int64), _LL]),
    ("cosma_find_seq_schedule", _INT, [_LL, ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    ("cosma_fit_ranks", _INT, [_I64, _I64, _I64, _INT, _D, ctypes.POINTER(_INT)]),
    ("cosma_stream_status", _INT, [_VP]),
    ("cosma_status_string", ctypes.c_char_p, [_INT]),
    ("cosma_device_sms", _INT, []),
    ("cosma_launch_count", _LL, []),
    ("cosma_profile_enable", _INT, [_INT]),
    ("cosma_profile_read", _INT, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_LL)]),
    ("cosma_profile_host", _INT, [ctypes.POINTER(ctypes.c_double), _INT]),
    ("cosma_plan_candidate", _INT, [_I64, _I64, _I64, _INT, _INT, ctypes.POINTER(cosma_plan)]),
    ("cosma_selector_features", _INT, [_I64, _I64, _I64, _INT, ctypes.POINTER(ctypes.c_float)]),
    ("cosma_mlp_forward", _INT, [_INT, _VP, _VP, _VP, _VP]),
    ("cosma_mlp_loss_grad", _INT, [_INT, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("cosma_mlp_adam", _INT, [_INT, _VP, _VP, _VP, _VP, _INT, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, _VP]),
    ("cosma_selector_set", _INT, [ctypes.POINTER(ctypes.c_float), _D, _D]),
    ("cosma_selector_restrict", _INT, [ctypes.c_uint]),
    ("cosma_selector_margin", _INT, [_INT, ctypes.c_float]),
    ("cosma_selector_predict", _INT, [_INT, ctypes.POINTER(ctypes.c_int64), _INT,
                                      ctypes.POINTER(_INT), ctypes.POINTER(ctypes.c_float)]),
    ("cosma_gemm_splitk_static", _INT, [_I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64,
                                        _INT, _INT, _VP]),
]
COSMA_STATIC_SCRATCH_BYTES = 32 << 20
COSMA_MLP_IN, COSMA_MLP_HIDDEN, COSMA_MLP_OUT = 7, 64, 16
COSMA_MLP_PARAMS = 64 * 7 + 64 + 64 * 64 + 64 + 16 * 64 + 16


def load(path=None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, where):
    if status != COSMA_OK:
        raise CosmaError(status, where)
    return status


def status_string(status):
    try:
        return load().cosma_status_string(status).decode()
    except Exception:  # library missing: still give a readable message
        return {0: "ok", -1: "invalid argument", -2: "unsupported", -3: "CUDA error",
                -4: "device wait timed out", -5: "non-finite input", -6: "no workspace"}.get(
                    status, "unknown status")


# ---- C-named wrappers (raw pointers and sizes) ---------------------------

def cosma_init(delta=0.03, selector=COSMA_SELECT_ANALYTIC, emu_slices=0, emu_slice_bits=0,
               wait_limit=0, grouped_tile=0):
    cfg = cosma_config(delta, selector, emu_slices, emu_slice_bits, wait_limit, grouped_tile)
    return load().cosma_init(ctypes.byref(cfg))


def cosma_get_config():
    cfg = cosma_config()
    _check(load().cosma_get_config(ctypes.byref(cfg)), "cosma_get_config")
    return cfg


def cosma_set_workspace(dptr, nbytes):
    return load().cosma_set_workspace(dptr, nbytes)


def cosma_finalize():
    load().cosma_finalize()


def cosma_gemm(m, n, k, A, lda, B, ldb, C, ldc, dtype, stream=0):
    return load().cosma_gemm(m, n, k, A, lda, B, ldb, C, ldc, dtype, stream)


def cosma_gemm_planned(m, n, k, A, lda, B, ldb, C, ldc, dtype, plan, stream=0):
    return load().cosma_gemm_planned(m, n, k, A, lda, B, ldb, C, ldc, dtype,
                                     ctypes.byref(plan), stream)


def cosma_gemm_grouped(problems, dtype, stream=0):
    arr = (cosma_problem * len(problems))(*problems)
    return load().cosma_gemm_grouped(len(problems), arr, dtype, stream)


def cosma_gemm_ex(trans_a, trans_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, dtype,
                  stream=0):
    return load().cosma_gemm_ex(trans_a, trans_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                dtype, stream)


def cosma_zgemm(op_a, op_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, engine, stream=0):
    """alpha, beta: Python complex numbers."""
    al = (_D * 2)(alpha.real, alpha.imag)
    be = (_D * 2)(beta.real, beta.imag)
    return load().cosma_zgemm(op_a, op_b, m, n, k, al, A, lda, B, ldb, be, C, ldc, engine, stream)


def cosma_cgemm(op_a, op_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, engine, stream=0):
    """alpha, beta: Python complex numbers (passed as float pairs)."""
    al = (ctypes.c_float * 2)(alpha.real, alpha.imag)
    be = (ctypes.c_float * 2)(beta.real, beta.imag)
    return load().cosma_cgemm(op_a, op_b, m, n, k, al, A, lda, B, ldb, be, C, ldc, engine, stream)


def cosma_gemm_host(m, n, k, A, lda, B, ldb, C, ldc, dtype, stream=0):
    return load().cosma_gemm_host(m, n, k, A, lda, B, ldb, C, ldc, dtype, stream)


def cosma_gemm_splitk_static(m, n, k, A, lda, B, ldb, C, ldc, dtype, pk, stream=0):
    return load().cosma_gemm_splitk_static(m, n, k, A, lda, B, ldb, C, ldc, dtype, pk, stream)


def cosma_plan_candidate(m, n, k, dtype, c):
    """Plan of candidate c, or None when it does not apply."""
    p = cosma_plan()
    rc = load().cosma_plan_candidate(m, n, k, dtype, c, ctypes.byref(p))
    if rc == COSMA_ERR_UNSUPPORTED:
        return None
    _check(rc, "cosma_plan_candidate")
    return p


def cosma_selector_features(m, n, k, dtype):
    x = (ctypes.c_float * COSMA_MLP_IN)()
    _check(load().cosma_selector_features(m, n, k, dtype, x), "cosma_selector_features")
    return list(x)


def cosma_mlp_forward(batch, X, params, Y, stream=0):
    return load().cosma_mlp_forward(batch, X, params, Y, stream)


def cosma_mlp_loss_grad(batch, X, cand, target, params, grad, loss, stream=0):
    return load().cosma_mlp_loss_grad(batch, X, cand, target, params, grad, loss, stream)


def cosma_mlp_adam(n, params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    return load().cosma_mlp_adam(n, params, grad, m, v, step, lr, beta1, beta2, eps, stream)


def cosma_selector_set(params, log2_lo=0.0, log2_hi=64.0):
    """params: sequence of COSMA_MLP_PARAMS floats, or None to remove the network."""
    if params is None:
        return load().cosma_selector_set(None, log2_lo, log2_hi)
    arr = (ctypes.c_float * COSMA_MLP_PARAMS)(*[float(x) for x in params])
    return load().cosma_selector_set(arr, log2_lo, log2_hi)


def cosma_selector_margin(dtype, log2_margin):
    """How much faster (log2 seconds) the network must predict a candidate than
    the analytic plan before the learned selector takes it, for one dtype."""
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return load().cosma_selector_margin(code, float(log2_margin))


def cosma_selector_restrict(dtypes):
    """Limit the installed network to the given dtype codes or names."""
    mask = 0
    for d in dtypes:
        mask |= 1 << (DTYPES[d] if isinstance(d, str) else int(d))
    return load().cosma_selector_restrict(mask)


def cosma_selector_predict(shapes, dtype):
    """Best candidate (and all predictions) for a list of (m, n, k)."""
    count = len(shapes)
    mnk = (ctypes.c_int64 * (3 * count))(*[int(v) for s in shapes for v in s])
    best = (ctypes.c_int * count)()
    pred = (ctypes.c_float * (count * COSMA_MLP_OUT))()
    _check(load().cosma_selector_predict(count, mnk, dtype, best, pred), "cosma_selector_predict")
    return list(best), [list(pred[i * COSMA_MLP_OUT:(i + 1) * COSMA_MLP_OUT]) for i in range(count)]


def cosma_plan_query(m, n, k, dtype, selector=COSMA_SELECT_ANALYTIC):
    p = cosma_plan()
    _check(load().cosma_plan_query(m, n, k, dtype, selector, ctypes.byref(p)), "cosma_plan_query")
    return p


def cosma_plan_units(m, n, k, plan):
    lib = load()
    total = lib.cosma_plan_units(m, n, k, ctypes.byref(plan), None, 0)
    if total < 0:
        raise CosmaError(int(total), "cosma_plan_units")
    buf = (ctypes.c_int64 * (6 * total))()
    lib.cosma_plan_units(m, n, k, ctypes.byref(plan), buf, total)
    return [tuple(buf[6 * i:6 * i + 6]) for i in range(total)]


def cosma_find_seq_schedule(S):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().cosma_find_seq_schedule(S, ctypes.byref(a), ctypes.byref(b)),
           "cosma_find_seq_schedule")
    return a.value, b.value


def cosma_fit_ranks(m, n, k, p, delta):
    g = (ctypes.c_int * 3)()
    _check(load().cosma_fit_ranks(m, n, k, p, delta, g), "cosma_fit_ranks")
    return tuple(g)


def cosma_stream_status(stream=0):
    return load().cosma_stream_status(stream)


def cosma_device_sms():
    return load().cosma_device_sms()


def cosma_launch_count():
    return load().cosma_launch_count()


def cosma_profile_enable(on=True):
    return load().cosma_profile_enable(1 if on else 0)


def cosma_profile_read():
    """(summed milliseconds of the dominant kernels, number of launches timed)."""
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(load().cosma_profile_read(ctypes.byref(ms), ctypes.byref(n)), "cosma_profile_read")
    return ms.value, n.value


HOST_PHASES = ("total_ms", "head_ms", "block_products_ms", "tail_ms", "copy_in_ms", "blocks")


def cosma_profile_host():
    """Phases of the last profiled cosma_gemm_host call, as a dict keyed by
    HOST_PHASES (milliseconds; 'blocks' is the number of block products)."""
    buf = (ctypes.c_double * len(HOST_PHASES))()
    n = load().cosma_profile_host(buf, len(HOST_PHASES))
    if n < 0:
        raise CosmaError(n, "cosma_profile_host")
    out = {name: float(buf[i]) for i, name in enumerate(HOST_PHASES[:n])}
    if "blocks" in out:
        out["blocks"] = int(out["blocks"])
    return out


# ---- torch convenience (marshalling only) --------------------------------

def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def gemm(A, B, C, dtype, stream=None, plan=None):
    """C = A B for row-major torch CUDA tensors (C preallocated).  Raises on error."""
    m, k = A.shape
    k2, n = B.shape
    assert k == k2 and tuple(C.shape) == (m, n)
    for t in (A, B, C):
        assert t.is_cuda and t.stride(1) == 1, "row-major CUDA tensors with unit column stride"
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    s = _stream_handle(stream)
    lda, ldb, ldc = max(A.stride(0), 1), max(B.stride(0), 1), max(C.stride(0), 1)
    if plan is None:
        rc = cosma_gemm(m, n, k, A.data_ptr(), lda, B.data_ptr(), ldb, C.data_ptr(), ldc, dtype, s)
    else:
        rc = cosma_gemm_planned(m, n, k, A.data_ptr(), lda, B.data_ptr(), ldb, C.data_ptr(),
                                ldc, dtype, plan, s)
    return _check(rc, "cosma_gemm")


def gemm_ex(A, B, C, dtype, alpha=1.0, beta=0.0, trans_a=False, trans_b=False, stream=None):
    """C = alpha op(A) op(B) + beta C for row-major torch CUDA tensors; A (B) holds
    op(A)^T (op(B)^T) when trans_a (trans_b).  Raises on error."""
    m, n = C.shape
    k = A.shape[0] if trans_a else A.shape[1]
    assert (A.shape[1] if trans_a else A.shape[0]) == m
    assert (B.shape[1] if trans_b else B.shape[0]) == k
    assert (B.shape[0] if trans_b else B.shape[1]) == n
    for t in (A, B, C):
        assert t.is_cuda and t.stride(1) == 1, "row-major CUDA tensors with unit column stride"
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    s = _stream_handle(stream)
    rc = cosma_gemm_ex(int(trans_a), int(trans_b), m, n, k, float(alpha), A.data_ptr(),
                       max(A.stride(0), 1), B.data_ptr(), max(B.stride(0), 1), float(beta),
                       C.data_ptr(), max(C.stride(0), 1), dtype, s)
    return _check(rc, "cosma_gemm_ex")


def gemm_complex(A, B, C, engine="f64_emu_bf16", alpha=1.0, beta=0.0, op_a=0, op_b=0,
                 stream=None):
    """C = alpha op(A) op(B) + beta C for row-major torch complex128 (cosma_zgemm;
    engine f64 or f64_emu_bf16) or complex64 (cosma_cgemm; engine f32 or
    f32_emu_tf32) CUDA tensors; op 0 none, 1 transpose, 2 conjugate transpose (A / B
    then hold the stored transposes).  Raises on error."""
    m, n = C.shape
    k = A.shape[0] if op_a else A.shape[1]
    assert (A.shape[1] if op_a else A.shape[0]) == m
    assert (B.shape[1] if op_b else B.shape[0]) == k
    assert (B.shape[0] if op_b else B.shape[1]) == n
    for t in (A, B, C):
        assert t.is_cuda and t.stride(1) == 1, "row-major CUDA tensors with unit column stride"
    if isinstance(engine, str):
        engine = DTYPES[engine]
    s = _stream_handle(stream)
    single = str(C.dtype) == "torch.complex64"
    fn = cosma_cgemm if single else cosma_zgemm
    rc = fn(int(op_a), int(op_b), m, n, k, complex(alpha), A.data_ptr(),
            max(A.stride(0), 1), B.data_ptr(), max(B.stride(0), 1), complex(beta),
            C.data_ptr(), max(C.stride(0), 1), engine, s)
    return _check(rc, "cosma_cgemm" if single else "cosma_zgemm")


def gemm_host(A, B, C, dtype, stream=None):
    """C = A B for row-major torch CPU tensors (page-locked for overlap), C
    preallocated; asynchronous on `stream` (synchronise before reading C)."""
    m, k = A.shape
    k2, n = B.shape
    assert k == k2 and tuple(C.shape) == (m, n)
    for t in (A, B, C):
        assert not t.is_cuda and t.stride(1) == 1, "row-major CPU tensors with unit column stride"
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    s = _stream_handle(stream)
    lda, ldb, ldc = max(A.stride(0), 1), max(B.stride(0), 1), max(C.stride(0), 1)
    rc = cosma_gemm_host(m, n, k, A.data_ptr(), lda, B.data_ptr(), ldb, C.data_ptr(), ldc, dtype, s)
    return _check(rc, "cosma_gemm_host")


def gemm_grouped(As, Bs, Cs, dtype, stream=None):
    """Grouped C_i = A_i B_i for lists of row-major torch CUDA tensors."""
    if isinstance(dtype, str):
        dtype = DTYPES[dtype]
    probs = []
    for A, B, C in zip(As, Bs, Cs):
        m, k = A.shape
        n = B.shape[1]
        probs.append(cosma_problem(m, n, k, A.data_ptr(), max(A.stride(0), 1), B.data_ptr(),
                                   max(B.stride(0), 1), C.data_ptr(), max(C.stride(0), 1)))
    return _check(cosma_gemm_grouped(probs, dtype, _stream_handle(stream)), "cosma_gemm_grouped")
