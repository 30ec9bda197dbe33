"""The allocation-free split-k entry point (cosma_gemm_splitk_static).

It serves callers that may not allocate device memory while running (global-
mode graph capture, programs that own all device memory through their own
pool, loops that cannot take cudaMalloc's implicit synchronisation); its
partial sums live in a fixed static device array instead of the library arena.
Checked through the C ABI, on two calls in a row: against the oracle (FP64
normwise <= 1e-13 against Dot2, FP32 elementwise within gamma_k |A||B|, the
native parity bars) and against the regular entry point with the same k split;
that it allocates nothing (free device memory unchanged across calls, and a call
recorded under global-mode stream capture, where any cudaMalloc fails the
capture, replays to the same bits).  Kept last in collection order.
"""
import numpy as np
import pytest

from oracle import gemm as og

from gpu_util import device_operands, host_operands, lib, out_tensor

pytestmark = pytest.mark.gpu


def _gamma(k, u):
    return k * u / (1 - k * u)


def _regular(m, n, k, dtype, A, B, pk):
    import torch
    cosma = lib()
    p = cosma.cosma_plan_query(m, n, k, cosma.DTYPES[dtype])
    tiles = -(-m // p.tile_m) * -(-n // p.tile_n)
    p.pk, p.order, p.pm, p.pn = pk, 1, 1, 1
    p.ctas = min(cosma.cosma_device_sms(), tiles * pk)
    C, _ = out_tensor(m, n, dtype)
    rc = cosma.cosma_gemm_planned(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                  C.data_ptr(), C.stride(0), cosma.DTYPES[dtype], p,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_OK
    return C


def _static_into(C, m, n, k, dtype, A, B, pk, stream):
    cosma = lib()
    return cosma.cosma_gemm_splitk_static(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(),
                                          B.stride(0), C.data_ptr(), C.stride(0),
                                          cosma.DTYPES[dtype], pk, stream)


def _static(m, n, k, dtype, A, B, pk):
    import torch
    cosma = lib()
    C, _ = out_tensor(m, n, dtype)
    rc = _static_into(C, m, n, k, dtype, A, B, pk, torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_OK, cosma.status_string(rc)
    return C


def _close(got, want, dtype, A, B, k):
    got = got.double().cpu().numpy()
    want = want.double().cpu().numpy()
    if dtype == "f64":
        assert og.normwise_rel_error(got, want) <= 1e-13
    else:
        absab = np.abs(A.double().cpu().numpy()) @ np.abs(B.double().cpu().numpy())
        assert np.all(np.abs(got - want) <= 2 * _gamma(k, 2.0 ** -24) * absab)


def _against_oracle(got, m, n, k, dtype, seed):
    Ah, Bh = host_operands(m, n, k, dtype, seed=seed)
    ref = og.gemm(Ah, Bh, "dot2")
    got = got.double().cpu().numpy()
    if dtype == "f64":
        assert og.normwise_rel_error(got, ref) <= 1e-13
    else:
        assert np.all(np.abs(got - ref) <= _gamma(k, 2.0 ** -24) * (np.abs(Ah) @ np.abs(Bh)))


CALLS = [((300, 260, 515), 3, 11), ((257, 129, 1000), 2, 12)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_static_scratch_two_calls_match_oracle_and_regular_entry(dtype):
    import torch
    cosma = lib()
    for (m, n, k), pk, seed in CALLS:  # two calls in a row, different shapes and splits
        A, B = device_operands(m, n, k, dtype, seed=seed)
        got = _static(m, n, k, dtype, A, B, pk)
        torch.cuda.synchronize()
        assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
        _against_oracle(got, m, n, k, dtype, seed)
        want = _regular(m, n, k, dtype, A, B, pk)
        torch.cuda.synchronize()
        _close(got, want, dtype, A, B, k)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_static_scratch_allocates_nothing(dtype):
    """After one call has looked the array up (and loaded the library's module),
    further calls leave free device memory unchanged, and a call recorded under
    global-mode stream capture -- in which a cudaMalloc from this thread would
    invalidate the capture -- replays to the bits of an eager call."""
    import torch
    cosma = lib()
    (m, n, k), pk, seed = CALLS[0]
    A, B = device_operands(m, n, k, dtype, seed=seed)
    warm = _static(m, n, k, dtype, A, B, pk)  # first call on the device: symbol lookup
    C1, _ = out_tensor(m, n, dtype)
    C2, _ = out_tensor(m, n, dtype)
    Cg, _ = out_tensor(m, n, dtype)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = torch.cuda.current_stream().cuda_stream
    assert _static_into(C1, m, n, k, dtype, A, B, pk, st) == cosma.COSMA_OK
    assert _static_into(C2, m, n, k, dtype, A, B, pk, st) == cosma.COSMA_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.equal(C1, warm) and torch.equal(C2, warm)

    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side, capture_error_mode="global"):
            rc = _static_into(Cg, m, n, k, dtype, A, B, pk, side.cuda_stream)
    assert rc == cosma.COSMA_OK, cosma.status_string(rc)
    Cg.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    assert torch.equal(Cg, warm)
    _against_oracle(Cg, m, n, k, dtype, seed)


def test_static_scratch_rejects_oversized_split():
    import torch
    cosma = lib()
    m = n = 1024
    k = 4096
    A, B = device_operands(m, n, k, "f64")
    C, _ = out_tensor(m, n, "f64")
    pk = cosma.COSMA_STATIC_SCRATCH_BYTES // (m * n * 8) + 1
    rc = cosma.cosma_gemm_splitk_static(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n,
                                        cosma.COSMA_F64, pk,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_ERR_NO_WORKSPACE
