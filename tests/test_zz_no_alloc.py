"""The allocation-free split-k entry point (cosma_gemm_splitk_static).

It serves callers that may not allocate device memory while running (global-
mode graph capture, programs that own all device memory through their own
pool, loops that cannot take cudaMalloc's implicit synchronisation); its
partial sums live in a fixed static device array instead of the library arena.
Checked through the C ABI against the regular entry point (cosma_gemm_planned
with the same k split) on two calls in a row, within the tolerances of the
native parity tests.  Kept last in collection order.
"""
import numpy as np
import pytest

from oracle import gemm as og

from gpu_util import device_operands, lib, out_tensor

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


def _static(m, n, k, dtype, A, B, pk):
    import torch
    cosma = lib()
    C, _ = out_tensor(m, n, dtype)
    rc = cosma.cosma_gemm_splitk_static(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(),
                                        B.stride(0), C.data_ptr(), C.stride(0),
                                        cosma.DTYPES[dtype], pk,
                                        torch.cuda.current_stream().cuda_stream)
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


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_static_scratch_two_calls_match_regular_entry(dtype):
    import torch
    cosma = lib()
    calls = [((300, 260, 515), 3, 11), ((257, 129, 1000), 2, 12)]
    for (m, n, k), pk, seed in calls:  # two calls in a row, different shapes and splits
        A, B = device_operands(m, n, k, dtype, seed=seed)
        got = _static(m, n, k, dtype, A, B, pk)
        want = _regular(m, n, k, dtype, A, B, pk)
        torch.cuda.synchronize()
        assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
        _close(got, want, dtype, A, B, k)


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
