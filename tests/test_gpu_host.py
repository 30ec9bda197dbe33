"""GPU tests of cosma_gemm_host: operands and result in host memory, copies
pipelined against the kernels by the library.

Parity: on shapes below the 8192 cut the call runs the same plan as
cosma_gemm on device copies of the operands, so the results are bit-equal;
with rows and columns cut in two (2 x 2 blocks, ragged second block) each
block is planned on its own, so the check is against the oracle on sampled
entries with the dtype's bound (FP64 and emulated FP64: 1e-13 / 1e-12 relative
to the row-column scale; FP32 / BF16: gamma_k |A||B| elementwise)."""
import numpy as np
import pytest

from gpu_util import (GEN_DT, OUT_DT, TORCH_DT, device_operands, host_operands, lib,
                      out_tensor, sample_indices, sampled_reference)
from oracle import gemm as og

pytestmark = pytest.mark.gpu

DTYPES = ["f64", "f32", "bf16", "f64_emu_bf16"]


def _host_copies(m, n, k, dtype, kind="uniform", seed=0, pin=True, lda=None, ldb=None):
    """Host (optionally page-locked) copies of the device operands."""
    import torch
    A, B = device_operands(m, n, k, dtype, kind, seed)
    tdt = getattr(torch, TORCH_DT[GEN_DT[dtype]])
    Ah = torch.zeros((m, lda or max(k, 1)), dtype=tdt, pin_memory=pin)[:, :k]
    Bh = torch.zeros((k, ldb or max(n, 1)), dtype=tdt, pin_memory=pin)[:, :n]
    Ah.copy_(A.cpu())
    Bh.copy_(B.cpu())
    return A, B, Ah, Bh


def _host_out(m, n, dtype, pin=True, ldc=None):
    import torch
    tdt = getattr(torch, OUT_DT[dtype])
    Cst = torch.full((m, ldc or max(n, 1)), float("nan"), dtype=tdt, pin_memory=pin)
    return Cst[:, :n]


def _status_ok(cosma):
    import torch
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (200, 136, 300), (129, 1000, 77), (513, 257, 1031)])
def test_host_equals_device_path(dtype, shape):
    import torch
    cosma = lib()
    m, n, k = shape
    A, B, Ah, Bh = _host_copies(m, n, k, dtype)
    C, _ = out_tensor(m, n, dtype)
    cosma.gemm(A, B, C, dtype)
    Ch = _host_out(m, n, dtype)
    cosma.gemm_host(Ah, Bh, Ch, dtype)
    torch.cuda.synchronize()
    _status_ok(cosma)
    assert torch.equal(Ch, C.cpu())


@pytest.mark.parametrize("dtype", DTYPES)
def test_host_padded_leading_dimensions_and_pageable(dtype):
    import torch
    cosma = lib()
    m, n, k = 300, 170, 261
    A, B, Ah, Bh = _host_copies(m, n, k, dtype, pin=False, lda=k + 5, ldb=n + 3)
    C, _ = out_tensor(m, n, dtype)
    cosma.gemm(A, B, C, dtype)
    Cst = torch.full((m, n + 7), -7.0, dtype=getattr(torch, OUT_DT[dtype]))
    Ch = Cst[:, :n]
    cosma.gemm_host(Ah, Bh, Ch, dtype)
    torch.cuda.synchronize()
    _status_ok(cosma)
    assert torch.equal(Ch, C.cpu())
    assert torch.all(Cst[:, n:] == -7.0)  # padding untouched


def _bound(dtype, Ar, Bc):
    absprod = np.abs(Ar) @ np.abs(Bc).T
    k = Ar.shape[1]
    if dtype == "f64":
        return 1e-13 * np.sqrt((Ar ** 2).sum(1))[:, None] * np.sqrt((Bc ** 2).sum(1))[None, :]
    if dtype == "f64_emu_bf16":
        return 1e-12 * np.sqrt((Ar ** 2).sum(1))[:, None] * np.sqrt((Bc ** 2).sum(1))[None, :]
    u = 2.0 ** -23 if dtype == "bf16" else 2.0 ** -24
    return (k * u / (1 - k * u)) * absprod


@pytest.mark.parametrize("dtype", DTYPES)
def test_host_two_by_two_blocks_sampled(dtype):
    """m, n >= 8192: rows and columns are cut in two (second blocks ragged)."""
    import torch
    cosma = lib()
    m, n, k = 8200, 8328, 96
    _, _, Ah, Bh = _host_copies(m, n, k, dtype, kind="uniform", seed=5)
    Ch = _host_out(m, n, dtype)
    cosma.gemm_host(Ah, Bh, Ch, dtype)
    torch.cuda.synchronize()
    _status_ok(cosma)
    C = Ch.double().numpy()
    assert np.isfinite(C).all()
    rr, cc = sample_indices(m, n, 400, seed=9, tile=256)
    # entries on both sides of the block cuts (4352 rows, 4352 columns)
    rr = np.concatenate([rr, [4351, 4352, 4351, 4352]])
    cc = np.concatenate([cc, [4351, 4351, 4352, 4352]])
    ref, Ar, Bc, ri, cj = sampled_reference(m, n, k, dtype, rr, cc, "uniform", 5)
    got = C[rr, cc]
    tol = np.array([_bound(dtype, Ar[ri[i]][None], Bc[cj[i]][None])[0, 0]
                    for i in range(len(rr))])
    assert np.all(np.abs(got - ref) <= tol + 1e-300), np.max(np.abs(got - ref) / (tol + 1e-300))


def test_host_two_by_two_emu_bit_equal_to_device():
    """Emulated FP64 is tile-independent per entry: the blocked host call and the
    whole-matrix device call agree bit for bit."""
    import torch
    cosma = lib()
    m, n, k = 8200, 8328, 200
    A, B, Ah, Bh = _host_copies(m, n, k, "f64_emu_bf16", kind="loguniform", seed=2)
    C, _ = out_tensor(m, n, "f64_emu_bf16")
    cosma.gemm(A, B, C, "f64_emu_bf16")
    Ch = _host_out(m, n, "f64_emu_bf16")
    cosma.gemm_host(Ah, Bh, Ch, "f64_emu_bf16")
    torch.cuda.synchronize()
    _status_ok(cosma)
    assert torch.equal(Ch, C.cpu())


def test_host_calls_in_a_row_and_graph_replay():
    """Two calls in a row reuse the staging; a captured call replays with new
    host contents (copies read the same page-locked addresses)."""
    import torch
    cosma = lib()
    m, n, k = 384, 320, 256
    dtype = "f64"
    _, _, Ah, Bh = _host_copies(m, n, k, dtype, seed=1)
    Ch = _host_out(m, n, dtype)
    cosma.gemm_host(Ah, Bh, Ch, dtype)
    cosma.gemm_host(Ah, Bh, Ch, dtype)  # staging sized: capture needs no allocation
    torch.cuda.synchronize()
    first = Ch.clone()
    ref = og.gemm(Ah.numpy(), Bh.numpy(), "dot2")
    assert og.normwise_rel_error(first.numpy(), ref) <= 1e-13

    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = cosma.cosma_gemm_host(m, n, k, Ah.data_ptr(), k, Bh.data_ptr(), n, Ch.data_ptr(), n,
                                   cosma.DTYPES[dtype], s.cuda_stream)
    assert rc == cosma.COSMA_OK
    Ah.mul_(-2.0)
    Ch.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(Ch, -2.0 * first)  # scaling by -2 is exact in every entry
    _status_ok(cosma)


def test_host_k_zero_and_errors():
    import torch
    cosma = lib()
    Ch = _host_out(5, 7, "f64")
    Ah = torch.zeros((5, 1), dtype=torch.float64, pin_memory=True)
    Bh = torch.zeros((1, 7), dtype=torch.float64, pin_memory=True)
    assert cosma.cosma_gemm_host(5, 7, 0, Ah.data_ptr(), 1, Bh.data_ptr(), 7, Ch.data_ptr(), 7,
                                 cosma.COSMA_F64, 0) == cosma.COSMA_OK
    torch.cuda.synchronize()
    assert torch.all(Ch == 0)
    # device pointers are refused (before any copy)
    Ah = torch.zeros((5, 3), dtype=torch.float64, pin_memory=True)
    Bh = torch.zeros((3, 7), dtype=torch.float64, pin_memory=True)
    Ad = torch.zeros((5, 3), dtype=torch.float64, device="cuda")
    Bd = torch.zeros((3, 7), dtype=torch.float64, device="cuda")
    Cd = torch.zeros((5, 7), dtype=torch.float64, device="cuda")
    assert cosma.cosma_gemm_host(5, 7, 3, Ad.data_ptr(), 3, Bd.data_ptr(), 7, Cd.data_ptr(), 7,
                                 cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_gemm_host(5, 7, 3, Ah.data_ptr(), 3, Bh.data_ptr(), 7, Cd.data_ptr(), 7,
                                 cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_gemm_host(5, 7, 3, Ah.data_ptr(), 3, Bh.data_ptr(), 7, Ch.data_ptr(), 7,
                                 cosma.COSMA_F64_EMU_INT8, 0) == cosma.COSMA_ERR_UNSUPPORTED


def test_host_phase_profile():
    """cosma_profile_host reports the phases of a profiled call: the head, the
    block products and the tail lie inside the whole call, the copies in end
    within it, and a 2 x 2 blocked call has four block products."""
    import torch
    cosma = lib()
    m = n = 8200
    k = 256
    dtype = "f64_emu_bf16"
    _, _, Ah, Bh = _host_copies(m, n, k, dtype, seed=3)
    Ch = _host_out(m, n, dtype)
    st = torch.cuda.current_stream().cuda_stream
    code = cosma.DTYPES[dtype]
    assert cosma.cosma_profile_enable(True) == 0
    try:
        rc = cosma.cosma_gemm_host(m, n, k, Ah.data_ptr(), Ah.stride(0), Bh.data_ptr(),
                                   Bh.stride(0), Ch.data_ptr(), Ch.stride(0), code, st)
        assert rc == 0
        ph = cosma.cosma_profile_host()
    finally:
        cosma.cosma_profile_enable(False)
        cosma.cosma_profile_read()  # clears the kernel event pairs of the call
    torch.cuda.synchronize()
    assert ph["blocks"] == 4
    assert 0 < ph["head_ms"] and 0 < ph["block_products_ms"] and 0 <= ph["tail_ms"]
    assert ph["head_ms"] + ph["block_products_ms"] + ph["tail_ms"] <= ph["total_ms"] * 1.001 + 1e-3
    assert 0 < ph["copy_in_ms"] <= ph["total_ms"] * 1.001 + 1e-3
    assert cosma.cosma_stream_status(st) == 0
