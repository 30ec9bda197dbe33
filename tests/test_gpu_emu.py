"""GPU parity of the emulated FP64 path (K-SPLIT / K-EMU / K-RECOMB on bf16
tensor cores) against the FP64 oracle, through the C ABI.

Tolerance: normwise relative error <= 1e-12 against the Dot2 oracle (the bar
stated for emulated FP64); integer-valued inputs bit-exact; non-finite inputs
reported as COSMA_ERR_NONFINITE.
"""
import numpy as np
import pytest

from oracle import gemm as og

from gpu_util import (device_operands, host_operands, lib, out_tensor, sample_indices,
                      sampled_reference)

pytestmark = pytest.mark.gpu
DT = "f64_emu_bf16"


def _run(m, n, k, kind="uniform", seed=0, lda=None, ldb=None, ldc=None, expect=0):
    import torch
    cosma = lib()
    A, B = device_operands(m, n, k, DT, kind, seed, lda, ldb)
    C, _ = out_tensor(m, n, DT, ldc)
    cosma.gemm(A, B, C, DT)
    torch.cuda.synchronize()
    st = cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream)
    assert st == expect, cosma.status_string(st)
    return C.cpu().numpy()


@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 5, 3), (128, 128, 64), (127, 129, 127),
                                   (129, 257, 1025), (200, 136, 1000), (512, 512, 512),
                                   (1000, 7, 129), (64, 64, 1)])
def test_emu_uniform(shape):
    m, n, k = shape
    C = _run(m, n, k)
    A, B = host_operands(m, n, k, DT)
    err = og.normwise_rel_error(C, og.gemm(A, B, "dot2"))
    assert err <= 1e-12, err


@pytest.mark.parametrize("shape", [(300, 200, 500), (256, 384, 2048)])
def test_emu_loguniform(shape):
    m, n, k = shape
    C = _run(m, n, k, kind="loguniform", seed=2)
    A, B = host_operands(m, n, k, DT, kind="loguniform", seed=2)
    err = og.normwise_rel_error(C, og.gemm(A, B, "dot2"))
    assert err <= 1e-12, err


@pytest.mark.parametrize("shape", [(128, 128, 64), (300, 257, 999)])
def test_emu_integer_bit_exact(shape):
    m, n, k = shape
    C = _run(m, n, k, kind="integer", seed=5)
    A, B = host_operands(m, n, k, DT, kind="integer", seed=5)
    assert np.array_equal(C, og.gemm(A, B, "naive"))


def test_emu_padded_leading_dimensions():
    m, n, k = 150, 170, 133
    C = _run(m, n, k, lda=135, ldb=171, ldc=173)
    A, B = host_operands(m, n, k, DT)
    assert og.normwise_rel_error(C, og.gemm(A, B, "dot2")) <= 1e-12


def test_emu_zero_rows_and_columns():
    import torch
    cosma = lib()
    m, n, k = 130, 140, 150
    A, B = device_operands(m, n, k, DT)
    A[5].zero_()
    B[:, 7].zero_()
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    ref = og.gemm(Ah, Bh, "dot2")
    got = C.cpu().numpy()
    assert not got[5].any() and not got[:, 7].any()
    assert og.normwise_rel_error(got, ref) <= 1e-12


def test_emu_nonfinite_flagged():
    import torch
    cosma = lib()
    A, B = device_operands(64, 64, 64, DT)
    A[3, 9] = float("nan")
    C, _ = out_tensor(64, 64, DT)
    cosma.gemm(A, B, C, DT)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == \
        cosma.COSMA_ERR_NONFINITE
    # the status word is cleared by the read; a clean call reports ok again
    _run(64, 64, 64)


@pytest.mark.parametrize("shape,kind", [((8192,) * 3, "uniform"), ((8192,) * 3, "loguniform"),
                                        ((16384,) * 3, "uniform"),
                                        ((4096, 4096, 1 << 20), "uniform"),    # largeK
                                        ((1 << 20, 4096, 4096), "uniform"),    # largeM
                                        ((65536, 65536, 1024), "uniform")])    # flat
def test_emu_full_size_sampled(shape, kind):
    import torch
    cosma = lib()
    m, n, k = shape
    A, B = device_operands(m, n, k, DT, kind=kind, seed=0)
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    del A, B
    rr, cc = sample_indices(m, n, 128 if k > 1 << 16 else 256, seed=m ^ n ^ k)
    ref, _, _, _, _ = sampled_reference(m, n, k, DT, rr, cc, kind=kind)
    got = C[torch.as_tensor(rr, device="cuda"), torch.as_tensor(cc, device="cuda")].cpu().numpy()
    del C
    torch.cuda.empty_cache()
    err = og.normwise_rel_error(got, ref)
    assert err <= 1e-12, err


def _tile_plan(m, n, k, tile):
    """An emulation plan with the given tile: 'pair256' (256 x 256 on a CTA pair,
    candidate 1), 'single' (128 x 128 on one SM, candidate 9) or 'pair128' (the
    256 x 128 pair tile: candidate 1's plan with narrower tiles)."""
    cosma = lib()
    p = cosma.cosma_plan_candidate(m, n, k, cosma.COSMA_F64_EMU_BF16, 9 if tile == "single" else 1)
    assert (p.tile_m, p.tile_n) == ((128, 128) if tile == "single" else (256, 256))
    if tile == "pair128":
        p.tile_n = 128
        p.stages = 9
    return p


@pytest.mark.parametrize("tile", ["pair256", "single", "pair128"])
@pytest.mark.parametrize("shape", [(128, 128, 64), (300, 257, 999), (513, 129, 2048)])
def test_emu_pair_and_single_sm_tiles(tile, shape):
    import torch
    cosma = lib()
    m, n, k = shape
    p = _tile_plan(m, n, k, tile)
    A, B = device_operands(m, n, k, DT, seed=4)
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT, plan=p)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    Ah, Bh = host_operands(m, n, k, DT, seed=4)
    assert og.normwise_rel_error(C.cpu().numpy(), og.gemm(Ah, Bh, "dot2")) <= 1e-12


@pytest.mark.parametrize("tile", ["pair256", "single", "pair128"])
def test_emu_long_k(tile):
    # k = 22001: six 4096-deep super-chunks, 36 merges of the running total, whose
    # fixed-point base rises to 7 bits (the lowest level pair is rounded to it)
    import torch
    cosma = lib()
    m, n, k = 130, 129, 22001
    p = _tile_plan(m, n, k, tile)
    A, B = device_operands(m, n, k, DT, seed=8)
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT, plan=p)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    Ah, Bh = host_operands(m, n, k, DT, seed=8)
    assert og.normwise_rel_error(C.cpu().numpy(), og.gemm(Ah, Bh, "dot2")) <= 1e-12


@pytest.mark.parametrize("slices,bits", [(4, 8), (5, 8), (7, 7), (8, 7), (7, 8), (6, 6)])
def test_emu_slice_configurations(slices, bits):
    """Other slice counts s and digit widths beta (cosma_config): the scaled
    integers keep beta s - 1 bits and the triangle q + r <= s + 1 of slice pairs,
    so the error stays below 2^-(beta s - 8) relative to the row and column norms
    (s = 6, beta = 8: 2^-40, the 1e-12 bar); integer inputs stay bit-exact (only
    their leading digit is nonzero).  Tiles of both kinds: a CTA pair (m >= 256) and
    single-SM tiles (m < 256)."""
    cosma = lib()
    try:
        assert cosma.cosma_init(emu_slices=slices, emu_slice_bits=bits) == 0
        for m, n, k in [(300, 260, 1000), (130, 200, 700)]:
            C = _run(m, n, k, seed=13)
            A, B = host_operands(m, n, k, DT, seed=13)
            ref = og.gemm(A, B, "dot2")
            scale = np.sqrt((A ** 2).sum(1))[:, None] * np.sqrt((B ** 2).sum(0))[None, :]
            tol = 2.0 ** -(bits * slices - 8) * scale
            bad = np.abs(C - ref) > tol
            assert not bad.any(), (slices, bits, m, float(np.max(np.abs(C - ref) / scale)))
            Ci = _run(m, n, k, kind="integer", seed=5)
            Ai, Bi = host_operands(m, n, k, DT, kind="integer", seed=5)
            assert np.array_equal(Ci, og.gemm(Ai, Bi, "naive"))
    finally:
        cosma.cosma_init()


@pytest.mark.parametrize("slices,bits", [(3, 8), (2, 7), (6, 8)])
@pytest.mark.parametrize("shape", [(260, 16, 64), (100, 40, 128)])
def test_emu_equals_the_methods_own_result(slices, bits, shape):
    """The GPU emulation against the step-by-step oracle of the method
    (oracle/ozaki.py: the same scales, digits and truncated triangle in exact
    integer arithmetic): both round the exact total to FP64 once, so they differ
    only where the fixed-point base rounds the lowest level pair -- far below the
    truncation itself; with 3 slices the product is off by ~2^-22 but the two
    agree to 2^-40 of sum |a||b|, so a wrong pair set or scale would show."""
    import torch
    from oracle import ozaki
    cosma = lib()
    m, n, k = shape
    try:
        assert cosma.cosma_init(emu_slices=slices, emu_slice_bits=bits) == 0
        C = _run(m, n, k, seed=31)
    finally:
        cosma.cosma_init()
    A, B = host_operands(m, n, k, DT, seed=31)
    ref_method = ozaki.gemm(A, B, bits, slices)
    absab = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref_method) <= 2.0 ** -40 * absab)
    # With 2 x 7 or 3 x 8 bits the whole running total fits the fixed point
    # without rounding any level (base 0 at these k: one super-chunk adds at most
    # 2^31 resp. 2^42.1), so both sides round the same exact number to FP64 once.
    if slices * bits <= 24:
        assert np.array_equal(C, ref_method)
    if slices * bits < 30:
        exact = og.gemm(A, B, "dot2")
        assert np.max(np.abs(C - exact) / absab) > 2.0 ** -36


@pytest.mark.parametrize("shape,kind", [((300, 520, 3000), "uniform"), ((513, 260, 1100), "loguniform"),
                                        ((260, 300, 9000), "uniform")])
def test_emu_tile_shapes_agree_bit_for_bit(shape, kind):
    """Every kernel forms the same exact fixed-point running total (level sums
    are exact integers and the total is integer arithmetic, rounded to FP64
    once), so 256 x 256 and 256 x 128 pair tiles and 128 x 128 single-SM tiles
    give identical bits, and all meet the oracle bar."""
    import torch
    cosma = lib()
    m, n, k = shape
    A, B = device_operands(m, n, k, DT, kind=kind, seed=21)
    out = []
    for tile in ("pair256", "pair128", "single"):
        C, _ = out_tensor(m, n, DT)
        cosma.gemm(A, B, C, DT, plan=_tile_plan(m, n, k, tile))
        torch.cuda.synchronize()
        assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
        out.append(C.cpu().numpy())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    Ah, Bh = host_operands(m, n, k, DT, kind=kind, seed=21)
    assert og.normwise_rel_error(out[0], og.gemm(Ah, Bh, "dot2")) <= 1e-12


def _split_plan(m, n, k, tile, pk):
    """The tile's plan with k cut into pk slices and as many CTAs (pairs) as the
    units can use."""
    cosma = lib()
    p = _tile_plan(m, n, k, tile)
    tiles = -(-m // p.tile_m) * -(-n // p.tile_n)
    p.pk = pk
    p.ctas = min(p.sms // 2 if p.tile_m == 256 else p.sms, tiles * pk)
    return p


@pytest.mark.parametrize("tile", ["pair256", "single", "pair128"])
@pytest.mark.parametrize("shape,kind,pks", [((300, 520, 4 * 4096 + 515), "uniform", (2, 3, 5)),
                                            ((513, 129, 3 * 4096), "loguniform", (3,)),
                                            ((1100, 700, 2 * 4096 + 64), "uniform", (2, 3))])
def test_emu_split_k_changes_no_bit(tile, shape, kind, pks):
    """k slices of whole 4096-deep super-chunks (a ragged last one included):
    each unit's exact fixed-point total joins one int64 total per element, which
    is rounded to FP64 once -- the sums an unsplit product forms, so every split
    gives the unsplit product's bits, and meets the oracle bar."""
    import torch
    cosma = lib()
    m, n, k = shape
    A, B = device_operands(m, n, k, DT, kind=kind, seed=23)
    out = []
    for pk in (1,) + pks:
        C, _ = out_tensor(m, n, DT)
        cosma.gemm(A, B, C, DT, plan=_split_plan(m, n, k, tile, pk))
        torch.cuda.synchronize()
        assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
        out.append(C.cpu().numpy())
    for got in out[1:]:
        assert np.array_equal(got, out[0])
    Ah, Bh = host_operands(m, n, k, DT, kind=kind, seed=23)
    assert og.normwise_rel_error(out[0], og.gemm(Ah, Bh, "dot2")) <= 1e-12


def test_emu_split_k_rejects_slices_shorter_than_a_super_chunk():
    import torch
    cosma = lib()
    m, n, k = 256, 256, 2 * 4096 + 1  # three super-chunks: at most three k slices
    A, B = device_operands(m, n, k, DT, seed=2)
    C, _ = out_tensor(m, n, DT)
    p = _split_plan(m, n, k, "pair256", 4)
    rc = cosma.cosma_gemm_planned(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n,
                                  cosma.COSMA_F64_EMU_BF16, p,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_ERR_INVALID_ARG
    p = _split_plan(m, n, k, "pair256", 3)
    p.order = 0
    p.pm = p.pn = 1
    p.ctas = 3
    rc = cosma.cosma_gemm_planned(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n,
                                  cosma.COSMA_F64_EMU_BF16, p,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_ERR_INVALID_ARG


@pytest.mark.parametrize("tile,pk", [("pair256", 1), ("single", 1), ("pair128", 1),
                                     ("pair256", 2)])
def test_emu_bounded_wait_reports_timeout_and_context_survives(tile, pk):
    """A wait limit of one cycle makes the emulation kernel's waits run out (the
    CTA pairs' lock-step rounds included): it must record COSMA_ERR_TIMEOUT, let
    the copies and products in flight land, free its tensor memory and exit; the
    next call with the default limit must be correct on the same context."""
    import torch
    cosma = lib()
    m, n, k = 1024, 1024, 4096 * pk
    A, B = device_operands(m, n, k, DT, seed=6)
    try:
        assert cosma.cosma_init(wait_limit=1) == 0
        C, _ = out_tensor(m, n, DT)
        cosma.gemm(A, B, C, DT, plan=_split_plan(m, n, k, tile, pk))
        st = cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream)
        assert st == cosma.COSMA_ERR_TIMEOUT
    finally:
        assert cosma.cosma_init(wait_limit=0) == 0
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT, plan=_split_plan(m, n, k, tile, pk))
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    rr, cc = sample_indices(m, n, 256, seed=3)
    ref, _, _, _, _ = sampled_reference(m, n, k, DT, rr, cc, seed=6)
    got = C[torch.as_tensor(rr, device="cuda"), torch.as_tensor(cc, device="cuda")].cpu().numpy()
    assert og.normwise_rel_error(got, ref) <= 1e-12
