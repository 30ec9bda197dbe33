"""GPU parity of the native FP64 / FP32 paths (K-F64, K-F32, Reduce) against
the oracle, through the C ABI.

Tolerances: FP64 normwise relative error <= 1e-13 against the Dot2 oracle;
integer-valued inputs bit-exact in FP64 and FP32.  FP32 elementwise within the
classical bound |C_hat - C| <= gamma_k |A||B| (gamma_k = k u / (1 - k u),
u = 2^-24), which holds for any summation order with or without FMA.
"""
import numpy as np
import pytest

from oracle import gemm as og

from gpu_util import (device_operands, host_operands, lib, out_tensor, sample_indices,
                      sampled_reference)

pytestmark = pytest.mark.gpu

SMALL = [(1, 1, 1), (7, 5, 3), (127, 129, 127), (129, 127, 129), (1000, 7, 129),
         (7, 1000, 129), (200, 136, 1000), (512, 512, 512), (64, 64, 1)]


def _run(m, n, k, dtype, kind="uniform", seed=0, plan=None, lda=None, ldb=None, ldc=None):
    import torch
    cosma = lib()
    A, B = device_operands(m, n, k, dtype, kind, seed, lda, ldb)
    C, _ = out_tensor(m, n, dtype, ldc)
    cosma.gemm(A, B, C, dtype, plan=plan)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    return C.double().cpu().numpy()


def _gamma(k, u):
    return k * u / (1 - k * u)


@pytest.mark.parametrize("shape", SMALL)
def test_f64_uniform_small(shape):
    m, n, k = shape
    C = _run(m, n, k, "f64")
    A, B = host_operands(m, n, k, "f64")
    ref = og.gemm(A, B, "dot2")
    assert og.normwise_rel_error(C, ref) <= 1e-13


def test_f64_config_512_seed0():
    # the 512^3 uniform[-1,1) seed-0 configuration, full comparison
    C = _run(512, 512, 512, "f64", seed=0)
    A, B = host_operands(512, 512, 512, "f64", seed=0)
    ref = og.gemm(A, B, "dot2")
    err = og.normwise_rel_error(C, ref)
    assert err <= 1e-13, err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(127, 129, 127), (512, 512, 512), (33, 1000, 777)])
def test_integer_inputs_bit_exact(dtype, shape):
    m, n, k = shape
    C = _run(m, n, k, dtype, kind="integer", seed=3)
    A, B = host_operands(m, n, k, dtype, kind="integer", seed=3)
    ref = og.gemm(A, B, "naive")  # exact: |C| <= 64 k < 2^24
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("shape", SMALL)
def test_f32_uniform_small(shape):
    m, n, k = shape
    C = _run(m, n, k, "f32")
    A, B = host_operands(m, n, k, "f32")
    ref = og.gemm(A, B, "dot2")
    absref = og.gemm(np.abs(A), np.abs(B), "naive")
    assert np.all(np.abs(C - ref) <= _gamma(k, 2.0 ** -24) * absref * (1 + 1e-12) + 1e-300)


def test_k_zero_sets_c_to_zero():
    for dt in ("f64", "f32"):
        C = _run(9, 11, 0, dt)
        assert C.shape == (9, 11) and not C.any()


def test_padded_leading_dimensions():
    m, n, k = 100, 70, 90
    C = _run(m, n, k, "f64", lda=97, ldb=75, ldc=81)
    A, B = host_operands(m, n, k, "f64")
    assert og.normwise_rel_error(C, og.gemm(A, B, "dot2")) <= 1e-13


def _forced_plan(m, n, k, dtype, tile, pk, order, ctas, pm=1, pn=1):
    cosma = lib()
    p = cosma.cosma_plan_query(m, n, k, cosma.DTYPES[dtype])
    kb = p.k_block
    p.tile_m, p.tile_n = tile
    p.pk, p.order, p.ctas, p.pm, p.pn = pk, order, ctas, pm, pn
    p.k_block = kb
    return p


# two tiles of each family: FP64 128 x 128 / 64 x 64, FP32 128 x 128 / 256 x 128 (the
# FP32 128 x 256 tile has its own tests below)
TILES = {"f64": [(128, 128), (64, 64)], "f32": [(128, 128), (256, 128)]}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("ti,pk,order,ctas,pm,pn", [
    (0, 1, 1, 7, 1, 1), (0, 3, 1, 20, 1, 1), (1, 2, 0, 2 * 2 * 2, 2, 2),
    (1, 5, 1, 148, 1, 1), (0, 2, 0, 2 * 1 * 2, 2, 1)])
def test_forced_plans_split_k_and_orders(dtype, ti, pk, order, ctas, pm, pn):
    m, n, k = 300, 260, 515
    p = _forced_plan(m, n, k, dtype, TILES[dtype][ti], pk, order, ctas, pm, pn)
    C = _run(m, n, k, dtype, plan=p)
    A, B = host_operands(m, n, k, dtype)
    ref = og.gemm(A, B, "dot2")
    if dtype == "f64":
        assert og.normwise_rel_error(C, ref) <= 1e-13
    else:
        absref = og.gemm(np.abs(A), np.abs(B), "naive")
        assert np.all(np.abs(C - ref) <= _gamma(k, 2.0 ** -24) * absref * (1 + 1e-12))


@pytest.mark.parametrize("pk,order,ctas,pm,pn", [(1, 1, 7, 1, 1), (3, 1, 20, 1, 1),
                                                  (2, 0, 2 * 2 * 2, 2, 2), (5, 1, 148, 1, 1)])
@pytest.mark.parametrize("vec", [True, False])
def test_f32_wide_tile_forced_plans(pk, order, ctas, pm, pn, vec):
    # 128 x 256 tiles (16 columns per thread); ragged m, n, k; unaligned pitches
    # take the 4-byte copies
    m, n, k = 300, 520, 515
    p = _forced_plan(m, n, k, "f32", (128, 256), pk, order, ctas, pm, pn)
    C = _run(m, n, k, "f32", plan=p, lda=None if vec else 517, ldb=None if vec else 523)
    A, B = host_operands(m, n, k, "f32")
    ref = og.gemm(A, B, "dot2")
    absref = og.gemm(np.abs(A), np.abs(B), "naive")
    assert np.all(np.abs(C - ref) <= _gamma(k, 2.0 ** -24) * absref * (1 + 1e-12))


def test_f32_wide_tile_integer_bit_exact():
    m, n, k = 257, 600, 333
    p = _forced_plan(m, n, k, "f32", (128, 256), 1, 1, 10)
    C = _run(m, n, k, "f32", kind="integer", seed=3, plan=p)
    A, B = host_operands(m, n, k, "f32", kind="integer", seed=3)
    assert np.array_equal(C, og.gemm(A, B, "naive"))


def test_invalid_plan_rejected():
    import torch
    cosma = lib()
    p = cosma.cosma_plan_query(64, 64, 64, cosma.COSMA_F64)
    p.tile_m = 96
    A, B = device_operands(64, 64, 64, "f64")
    C, _ = out_tensor(64, 64, "f64")
    rc = cosma.cosma_gemm_planned(64, 64, 64, A.data_ptr(), 64, B.data_ptr(), 64, C.data_ptr(),
                                  64, cosma.COSMA_F64, p, torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_ERR_INVALID_ARG


def test_device_generator_matches_host():
    import torch
    import cosma_inputs as ci
    from cosma_inputs import device as cid
    for kind in ("uniform", "integer", "loguniform"):
        for g in ("f64", "f32", "bf16"):
            t = cid.new(37, 301, kind, g, seed=77, stream_id=5)
            h = ci.matrix(37, 301, kind, g, seed=77, stream=5)
            if g == "bf16":
                assert torch.equal(t.cpu(), h)
            else:
                assert np.array_equal(t.cpu().numpy(), h)


# ---- full-size configurations (sampled entries, launch config of the bench) ----

FULL = {"square": (16384, 16384, 16384), "largeK": (4096, 4096, 1 << 20),
        "largeM": (1 << 20, 4096, 4096), "flat": (65536, 65536, 1024)}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("family", list(FULL))
def test_full_size_sampled(dtype, family):
    import torch
    m, n, k = FULL[family]
    cosma = lib()
    A, B = device_operands(m, n, k, dtype, seed=0)
    C, _ = out_tensor(m, n, dtype)
    cosma.gemm(A, B, C, dtype)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    del A, B
    rr, cc = sample_indices(m, n, 96, seed=list(FULL).index(family) + 10)
    ref, Ar, Bc, ri, cj = sampled_reference(m, n, k, dtype, rr, cc)
    got = C[torch.as_tensor(rr, device="cuda"), torch.as_tensor(cc, device="cuda")]
    got = got.double().cpu().numpy()
    del C
    torch.cuda.empty_cache()
    if dtype == "f64":
        assert og.normwise_rel_error(got, ref) <= 1e-13
    else:
        absref = np.einsum("ij,ij->i", np.abs(Ar[ri]), np.abs(Bc[cj]))
        assert np.all(np.abs(got - ref) <= _gamma(k, 2.0 ** -24) * absref)


@pytest.mark.parametrize("shape,lda,ldb,ldc", [((129, 260, 1000), None, None, None),
                                               ((300, 260, 1001), 1004, 264, 268),
                                               ((1, 4, 3), 4, None, None)])
def test_f32_aligned_ragged_async_path(shape, lda, ldb, ldc):
    # 16-byte aligned rows take the cp.async ring; ragged m, n, k are zero-filled
    m, n, k = shape
    C = _run(m, n, k, "f32", lda=lda, ldb=ldb, ldc=ldc)
    A, B = host_operands(m, n, k, "f32")
    ref = og.gemm(A, B, "dot2")
    absref = og.gemm(np.abs(A), np.abs(B), "naive")
    assert np.all(np.abs(C - ref) <= _gamma(k, 2.0 ** -24) * absref * (1 + 1e-12) + 1e-300)
