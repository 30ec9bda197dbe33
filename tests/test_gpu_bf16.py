"""GPU parity of K-BF16 (tcgen05 + TMA + TMEM) against the oracle, through the
C ABI, plus the bounded-wait failure path.

Inputs are bf16 values (exact in f32/f64), so each product is exact in f32 and
only the f32 accumulation rounds: elementwise |C_hat - C| <= gamma_k |A||B| with
u = 2^-23 (one bit of slack for a truncating tensor-core adder).  Integer
inputs with |C| < 2^24 must be bit-exact.
"""
import numpy as np
import pytest

from oracle import gemm as og

from gpu_util import device_operands, host_operands, lib, out_tensor

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (7, 5, 3), (128, 256, 64), (127, 129, 127), (129, 257, 65),
          (200, 136, 1000), (512, 512, 512), (300, 700, 129), (1000, 7, 129), (64, 64, 1)]


def _gamma(k, u=2.0 ** -23):
    return k * u / (1 - k * u)


def _run(m, n, k, kind="uniform", seed=0, plan=None, lda=None, ldb=None, ldc=None):
    import torch
    cosma = lib()
    A, B = device_operands(m, n, k, "bf16", kind, seed, lda, ldb)
    C, _ = out_tensor(m, n, "bf16", ldc)
    cosma.gemm(A, B, C, "bf16", plan=plan)
    torch.cuda.synchronize()
    st = cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream)
    assert st == 0, cosma.status_string(st)
    return C.double().cpu().numpy()


def _check(C, m, n, k, kind="uniform", seed=0):
    A, B = host_operands(m, n, k, "bf16", kind, seed)
    ref = og.gemm(A, B, "dot2")
    if kind == "integer":
        assert np.array_equal(C, ref)
        return
    absref = og.gemm(np.abs(A), np.abs(B), "naive")
    bad = np.abs(C - ref) > _gamma(k) * absref * (1 + 1e-12) + 1e-300
    assert not bad.any(), f"{bad.sum()} entries out of bound, first at {np.argwhere(bad)[0]}"


@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_uniform(shape):
    m, n, k = shape
    _check(_run(m, n, k), m, n, k)


@pytest.mark.parametrize("shape", [(128, 256, 64), (255, 300, 777), (512, 512, 2048)])
def test_bf16_integer_bit_exact(shape):
    m, n, k = shape
    _check(_run(m, n, k, kind="integer", seed=4), m, n, k, kind="integer", seed=4)


def test_bf16_odd_leading_dimensions_pack_path():
    m, n, k = 150, 170, 133  # lda = 133 is not a multiple of 8: A is packed first
    _check(_run(m, n, k, lda=133, ldb=171, ldc=173), m, n, k)


@pytest.mark.parametrize("kind", ["integer", "uniform"])
@pytest.mark.parametrize("lda", [140001, 140008])
def test_bf16_far_apart_rows_read_through_k_blocked_copy(kind, lda):
    """Rows of A 280 KB apart (>= 256 KB) are read through a k-blocked copy
    [k/64][m][64]: ragged k (140001 = 2187 x 64 + 33, zero-filled), an odd pitch
    (element-wise copy) and a pitch of 8 elements (16-byte copy).  Integer inputs
    bit-exact, uniform ones within gamma_k |A||B|."""
    m, n, k = 130, 136, 140001
    _check(_run(m, n, k, kind=kind, seed=8, lda=lda), m, n, k, kind=kind, seed=8)


@pytest.mark.parametrize("tile_n,pk,order,ctas,pm,pn", [
    (256, 1, 1, 5, 1, 1), (128, 1, 1, 3, 1, 1), (256, 3, 1, 40, 1, 1), (128, 2, 0, 8, 2, 2),
    (256, 2, 0, 4, 2, 1)])
def test_bf16_forced_plans(tile_n, pk, order, ctas, pm, pn):
    cosma = lib()
    m, n, k = 300, 520, 700
    p = cosma.cosma_plan_query(m, n, k, cosma.COSMA_BF16)
    p.tile_n, p.pk, p.order, p.ctas, p.pm, p.pn = tile_n, pk, order, ctas, pm, pn
    _check(_run(m, n, k, plan=p), m, n, k)


def test_bf16_square_16384_sampled():
    import torch
    from gpu_util import sample_indices, sampled_reference
    cosma = lib()
    m = n = k = 16384
    A, B = device_operands(m, n, k, "bf16")
    C, _ = out_tensor(m, n, "bf16")
    cosma.gemm(A, B, C, "bf16")
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    rr, cc = sample_indices(m, n, 128, seed=3)
    ref, Ar, Bc, ri, cj = sampled_reference(m, n, k, "bf16", rr, cc)
    got = C[torch.as_tensor(rr, device="cuda"), torch.as_tensor(cc, device="cuda")]
    got = got.double().cpu().numpy()
    absref = np.einsum("ij,ij->i", np.abs(Ar[ri]), np.abs(Bc[cj]))
    assert np.all(np.abs(got - ref) <= _gamma(k) * absref)


def test_bounded_wait_reports_timeout_and_context_survives():
    """A wait limit of one cycle makes the tensor-core kernel's waits run out:
    it must record COSMA_ERR_TIMEOUT, drain and exit; the next call with the
    default limit must succeed on the same context."""
    import torch
    cosma = lib()
    try:
        assert cosma.cosma_init(wait_limit=1) == 0
        A, B = device_operands(1024, 1024, 4096, "bf16")
        C, _ = out_tensor(1024, 1024, "bf16")
        cosma.gemm(A, B, C, "bf16")
        st = cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream)
        assert st == cosma.COSMA_ERR_TIMEOUT
    finally:
        assert cosma.cosma_init(wait_limit=0) == 0
    m, n, k = 256, 384, 320
    _check(_run(m, n, k, seed=9), m, n, k, seed=9)


@pytest.mark.parametrize("kind", ["uniform", "integer"])
def test_bf16_b_loaded_directly_or_transposed(kind):
    """ldb % 8 == 0 loads B as it is (MN-major operand); an odd ldb transposes it
    into the workspace first (K-major).  Both meet the bound; integer inputs agree
    bit for bit."""
    m, n, k = 300, 520, 700
    Cd = _run(m, n, k, kind=kind, seed=6)              # ldb = 520: direct
    Ct = _run(m, n, k, kind=kind, seed=6, ldb=521)     # transposed
    _check(Cd, m, n, k, kind=kind, seed=6)
    _check(Ct, m, n, k, kind=kind, seed=6)
    if kind == "integer":
        assert np.array_equal(Cd, Ct)
