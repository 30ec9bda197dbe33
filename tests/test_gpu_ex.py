"""GPU parity of cosma_gemm_ex (C = alpha op(A) op(B) + beta C) against the oracle's
gemm_ex, through the C ABI, for every dtype and all four transpose cases.

Bound, elementwise: |C_hat - C| <= |alpha| err_prod + 4 u_out (|alpha P| + |beta C0|),
err_prod being each path's product bound -- gamma_k |A||B| for the FMA and bf16
paths (u = 2^-53 / 2^-24 / 2^-23), 1e-12 ||a_i|| ||b_j|| for the FP64 emulation,
(1.002 gamma_3k(2^-23) + 3.01 2^-22) |A||B| for three TF32 products -- and
u_out the unit roundoff of C's type (alpha and beta are applied in it).  alpha and
beta are chosen exactly representable in f32.
"""
import numpy as np
import pytest

from gpu_util import OUT_DT, device_operands, host_operands, lib
from oracle import gemm as og

pytestmark = pytest.mark.gpu

DTYPES = ["f64", "f32", "bf16", "f64_emu_bf16", "f32_emu_tf32"]
U_PROD = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -23}
U_OUT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24, "f64_emu_bf16": 2.0 ** -53,
         "f32_emu_tf32": 2.0 ** -24}


def _operands(m, n, k, dtype, ta, tb, seed):
    """Device storage (transposed when asked) and the host copies of it."""
    import torch
    A, B = device_operands(m, n, k, dtype, "uniform", seed)
    Ah, Bh = host_operands(m, n, k, dtype, "uniform", seed)
    if ta:
        A, Ah = A.t().contiguous(), np.ascontiguousarray(Ah.T)
    if tb:
        B, Bh = B.t().contiguous(), np.ascontiguousarray(Bh.T)
    return A, B, Ah, Bh


def _c0(m, n, dtype, seed):
    import torch
    rng = np.random.default_rng(seed)
    C0 = rng.uniform(-1, 1, (m, n))
    tdt = getattr(torch, OUT_DT[dtype])
    C = torch.tensor(C0, dtype=tdt, device="cuda")
    return C, C.double().cpu().numpy()


def _bound(dtype, Ah, Bh, ta, tb, C0, alpha, beta):
    opA = Ah.T if ta else Ah
    opB = Bh.T if tb else Bh
    k = opA.shape[1]
    P = og.gemm(opA, opB, "dot2")
    if dtype == "f64_emu_bf16":
        prod = 1e-12 * np.sqrt((opA ** 2).sum(1))[:, None] * np.sqrt((opB ** 2).sum(0))[None, :]
    elif dtype == "f32_emu_tf32":
        g = 3 * k * 2.0 ** -23 / (1 - 3 * k * 2.0 ** -23)
        prod = (1.002 * g + 3.01 * 2.0 ** -22) * og.gemm(np.abs(opA), np.abs(opB), "naive")
    else:
        u = U_PROD[dtype]
        prod = (k * u / (1 - k * u)) * og.gemm(np.abs(opA), np.abs(opB), "naive")
    return abs(alpha) * prod + 4 * U_OUT[dtype] * (np.abs(alpha * P) + np.abs(beta * C0)) + 1e-300


def _run(dtype, m, n, k, ta, tb, alpha, beta, seed=3):
    import torch
    cosma = lib()
    A, B, Ah, Bh = _operands(m, n, k, dtype, ta, tb, seed)
    C, C0 = _c0(m, n, dtype, seed + 100)
    cosma.gemm_ex(A, B, C, dtype, alpha=alpha, beta=beta, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    return C.double().cpu().numpy(), Ah, Bh, C0


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.75, 1.5), (0.5, -2.0)])
def test_gemm_ex_matches_oracle(dtype, ta, tb, alpha, beta):
    m, n, k = 129, 200, 131
    got, Ah, Bh, C0 = _run(dtype, m, n, k, ta, tb, alpha, beta)
    ref = og.gemm_ex(Ah, Bh, C0, alpha, beta, bool(ta), bool(tb))
    tol = _bound(dtype, Ah, Bh, ta, tb, C0, alpha, beta)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{bad.sum()} entries out of bound, first at {np.argwhere(bad)[0]}"


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f32_emu_tf32", "f64_emu_bf16"])
def test_gemm_ex_split_k_reduce_applies_alpha_beta(dtype):
    cosma = lib()
    m, n, k = 96, 80, 6000  # emulated FP64: two 4096-deep super-chunks, one per k slice
    plan = cosma.cosma_plan_query(m, n, k, cosma.DTYPES[dtype])
    assert plan.pk > 1  # the Reduce (emulation: the finishing pass) applies alpha and beta
    got, Ah, Bh, C0 = _run(dtype, m, n, k, 1, 0, -1.25, 0.5)
    ref = og.gemm_ex(Ah, Bh, C0, -1.25, 0.5, True, False)
    assert np.all(np.abs(got - ref) <= _bound(dtype, Ah, Bh, 1, 0, C0, -1.25, 0.5))


@pytest.mark.parametrize("dtype", DTYPES)
def test_gemm_ex_beta_zero_ignores_nan_and_alpha_zero_scales(dtype):
    import torch
    cosma = lib()
    m, n, k = 70, 90, 50
    A, B, Ah, Bh = _operands(m, n, k, dtype, 0, 0, 5)
    tdt = getattr(torch, OUT_DT[dtype])
    C = torch.full((m, n), float("nan"), dtype=tdt, device="cuda")
    cosma.gemm_ex(A, B, C, dtype, alpha=1.0, beta=0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(C).all()
    # alpha == 0: C = beta C, A and B not read (null pointers accepted)
    C2, C0 = _c0(m, n, dtype, 9)
    rc = cosma.cosma_gemm_ex(0, 0, m, n, k, 0.0, 0, k, 0, n, -0.5, C2.data_ptr(), n,
                             cosma.DTYPES[dtype], torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_OK
    torch.cuda.synchronize()
    assert np.array_equal(C2.double().cpu().numpy(), -0.5 * C0)
    # k == 0: C = beta C
    C3, C0 = _c0(m, n, dtype, 10)
    rc = cosma.cosma_gemm_ex(1, 1, m, n, 0, 2.0, 0, m, 0, 1, 2.0, C3.data_ptr(), n,
                             cosma.DTYPES[dtype], torch.cuda.current_stream().cuda_stream)
    assert rc == cosma.COSMA_OK
    torch.cuda.synchronize()
    assert np.array_equal(C3.double().cpu().numpy(), 2.0 * C0)
