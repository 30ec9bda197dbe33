"""GPU parity of cosma_zgemm (complex double C = alpha op(A) op(B) + beta C, run as
four real products) against the oracle's zgemm, through the C ABI.

Operands: real and imaginary parts from the shared generator (uniform [-1, 1),
seeds s and s + 1).  Bound, elementwise: |C_hat - C| <= 1e-12 |alpha| sum_t
|a_it| |b_tj| + 4 u (|alpha P| + |beta C0|), u = 2^-53: the real products meet
1e-12 relative to their row and column norms on either engine, and the complex
combination adds a few roundings.
"""
import numpy as np
import pytest

import cosma_inputs as ci
from gpu_util import lib
from oracle import gemm as og

pytestmark = pytest.mark.gpu


def _cmatrix(rows, cols, seed, stream):
    re = np.asarray(ci.matrix(rows, cols, "uniform", "f64", seed, stream), dtype=np.float64)
    im = np.asarray(ci.matrix(rows, cols, "uniform", "f64", seed + 1, stream), dtype=np.float64)
    return re + 1j * im


def _run(engine, m, n, k, op_a, op_b, alpha, beta, seed=7):
    import torch
    cosma = lib()
    Ah = _cmatrix(k, m, seed, ci.STREAM_A) if op_a else _cmatrix(m, k, seed, ci.STREAM_A)
    Bh = _cmatrix(n, k, seed, ci.STREAM_B) if op_b else _cmatrix(k, n, seed, ci.STREAM_B)
    C0 = _cmatrix(m, n, seed + 10, ci.STREAM_A)
    A = torch.tensor(Ah, dtype=torch.complex128, device="cuda")
    B = torch.tensor(Bh, dtype=torch.complex128, device="cuda")
    C = torch.tensor(C0, dtype=torch.complex128, device="cuda")
    cosma.gemm_complex(A, B, C, engine, alpha=alpha, beta=beta, op_a=op_a, op_b=op_b)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    return C.cpu().numpy(), Ah, Bh, C0


def _check(got, Ah, Bh, C0, alpha, beta, op_a, op_b):
    ref = og.zgemm(Ah, Bh, C0, alpha, beta, op_a, op_b)
    absA = np.abs(Ah.T if op_a else Ah)
    absB = np.abs(Bh.T if op_b else Bh)
    P = og.zgemm(Ah, Bh, C0, 1.0, 0.0, op_a, op_b)
    tol = (1e-12 * abs(alpha) * (absA @ absB) +
           4 * 2.0 ** -53 * (np.abs(alpha * P) + np.abs(beta * C0)) + 1e-300)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{bad.sum()} entries out of bound, first at {np.argwhere(bad)[0]}"


@pytest.mark.parametrize("op_a", [0, 1, 2])
@pytest.mark.parametrize("op_b", [0, 1, 2])
def test_zgemm_emulated_all_ops(op_a, op_b):
    m, n, k = 65, 70, 90
    alpha, beta = 0.5 - 0.25j, -1 + 2j
    got, Ah, Bh, C0 = _run("f64_emu_bf16", m, n, k, op_a, op_b, alpha, beta)
    _check(got, Ah, Bh, C0, alpha, beta, op_a, op_b)


@pytest.mark.parametrize("op_a,op_b", [(0, 0), (2, 1), (1, 2)])
def test_zgemm_native_f64(op_a, op_b):
    m, n, k = 130, 129, 257
    alpha, beta = 1.0, 0.0
    got, Ah, Bh, C0 = _run("f64", m, n, k, op_a, op_b, alpha, beta)
    _check(got, Ah, Bh, C0, alpha, beta, op_a, op_b)


def test_zgemm_beta_zero_ignores_nan_and_alpha_zero():
    import torch
    cosma = lib()
    m, n, k = 20, 30, 40
    A = torch.tensor(_cmatrix(m, k, 3, ci.STREAM_A), dtype=torch.complex128, device="cuda")
    B = torch.tensor(_cmatrix(k, n, 3, ci.STREAM_B), dtype=torch.complex128, device="cuda")
    C = torch.full((m, n), complex(float("nan"), 0), dtype=torch.complex128, device="cuda")
    cosma.gemm_complex(A, B, C, "f64_emu_bf16", alpha=1.0, beta=0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(C)).all()
    C0 = _cmatrix(m, n, 4, ci.STREAM_A)
    C2 = torch.tensor(C0, dtype=torch.complex128, device="cuda")
    cosma.gemm_complex(A, B, C2, "f64", alpha=0.0, beta=2j)
    torch.cuda.synchronize()
    assert np.array_equal(C2.cpu().numpy(), 2j * C0)
