"""GPU parity of cosma_zgemm and cosma_cgemm (complex double / single
C = alpha op(A) op(B) + beta C, run as four real products) against the oracle's
zgemm (complex128; single-precision operands are rounded to complex64 first),
through the C ABI.  The single-precision bound is stated at _check_c.

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


# ---- complex single (cosma_cgemm) ----------------------------------------------

def _run_c(engine, m, n, k, op_a, op_b, alpha, beta, seed=7):
    import torch
    cosma = lib()
    Ah = _cmatrix(k, m, seed, ci.STREAM_A) if op_a else _cmatrix(m, k, seed, ci.STREAM_A)
    Bh = _cmatrix(n, k, seed, ci.STREAM_B) if op_b else _cmatrix(k, n, seed, ci.STREAM_B)
    C0 = _cmatrix(m, n, seed + 10, ci.STREAM_A)
    Ah, Bh, C0 = (x.astype(np.complex64).astype(np.complex128) for x in (Ah, Bh, C0))
    A = torch.tensor(Ah, dtype=torch.complex64, device="cuda")
    B = torch.tensor(Bh, dtype=torch.complex64, device="cuda")
    C = torch.tensor(C0, dtype=torch.complex64, device="cuda")
    cosma.gemm_complex(A, B, C, engine, alpha=alpha, beta=beta, op_a=op_a, op_b=op_b)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    return C.cpu().numpy().astype(np.complex128), Ah, Bh, C0


def _check_c(engine, got, Ah, Bh, C0, alpha, beta, op_a, op_b):
    """Per real product e |X||Y| (FMA: gamma_k(2^-24); three TF32 products:
    1.002 gamma_3k(2^-23) + 3.01 2^-22), over the four products and the f32
    roundings of their combination: elementwise
    (e + 4u) |alpha| (|Ar| + |Ai|)(|Br| + |Bi|) + 4u (|alpha P| + |beta C0|), u = 2^-24;
    and, for TF32, 1e-5 normwise (a dropped correction term is ~2^-12)."""
    ref = og.zgemm(Ah, Bh, C0, alpha, beta, op_a, op_b)
    opA = Ah.T if op_a else Ah
    opB = Bh.T if op_b else Bh
    k = opA.shape[1]
    u = 2.0 ** -24
    if engine == "f32":
        e = k * u / (1 - k * u)
    else:
        g = 3 * k * 2.0 ** -23 / (1 - 3 * k * 2.0 ** -23)
        e = 1.002 * g + 3.01 * 2.0 ** -22
    mag = (np.abs(opA.real) + np.abs(opA.imag)) @ (np.abs(opB.real) + np.abs(opB.imag))
    P = og.zgemm(Ah, Bh, C0, 1.0, 0.0, op_a, op_b)
    tol = (e + 4 * u) * abs(alpha) * mag + 4 * u * (np.abs(alpha * P) + np.abs(beta * C0)) + 1e-30
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{bad.sum()} entries out of bound, first at {np.argwhere(bad)[0]}"
    if engine == "f32_emu_tf32":
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("op_a", [0, 1, 2])
@pytest.mark.parametrize("op_b", [0, 1, 2])
def test_cgemm_tf32_all_ops(op_a, op_b):
    m, n, k = 65, 70, 90
    alpha, beta = 0.5 - 0.25j, -1 + 2j
    got, Ah, Bh, C0 = _run_c("f32_emu_tf32", m, n, k, op_a, op_b, alpha, beta)
    _check_c("f32_emu_tf32", got, Ah, Bh, C0, alpha, beta, op_a, op_b)


@pytest.mark.parametrize("engine", ["f32", "f32_emu_tf32"])
@pytest.mark.parametrize("op_a,op_b", [(0, 0), (2, 1), (1, 2)])
def test_cgemm_engines_larger(engine, op_a, op_b):
    m, n, k = 300, 257, 1100
    alpha, beta = 1.0, 0.0
    got, Ah, Bh, C0 = _run_c(engine, m, n, k, op_a, op_b, alpha, beta)
    _check_c(engine, got, Ah, Bh, C0, alpha, beta, op_a, op_b)


def test_cgemm_beta_zero_ignores_nan_and_alpha_zero():
    import torch
    cosma = lib()
    m, n, k = 20, 30, 40
    A = torch.tensor(_cmatrix(m, k, 3, ci.STREAM_A), dtype=torch.complex64, device="cuda")
    B = torch.tensor(_cmatrix(k, n, 3, ci.STREAM_B), dtype=torch.complex64, device="cuda")
    C = torch.full((m, n), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    cosma.gemm_complex(A, B, C, "f32_emu_tf32", alpha=1.0, beta=0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(C)).all()
    C0 = _cmatrix(m, n, 4, ci.STREAM_A).astype(np.complex64)
    C2 = torch.tensor(C0, dtype=torch.complex64, device="cuda")
    cosma.gemm_complex(A, B, C2, "f32", alpha=0.0, beta=2j)
    torch.cuda.synchronize()
    assert np.array_equal(C2.cpu().numpy(), (2j * C0).astype(np.complex64))
