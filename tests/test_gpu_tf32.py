"""GPU parity of the FP32 path built from three TF32 products (COSMA_F32_EMU_TF32)
against the oracle, through the C ABI.

Each operand entry x is split into h = tf32(x) and l = tf32(x - h), both rounded
to nearest (unit roundoff 2^-11), so |x - h - l| <= 2^-22 |x|; C is accumulated
in fp32 on the tensor cores from h_a h_b + h_a l_b + l_a h_b.  The dropped terms
(l_a l_b and the two split remainders) stay below 3.01 2^-22 |a||b| per product,
and 3k fp32 additions with at most 2^-23 relative error each (the accumulator
may truncate) add gamma_3k(2^-23) (1.002 |a||b|).  So, elementwise,

    |C_hat - C| <= (1.002 gamma_3k(2^-23) + 3.01 2^-22) |A||B|.

That bound does not notice a missing correction term at small k, so a second,
normwise check asks for 1e-5: one TF32 product alone is off by about 2^-12.
Integer inputs of at most 11 significant bits are exact in TF32 (l = 0) and
their products and sums stay below 2^24, so they are bit-exact.
"""
import numpy as np
import pytest

from gpu_util import device_operands, host_operands, lib, out_tensor, sample_indices
from oracle import gemm as og

pytestmark = pytest.mark.gpu

DT = "f32_emu_tf32"
SHAPES = [(1, 1, 1), (7, 5, 3), (127, 129, 127), (129, 257, 129), (1000, 7, 129),
          (7, 1000, 33), (200, 136, 1000), (512, 512, 512), (64, 64, 1), (300, 260, 4097)]


def _run(m, n, k, kind="uniform", seed=0, plan=None, lda=None, ldb=None, ldc=None):
    import torch
    cosma = lib()
    A, B = device_operands(m, n, k, DT, kind, seed, lda, ldb)
    C, _ = out_tensor(m, n, DT, ldc)
    cosma.gemm(A, B, C, DT, plan=plan)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    return C.double().cpu().numpy()


def bound(A, B):
    k = A.shape[1]
    g = 3 * k * 2.0 ** -23 / (1 - 3 * k * 2.0 ** -23)
    return (1.002 * g + 3.01 * 2.0 ** -22) * og.gemm(np.abs(A), np.abs(B), "naive") + 1e-300


def _check(C, A, B):
    ref = og.gemm(A, B, "dot2")
    bad = np.abs(C - ref) > bound(A, B)
    assert not bad.any(), f"{bad.sum()} entries out of bound, first at {np.argwhere(bad)[0]}"
    if ref.size and np.abs(ref).max() > 0:
        assert og.normwise_rel_error(C, ref) <= 1e-5


@pytest.mark.parametrize("shape", SHAPES)
def test_tf32x3_uniform(shape):
    m, n, k = shape
    C = _run(m, n, k)
    A, B = host_operands(m, n, k, DT)
    _check(C, A, B)


@pytest.mark.parametrize("shape", [(127, 129, 127), (512, 512, 512), (33, 1000, 777)])
def test_tf32x3_integer_inputs_bit_exact(shape):
    m, n, k = shape
    C = _run(m, n, k, kind="integer", seed=3)
    A, B = host_operands(m, n, k, DT, kind="integer", seed=3)
    assert np.array_equal(C, og.gemm(A, B, "naive"))


def test_tf32x3_wide_exponent_range():
    # log-uniform magnitudes: the lo parts carry most of the correction
    m, n, k = 257, 130, 300
    C = _run(m, n, k, kind="loguniform", seed=5)
    A, B = host_operands(m, n, k, DT, kind="loguniform", seed=5)
    _check(C, A, B)


def test_tf32x3_more_accurate_than_one_tf32_product():
    import torch
    m, n, k = 256, 256, 2048
    C = _run(m, n, k, seed=11)
    A, B = host_operands(m, n, k, DT, seed=11)
    ref = og.gemm(A, B, "dot2")
    # one product of the TF32 roundings alone, formed exactly on the host
    At = torch.tensor(A, dtype=torch.float32)
    Bt = torch.tensor(B, dtype=torch.float32)
    h = lambda x: (x.view(torch.int32) + 0x1000).bitwise_and(-0x2000).view(torch.float32)
    one = og.gemm(h(At).double().numpy(), h(Bt).double().numpy(), "dot2")
    e3 = og.normwise_rel_error(C, ref)
    e1 = og.normwise_rel_error(one, ref)
    assert e3 < e1 / 50, (e3, e1)


def test_tf32x3_padded_leading_dimensions():
    m, n, k = 100, 70, 90
    C = _run(m, n, k, lda=97, ldb=75, ldc=81)
    A, B = host_operands(m, n, k, DT)
    _check(C, A, B)


def test_tf32x3_k_zero_sets_c_to_zero():
    C = _run(9, 11, 0)
    assert C.shape == (9, 11) and not C.any()


def _forced_plan(m, n, k, tile, pk, order, ctas, pm=1, pn=1):
    cosma = lib()
    p = cosma.cosma_plan_query(m, n, k, cosma.DTYPES[DT])
    assert cosma.KERNELS[p.kernel] == "tf32x3"
    p.tile_m, p.tile_n = tile
    p.pk, p.order, p.ctas, p.pm, p.pn = pk, order, ctas, pm, pn
    return p


@pytest.mark.parametrize("pk,order,ctas,pm,pn", [
    (1, 1, 7, 1, 1), (3, 1, 20, 1, 1), (2, 0, 2 * 2 * 2, 2, 2), (5, 1, 148, 1, 1),
    (17, 1, 152, 1, 1)])
def test_tf32x3_forced_plans(pk, order, ctas, pm, pn):
    # odd k-block counts per unit leave a one-block last segment
    m, n, k = 300, 520, 515
    p = _forced_plan(m, n, k, (128, 128), pk, order, ctas, pm, pn)
    C = _run(m, n, k, plan=p)
    A, B = host_operands(m, n, k, DT)
    _check(C, A, B)


def test_tf32x3_full_size_sampled():
    # 16384^3 in the launch configuration the benchmark times; sampled entries
    import torch
    from gpu_util import sampled_reference
    cosma = lib()
    m = n = k = 16384
    A, B = device_operands(m, n, k, DT, "uniform", 0)
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    rr, cc = sample_indices(m, n, 128, seed=4)
    ref, Ar, Bc, ri, cj = sampled_reference(m, n, k, DT, rr, cc)
    got = C[torch.as_tensor(rr, device="cuda"), torch.as_tensor(cc, device="cuda")]
    got = got.double().cpu().numpy()
    absref = np.einsum("ij,ij->i", np.abs(Ar[ri]), np.abs(Bc[cj]))
    g = 3 * k * 2.0 ** -23 / (1 - 3 * k * 2.0 ** -23)
    assert np.all(np.abs(got - ref) <= (1.002 * g + 3.01 * 2.0 ** -22) * absref)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("shape", [(1, 1, 1), (200, 136, 300), (513, 257, 1031)])
def test_tf32x3_host_path_equals_device_path(shape):
    import torch
    cosma = lib()
    m, n, k = shape
    A, B = device_operands(m, n, k, DT, "uniform", 0)
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT)
    Ah = A.cpu().pin_memory()
    Bh = B.cpu().pin_memory()
    Ch = torch.full((m, n), float("nan"), dtype=torch.float32).pin_memory()
    cosma.gemm_host(Ah, Bh, Ch, DT)
    torch.cuda.synchronize()
    assert torch.equal(Ch, C.cpu())


_SUB = """
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import cosma_inputs as ci
from cosma_inputs import device as cid
from paper_1908_09606_gb300 import cosma
cosma.load()
m, n, k = {m}, {n}, {k}
A = cid.new(m, k, "uniform", "f32", seed=2, stream_id=ci.STREAM_A)
B = cid.new(k, n, "uniform", "f32", seed=2, stream_id=ci.STREAM_B)
C = torch.empty((m, n), dtype=torch.float32, device="cuda")
cosma.gemm(A, B, C, "f32_emu_tf32")
torch.cuda.synchronize()
assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
np.save({out!r}, C.cpu().numpy())
"""


def test_tf32x3_lockstep_ticks_do_not_change_results(tmp_path):
    """Lock-step ticks (default: cooperative launch), ticks under a plain launch
    (COSMA_TF32_LOCKSTEP=2) and free CTAs (=0) only reorder the loads: every
    entry's sum is formed in the same order, so the results are bit-equal."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    m, n, k = 1100, 1536, 2500   # 108 tiles on 152 SMs, 79 k blocks = 3 ticks
    outs = []
    for mode in ("1", "2", "0"):
        out = str(tmp_path / f"c{mode}.npy")
        code = _SUB.format(root=root, m=m, n=n, k=k, out=out)
        env = dict(os.environ, COSMA_TF32_LOCKSTEP=mode)
        subprocess.run([sys.executable, "-c", code], env=env, cwd=root, check=True,
                       timeout=600)
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    A, B = host_operands(m, n, k, DT, seed=2)
    _check(outs[0].astype(np.float64), A, B)


def test_tf32x3_bounded_wait_reports_timeout_and_context_survives():
    import torch
    cosma = lib()
    try:
        assert cosma.cosma_init(wait_limit=1) == 0
        A, B = device_operands(1024, 1024, 4096, DT)
        C, _ = out_tensor(1024, 1024, DT)
        cosma.gemm(A, B, C, DT)
        st = cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream)
        assert st == cosma.COSMA_ERR_TIMEOUT
    finally:
        assert cosma.cosma_init(wait_limit=0) == 0
    C = _run(256, 384, 320, seed=9)
    A, B = host_operands(256, 384, 320, DT, seed=9)
    _check(C, A, B)


def test_tf32x3_nonfinite_inputs_give_nonfinite_entries():
    """An Inf or NaN in A or B makes exactly the entries non-finite that an IEEE
    product makes non-finite (every operand entry here is nonzero); an Inf may come
    out as NaN (Inf times a zero or opposite-signed lo part).  The other entries
    stay within the bound."""
    import torch
    cosma = lib()
    m, n, k = 130, 140, 150
    A, B = device_operands(m, n, k, DT, "uniform", 4)
    A[3, 17] = float("inf")
    A[5, 40] = float("nan")
    B[99, 7] = float("-inf")
    C, _ = out_tensor(m, n, DT)
    cosma.gemm(A, B, C, DT)
    torch.cuda.synchronize()
    got = C.double().cpu().numpy()
    bad = np.zeros((m, n), dtype=bool)
    bad[3, :] = bad[5, :] = True
    bad[:, 7] = True
    assert not np.isfinite(got[bad]).any()
    Ah = A.double().cpu().numpy()
    Bh = B.double().cpu().numpy()
    Ah[3, 17] = Ah[5, 40] = 0.0
    Bh[99, 7] = 0.0
    ref = og.gemm(Ah, Bh, "dot2")
    tol = bound(Ah, Bh)
    assert np.all(np.abs(got[~bad] - ref[~bad]) <= tol[~bad])
