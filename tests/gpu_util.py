"""Helpers shared by the GPU parity tests: device inputs from the shared
generator, oracle references for full products or sampled entries."""
import numpy as np

import cosma_inputs as ci
from oracle import gemm as og

TORCH_DT = {"f64": "float64", "f32": "float32", "bf16": "bfloat16"}
# operand element type generated for each library dtype
GEN_DT = {"f64": "f64", "f32": "f32", "bf16": "bf16", "f64_emu_bf16": "f64",
          "f32_emu_tf32": "f32"}
OUT_DT = {"f64": "float64", "f32": "float32", "bf16": "float32", "f64_emu_bf16": "float64",
          "f32_emu_tf32": "float32"}


def lib():
    from paper_1908_09606_gb300 import cosma
    cosma.load()
    return cosma


def device_operands(m, n, k, dtype, kind="uniform", seed=0, lda=None, ldb=None):
    """A (m x k) and B (k x n) on the device, optionally inside wider storage."""
    import torch
    from cosma_inputs import device as cid
    g = GEN_DT[dtype]
    tdt = getattr(torch, TORCH_DT[g])
    Ast = torch.zeros((m, lda or max(k, 1)), dtype=tdt, device="cuda")
    Bst = torch.zeros((k, ldb or max(n, 1)), dtype=tdt, device="cuda")
    A = Ast[:, :k]
    B = Bst[:, :n]
    if m and k:
        cid.fill(A, kind, g, seed, ci.STREAM_A)
    if k and n:
        cid.fill(B, kind, g, seed, ci.STREAM_B)
    return A, B


def host_operands(m, n, k, dtype, kind="uniform", seed=0):
    g = GEN_DT[dtype]
    A = ci.matrix(m, k, kind, g, seed, ci.STREAM_A)
    B = ci.matrix(k, n, kind, g, seed, ci.STREAM_B)
    if g == "bf16":
        A = A.float().numpy()
        B = B.float().numpy()
    return np.asarray(A, dtype=np.float64), np.asarray(B, dtype=np.float64)


def out_tensor(m, n, dtype, ldc=None, fill=float("nan")):
    import torch
    tdt = getattr(torch, OUT_DT[dtype])
    Cst = torch.full((m, ldc or max(n, 1)), fill, dtype=tdt, device="cuda")
    return Cst[:, :n], Cst


def sample_indices(m, n, count, seed, tile=128):
    """Rows/cols hitting tile edges and ragged tails, plus random entries."""
    rng = np.random.default_rng(seed)
    edge_r = sorted({0, 1, tile - 1, tile, m // 2, m - 2, m - 1} & set(range(m)))
    edge_c = sorted({0, 1, tile - 1, tile, 255, 256, n // 2, n - 2, n - 1} & set(range(n)))
    rr = [r for r in edge_r for _ in edge_c]
    cc = [c for _ in edge_r for c in edge_c]
    rr += list(rng.integers(0, m, count))
    cc += list(rng.integers(0, n, count))
    return np.array(rr, dtype=np.int64), np.array(cc, dtype=np.int64)


def sampled_reference(m, n, k, dtype, rr, cc, kind="uniform", seed=0):
    """Dot2 oracle values C[rr[i], cc[i]] regenerating only the needed rows/cols."""
    g = GEN_DT[dtype]
    ur, ri = np.unique(rr, return_inverse=True)
    uc, cj = np.unique(cc, return_inverse=True)
    Ar = ci.rows(ur, k, kind, g, seed, ci.STREAM_A)
    Bc = ci.cols(uc, k, n, kind, g, seed, ci.STREAM_B)
    if g == "bf16":
        Ar, Bc = Ar.float().numpy(), Bc.float().numpy()
    Ar = np.asarray(Ar, dtype=np.float64)
    Bc = np.asarray(Bc, dtype=np.float64)
    return og.dot2_pairs(Ar[ri], Bc[cj]), Ar, Bc, ri, cj
