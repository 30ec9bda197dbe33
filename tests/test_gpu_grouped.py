"""GPU parity of the grouped persistent launch (K-GROUPED) against the oracle,
through the C ABI, and its capture in a CUDA graph.

Problem sizes: m, n, k each round(64 * 64^u), u uniform in [0, 1) from the
shared generator (seed 1, stream 7) -- log-uniform in [64, 4096].  Operands of
problem i come from seed 1000 + i.  Each problem is checked on sampled
entries (tile corners, ragged edges, random) against the Dot2 oracle within
gamma_k |A||B| (u = 2^-23 for the tensor-core f32 accumulation, 2^-24 for FMA).
"""
import numpy as np
import pytest

import cosma_inputs as ci
from oracle import gemm as og

from gpu_util import lib

pytestmark = pytest.mark.gpu


def problem_dims(count, seed=1):
    return ci.grouped_dims(count, seed)


def _pad(x, r):
    return max(1, -(-int(x) // r) * r)


def make_group(dims, dtype, pad=False):
    """Operands of each problem; pad=True gives every row a 16-byte-multiple pitch
    (B loaded as it is, C written by tensor stores), else pitches equal the
    widths (most B transposed first, most C stored row by row)."""
    import torch
    from cosma_inputs import device as cid
    g = "bf16" if dtype == "bf16" else "f32"
    tdt = torch.bfloat16 if g == "bf16" else torch.float32
    r = 8 if g == "bf16" else 4
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(dims):
        lda, ldb, ldc = (_pad(k, r), _pad(n, r), _pad(n, 4)) if pad else (k, n, n)
        A = torch.empty((m, max(lda, 1)), dtype=tdt, device="cuda")[:, :k]
        B = torch.empty((k, max(ldb, 1)), dtype=tdt, device="cuda")[:, :n]
        if m and k:
            cid.fill(A, "uniform", g, 1000 + i, ci.STREAM_A)
        if k and n:
            cid.fill(B, "uniform", g, 1000 + i, ci.STREAM_B)
        As.append(A)
        Bs.append(B)
        Cs.append(torch.full((m, max(ldc, 1)), float("nan"), dtype=torch.float32,
                             device="cuda")[:, :n])
    return As, Bs, Cs


def check_group(dims, Cs, dtype, per_problem=6, u=None):
    u = u or (2.0 ** -23 if dtype == "bf16" else 2.0 ** -24)
    g = "bf16" if dtype == "bf16" else "f32"
    rng = np.random.default_rng(5)
    for i, (m, n, k) in enumerate(dims):
        if m == 0 or n == 0:
            continue
        C = Cs[i].double().cpu().numpy()
        if k == 0:
            assert not C.any()
            continue
        # tile corners of the 128- and 256-row tiles, the halves of pair tiles
        rr = np.array([0, m - 1, min(127, m - 1), min(128, m - 1), min(255, m - 1)]
                      + list(rng.integers(0, m, per_problem)))
        cc = np.array([0, n - 1, min(127, n - 1), min(128, n - 1), min(255, n - 1)]
                      + list(rng.integers(0, n, per_problem)))
        Ar = ci.rows(rr, k, "uniform", g, 1000 + i, ci.STREAM_A)
        Bc = ci.cols(cc, k, n, "uniform", g, 1000 + i, ci.STREAM_B)
        if g == "bf16":
            Ar, Bc = Ar.float().numpy(), Bc.float().numpy()
        Ar, Bc = np.asarray(Ar, np.float64), np.asarray(Bc, np.float64)
        ref = og.dot2_pairs(Ar, Bc)
        absr = np.einsum("ij,ij->i", np.abs(Ar), np.abs(Bc))
        gam = k * u / (1 - k * u)
        got = C[rr, cc]
        assert np.all(np.abs(got - ref) <= gam * absr + 1e-300), (i, m, n, k)


def run_group(As, Bs, Cs, dtype):
    import torch
    cosma = lib()
    cosma.gemm_grouped(As, Bs, Cs, dtype)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0


@pytest.mark.parametrize("tile", [0, 128, 256, 512])
def test_grouped_bf16_512_problems(tile):
    cosma = lib()
    dims = problem_dims(512)
    As, Bs, Cs = make_group(dims, "bf16")
    try:
        assert cosma.cosma_init(grouped_tile=tile) == 0
        run_group(As, Bs, Cs, "bf16")
    finally:
        cosma.cosma_init()
    check_group(dims, Cs, "bf16", per_problem=4 if tile else 8)


@pytest.mark.parametrize("tile", [64, 128])
def test_grouped_f32(tile):
    cosma = lib()
    dims = problem_dims(96)
    As, Bs, Cs = make_group(dims, "f32")
    try:
        assert cosma.cosma_init(grouped_tile=tile) == 0
        run_group(As, Bs, Cs, "f32")
    finally:
        cosma.cosma_init()
    check_group(dims, Cs, "f32")


@pytest.mark.parametrize("dtype,tile", [("bf16", 0), ("f32", 0), ("bf16", 512)])
def test_grouped_empty_and_k0_problems(dtype, tile):
    cosma = lib()
    dims = np.array([[0, 5, 7], [9, 0, 3], [130, 70, 0], [1, 1, 1], [129, 257, 65], [7, 9, 3000],
                     [300, 520, 200], [257, 129, 64]])
    As, Bs, Cs = make_group(dims, dtype)
    try:
        assert cosma.cosma_init(grouped_tile=tile) == 0
        run_group(As, Bs, Cs, dtype)
    finally:
        cosma.cosma_init()
    check_group(dims, Cs, dtype)


def test_grouped_bf16_unaligned_a_is_packed():
    import torch
    from cosma_inputs import device as cid
    cosma = lib()
    store = torch.zeros((100, 140), dtype=torch.bfloat16, device="cuda")
    A = store[:, 1:131]  # base 2 bytes off a 16-byte boundary, pitch 280 bytes
    cid.fill(A, "uniform", "bf16", 1000, ci.STREAM_A)
    B = torch.empty((130, 90), dtype=torch.bfloat16, device="cuda")
    cid.fill(B, "uniform", "bf16", 1000, ci.STREAM_B)
    C = torch.full((100, 90), float("nan"), dtype=torch.float32, device="cuda")
    cosma.gemm_grouped([A], [B], [C], "bf16")
    torch.cuda.synchronize()
    check_group(np.array([[100, 90, 130]]), [C], "bf16")


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_grouped_captured_in_cuda_graph(dtype):
    import torch
    cosma = lib()
    dims = problem_dims(64, seed=3)
    As, Bs, Cs = make_group(dims, dtype)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        cosma.gemm_grouped(As, Bs, Cs, dtype)      # eager: builds and caches the table
    torch.cuda.synchronize()
    eager = [c.clone() for c in Cs]
    for c in Cs:
        c.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cosma.gemm_grouped(As, Bs, Cs, dtype)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for c, e in zip(Cs, eager):
        assert torch.equal(c, e)
    check_group(dims, Cs, dtype, per_problem=3)


@pytest.mark.parametrize("tile", [0, 512])
def test_grouped_bf16_padded_pitches_direct_b_and_tensor_stores(tile):
    """Every B loaded as it is (MN-major) and every C written by tensor stores;
    the padding columns of C stay untouched.  Tile 512: 256 x 256 tiles on CTA
    pairs, each CTA holding 128 of the tile's B columns."""
    import torch
    cosma = lib()
    dims = problem_dims(96, seed=4)
    As, Bs, Cs = make_group(dims, "bf16", pad=True)
    stores = [c.as_strided((c.shape[0], c.stride(0)), (c.stride(0), 1)) for c in Cs]
    for st in stores:
        st.fill_(-3.0)
    try:
        assert cosma.cosma_init(grouped_tile=tile) == 0
        run_group(As, Bs, Cs, "bf16")
    finally:
        cosma.cosma_init()
    check_group(dims, Cs, "bf16", per_problem=6)
    for (m, n, k), st in zip(dims, stores):
        if st.shape[1] > n:
            assert torch.all(st[:, n:] == -3.0)


@pytest.mark.parametrize("dtype,tiles", [("bf16", (128, 256, 512)), ("f32", (64, 128))])
def test_grouped_autotuner_picks_a_tile_and_results_hold(dtype, tiles):
    from paper_1908_09606_gb300 import autotune
    cosma = lib()
    dims = problem_dims(40)
    As, Bs, Cs = make_group(dims, dtype)
    try:
        tile, times = autotune.tune_grouped(As, Bs, Cs, dtype, reps=2)
        assert tile in tiles and set(times) == set(tiles)
        assert times[tile] == min(times.values()) and all(t > 0 for t in times.values())
        assert cosma.cosma_get_config().grouped_tile == tile
        run_group(As, Bs, Cs, dtype)
    finally:
        cosma.cosma_init()
    check_group(dims, Cs, dtype)


def test_grouped_graph_stays_valid_after_the_table_cache_turns_over():
    """Nine other groups pass through the eight-slot table cache after a group
    was captured; its table is retired, not overwritten, so the replay still
    equals the eager call."""
    import torch
    cosma = lib()
    dtype = "f32"
    dims = problem_dims(16, seed=4)
    As, Bs, Cs = make_group(dims, dtype)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        cosma.gemm_grouped(As, Bs, Cs, dtype)      # eager: builds and caches the table
    torch.cuda.synchronize()
    eager = [c.clone() for c in Cs]
    for c in Cs:
        c.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cosma.gemm_grouped(As, Bs, Cs, dtype)
    others = []
    for j in range(9):
        d = np.minimum(problem_dims(3, seed=20 + j), 1024)
        Ao, Bo, Co = make_group(d, dtype)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            cosma.gemm_grouped(Ao, Bo, Co, dtype)
        others.append((d, Ao, Bo, Co))
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    for c, e in zip(Cs, eager):
        assert torch.equal(c, e)
    d, _, _, Co = others[-1]
    check_group(d, Co, dtype, per_problem=3)


@pytest.mark.parametrize("tile", [256, 512])
def test_grouped_bounded_wait_reports_timeout_and_context_survives(tile):
    """A one-cycle wait limit makes the tensor-core grouped kernel's waits run out
    (one CTA per tile, or CTA pairs): it records COSMA_ERR_TIMEOUT, drains the copies
    its CTAs may have in flight, frees its tensor memory and exits; the next call
    with the default limit is correct."""
    import torch
    cosma = lib()
    dims = problem_dims(32, seed=6)
    As, Bs, Cs = make_group(dims, "bf16", pad=True)
    try:
        assert cosma.cosma_init(grouped_tile=tile, wait_limit=1) == 0
        cosma.gemm_grouped(As, Bs, Cs, "bf16")
        torch.cuda.synchronize()
        assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == \
            cosma.COSMA_ERR_TIMEOUT
        assert cosma.cosma_init(grouped_tile=tile) == 0
        run_group(As, Bs, Cs, "bf16")
    finally:
        cosma.cosma_init()
    check_group(dims, Cs, "bf16", per_problem=4)
