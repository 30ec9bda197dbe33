"""GPU parity of the selector's MLP kernels (K-MLP-FWD / K-MLP-BWD / K-MLP-ADAM)
against the FP64 oracle (oracle/mlp.py), through the C ABI, and a small
end-to-end run of the learned selector (collect -> train -> predict -> plan).

Tolerances: FP32 kernels vs FP64 oracle, relative error <= 1e-5 (forward),
<= 1e-4 (gradient, normwise), Adam <= 1e-5.  Gradients are deterministic
(fixed-order reduction): two runs must agree bit for bit.
"""
import numpy as np
import pytest

import cosma_inputs as ci
from oracle import mlp as om

from gpu_util import lib

pytestmark = pytest.mark.gpu


def _setup(B=300, seed=3):
    n = om.nparams()
    p = 0.2 * ci.entries(np.arange(n), np.zeros(n), 1, "uniform", "f64", seed, 3)
    p = p.astype(np.float32).astype(np.float64)
    X = ci.matrix(B, om.IN, "uniform", "f32", seed, 4).astype(np.float64)
    cand = ((ci.entries(np.arange(B), np.zeros(B), 1, "integer", "f64", seed, 5) + 8) % om.OUT).astype(np.int32)
    t = ci.entries(np.arange(B), np.zeros(B), 1, "uniform", "f32", seed, 6).astype(np.float64)
    return p, X, cand, t


def _dev(a, dt):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def test_forward_matches_oracle():
    import torch
    cosma = lib()
    p, X, _, _ = _setup()
    Y = torch.empty((X.shape[0], om.OUT), dtype=torch.float32, device="cuda")
    pd, Xd = _dev(p, torch.float32), _dev(X, torch.float32)
    assert cosma.cosma_mlp_forward(X.shape[0], Xd.data_ptr(), pd.data_ptr(), Y.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream) == 0
    ref, _ = om.forward(p, X)
    got = Y.double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def _grad(cosma, p, X, cand, t):
    import torch
    g = torch.empty(om.nparams(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    # keep every device buffer referenced until the kernels have run
    Xd, cd, td, pd = (_dev(X, torch.float32), _dev(cand, torch.int32), _dev(t, torch.float32),
                      _dev(p, torch.float32))
    rc = cosma.cosma_mlp_loss_grad(X.shape[0], Xd.data_ptr(), cd.data_ptr(), td.data_ptr(),
                                   pd.data_ptr(), g.data_ptr(), loss.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return g.double().cpu().numpy(), float(loss.item())


@pytest.mark.parametrize("B", [1, 63, 300, 1000])
def test_loss_and_gradient_match_oracle(B):
    cosma = lib()
    p, X, cand, t = _setup(B=B)
    g, L = _grad(cosma, p, X, cand, t)
    gref = om.grad(p, X, cand, t)
    Lref = om.loss(p, X, cand, t)
    assert abs(L - Lref) <= 1e-5 * max(1.0, abs(Lref))
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_out_of_range_candidates_are_skipped():
    cosma = lib()
    p, X, cand, t = _setup(B=50)
    bad = cand.copy()
    bad[::2] = 9999
    g, _ = _grad(cosma, p, X, bad, t)
    keep = bad < om.OUT
    gref = om.grad(p, X[keep], cand[keep], t[keep]) * keep.sum() / len(keep)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_gradient_is_deterministic():
    cosma = lib()
    p, X, cand, t = _setup(B=777)
    g1, _ = _grad(cosma, p, X, cand, t)
    g2, _ = _grad(cosma, p, X, cand, t)
    assert np.array_equal(g1, g2)


def test_adam_matches_oracle():
    import torch
    cosma = lib()
    p, X, cand, t = _setup()
    n = om.nparams()
    pd = _dev(p, torch.float32)
    md = torch.zeros(n, dtype=torch.float32, device="cuda")
    vd = torch.zeros(n, dtype=torch.float32, device="cuda")
    pr, mr, vr = p.copy(), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = 0.1 * ci.entries(np.arange(n), np.zeros(n), 1, "uniform", "f32", step, 8).astype(np.float64)
        gd = _dev(g, torch.float32)  # referenced until the next iteration
        assert cosma.cosma_mlp_adam(n, pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(),
                                    step, 1e-3, 0.9, 0.999, 1e-8,
                                    torch.cuda.current_stream().cuda_stream) == 0
        pr, mr, vr = om.adam_step(pr, g, mr, vr, step, 1e-3, 0.9, 0.999, 1e-8)
    torch.cuda.synchronize()
    assert np.max(np.abs(pd.double().cpu().numpy() - pr)) <= 1e-5 * 1e-3 * 10 + 1e-7


def test_training_fits_a_known_cost_model():
    # targets from a fixed smooth function of the features: training with the
    # library's kernels must drive the loss down by an order of magnitude
    from paper_1908_09606_gb300 import autotune
    cosma = lib()
    N = 4000
    u = ci.matrix(N, 3, "uniform", "f64", 12, 0)
    dims = np.round(256 * 256 ** ((u + 1) / 2)).astype(int)
    cand = ((ci.entries(np.arange(N), np.zeros(N), 1, "integer", "f64", 12, 1) + 8) % 16).astype(np.int32)
    rows = [{"m": int(m), "n": int(n), "k": int(k), "dtype": 2, "cand": int(c),
             "seconds": float(2.0 * m * n * k / (1e15 * (0.5 + 0.03 * c)) + 1e-5)}
            for (m, n, k), c in zip(dims, cand)]
    X, c, y = autotune.features(rows)
    p, hist, _ = autotune.train(X, c, y, epochs=60, batch=256, lr=3e-3, seed=1)
    assert hist[-1] < 0.1 * hist[0], hist[::10]


def test_training_resumes_from_checkpoint_bit_for_bit():
    """Parameters, Adam moments, step count and the permutation stream are restored:
    8 epochs + resume to 20 equals 20 epochs in one run (deterministic kernels)."""
    import os
    import tempfile
    from paper_1908_09606_gb300 import autotune
    lib()
    N = 1500
    u = ci.matrix(N, 3, "uniform", "f64", 14, 0)
    dims = np.round(256 * 256 ** ((u + 1) / 2)).astype(int)
    cand = ((ci.entries(np.arange(N), np.zeros(N), 1, "integer", "f64", 14, 1) + 8) % 16).astype(np.int32)
    rows = [{"m": int(m), "n": int(n), "k": int(k), "dtype": 2, "cand": int(c),
             "seconds": float(2.0 * m * n * k / (1e15 * (0.5 + 0.03 * c)) + 1e-5)}
            for (m, n, k), c in zip(dims, cand)]
    X, c, y = autotune.features(rows)
    whole, hist_whole, _ = autotune.train(X, c, y, epochs=20, batch=128, lr=3e-3, seed=4)
    with tempfile.TemporaryDirectory() as d:
        ck = os.path.join(d, "ck.npz")
        autotune.train(X, c, y, epochs=8, batch=128, lr=3e-3, seed=4, checkpoint=ck)
        resumed, hist_res, _ = autotune.train(X, c, y, epochs=20, batch=128, lr=3e-3, seed=4,
                                              checkpoint=ck)
    assert np.array_equal(whole, resumed)
    assert np.array_equal(np.array(hist_whole), np.array(hist_res))


def test_selector_end_to_end_small():
    import torch
    from paper_1908_09606_gb300 import autotune
    from gpu_util import device_operands, host_operands, out_tensor
    from oracle import gemm as og
    cosma = lib()
    shapes = autotune.random_shapes(40, seed=5, lo=256, hi=2048)
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "t.jsonl")
        rows = autotune.collect(path, shapes, cosma.COSMA_BF16, cap_bytes=64e6, reps=1)
        rows2 = autotune.collect(path, shapes, cosma.COSMA_BF16, cap_bytes=64e6, reps=1)
        assert len(rows2) == len(rows)  # resumed: nothing timed twice
    X, c, y = autotune.features(rows)
    p, hist, _ = autotune.train(X, c, y, epochs=150, batch=128, lr=3e-3, seed=2)
    assert hist[-1] < hist[0]
    assert cosma.cosma_selector_set(p, 8.0, 11.0) == 0
    test = autotune.random_shapes(6, seed=6, lo=256, hi=2048)
    best, pred = cosma.cosma_selector_predict(test, cosma.COSMA_BF16)
    for (m, n, k), b in zip(test, best):
        # -1: the analytic plan is kept (it lies outside the candidate set)
        assert b == -1 or cosma.cosma_plan_candidate(m, n, k, cosma.COSMA_BF16, b) is not None
    # the learned selector drives planning; results stay correct
    try:
        assert cosma.cosma_init(selector=cosma.COSMA_SELECT_LEARNED) == 0
        m, n, k = test[0]
        pl = cosma.cosma_plan_query(m, n, k, cosma.COSMA_BF16, cosma.COSMA_SELECT_LEARNED)
        want = (cosma.cosma_plan_candidate(m, n, k, cosma.COSMA_BF16, best[0]) if best[0] >= 0
                else cosma.cosma_plan_query(m, n, k, cosma.COSMA_BF16, cosma.COSMA_SELECT_ANALYTIC))
        assert (pl.tile_n, pl.pk, pl.order) == (want.tile_n, want.pk, want.order)
        A, B = device_operands(m, n, k, "bf16")
        C, _ = out_tensor(m, n, "bf16")
        cosma.gemm(A, B, C, "bf16")
        torch.cuda.synchronize()
        Ah, Bh = host_operands(m, n, k, "bf16")
        ref = og.gemm(Ah, Bh, "dot2")
        absref = og.gemm(np.abs(Ah), np.abs(Bh), "naive")
        gam = k * 2.0 ** -23 / (1 - k * 2.0 ** -23)
        assert np.all(np.abs(C.double().cpu().numpy() - ref) <= gam * absref + 1e-300)
    finally:
        cosma.cosma_init()
        cosma.cosma_selector_set(None)


@pytest.mark.parametrize("dtype", ["bf16", "f32", "f64", "f64_emu_bf16"])
def test_shipped_selector_gain_on_held_out_shapes(dtype):
    """The shipped network (trained with the library's own kernels on a GB300 on
    all four dtypes) on shapes it never saw: every candidate timed (median of 3).
    The learned selector's median regret against exhaustive search is <= 5 %,
    and its mean regret is no worse than the analytic plan's: where the two
    choose the same plan they share one measurement, so the comparison is decided
    on the shapes where the network overrides the analytic plan."""
    import numpy as np
    from paper_1908_09606_gb300 import autotune
    cosma = lib()
    dt = cosma.DTYPES[dtype]
    autotune.install()
    try:
        cap = autotune.TUNE[dt]["max_flops"] / 8
        shapes = autotune.random_shapes(16, seed=300 + dt, lo=256, hi=8192, cap_bytes=1e9,
                                        dtype=dt, max_flops=cap)
        recs = autotune.evaluate(shapes, dt, cap_bytes=1e9, reps=3)
        rs = np.array([r["regret_sel"] for r in recs])
        ra = np.array([r["regret_analytic"] for r in recs])
        differ = sum(r["pick"] >= 0 and r["pick"] != r["analytic"] for r in recs)
        print(f"{dtype}: learned median / mean regret {np.median(rs):.3f} / {np.mean(rs):.3f}, "
              f"analytic {np.median(ra):.3f} / {np.mean(ra):.3f}; overrides {differ}")
        assert len(recs) >= 12
        assert np.median(rs) <= 0.05
        assert np.mean(rs) <= np.mean(ra) + 0.005
    finally:
        cosma.cosma_init()  # back to the default (analytic) configuration
        cosma.cosma_selector_set(None)
