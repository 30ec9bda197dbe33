"""Autotuner, selector training and regret evaluation (a8 of the hot path).

  collect()   times every applicable plan candidate (cosma_plan_candidate,
              cosma_gemm_planned, CUDA events, median of `reps` after a
              warm-up) on random shapes and appends (shape, dtype, candidate,
              seconds) rows to a JSONL file; rows already present are skipped,
              so an interrupted run resumes where it stopped.
  train()     fits the MLP cost model on those rows with the library's own
              kernels (cosma_mlp_loss_grad + cosma_mlp_adam on the GPU),
              checkpointing parameters and Adam state after every epoch; one
              network for every dtype (the dtype is a one-hot input).
  evaluate()  exhaustive timing on held-out shapes: regret of the learned
              choice and of the analytic plan against the best candidate (the
              two share a measurement where they pick the same plan).
  tune_grouped()  times one grouped launch with each tile width the grouped
              kernels implement and keeps the fastest as the configured default.

Shapes: m, n, k log-uniform in [lo, hi] from the shared generator, rejecting
shapes with an operand above `cap_bytes`.  Every compute step runs in the
CUDA library; this module only orchestrates and keeps records.
"""

import json
import math
import os
import time

import numpy as np

from . import cosma

DTYPE_BYTES = {cosma.COSMA_BF16: (2, 4), cosma.COSMA_F32: (4, 4), cosma.COSMA_F64: (8, 8),
               cosma.COSMA_F64_EMU_BF16: (8, 8)}


def random_shapes(count, seed, lo=256, hi=65536, cap_bytes=16e9, dtype=cosma.COSMA_BF16,
                  max_flops=None):
    import cosma_inputs as ci
    win, wout = DTYPE_BYTES[dtype]
    out, i = [], 0
    while len(out) < count:
        e = np.arange(3 * i, 3 * i + 3)
        u = (ci.entries(e, np.zeros(3), 1, "uniform", "f64", seed, 11) + 1.0) / 2.0
        m, n, k = (int(round(lo * (hi / lo) ** x)) for x in u)
        i += 1
        if max(m * k * win, k * n * win, m * n * wout) > cap_bytes:
            continue
        if max_flops and 2.0 * m * n * k > max_flops:
            continue
        out.append((m, n, k))
    return out


class Operands:
    """Device buffers reused for every shape (views of their leading part)."""

    def __init__(self, dtype, cap_bytes):
        import torch
        from cosma_inputs import device as cid
        win, wout = DTYPE_BYTES[dtype]
        tin = {2: torch.bfloat16, 4: torch.float32, 8: torch.float64}[win]
        tout = {4: torch.float32, 8: torch.float64}[wout]
        g = {2: "bf16", 4: "f32", 8: "f64"}[win]
        self.A = torch.empty(int(cap_bytes // win), dtype=tin, device="cuda")
        self.B = torch.empty(int(cap_bytes // win), dtype=tin, device="cuda")
        self.C = torch.empty(int(cap_bytes // wout), dtype=tout, device="cuda")
        cid.fill(self.A.view(1, -1), "uniform", g, 21, 0)
        cid.fill(self.B.view(1, -1), "uniform", g, 21, 1)

    def ptrs(self):
        return self.A.data_ptr(), self.B.data_ptr(), self.C.data_ptr()


# Per dtype: the largest product timed (2mnk; FP64 runs at about 1.2 TFLOP/s) and
# the collection budget in seconds of main().
TUNE = {cosma.COSMA_BF16: {"max_flops": 4e13, "budget_s": 240},
        cosma.COSMA_F32: {"max_flops": 2e12, "budget_s": 200},
        cosma.COSMA_F64: {"max_flops": 5e10, "budget_s": 240},
        cosma.COSMA_F64_EMU_BF16: {"max_flops": 2e12, "budget_s": 120}}


def time_plan(m, n, k, dtype, plan, ops, reps=3):
    """Median seconds of `reps` products with the given plan (None -> analytic),
    after one untimed warm-up."""
    import torch
    a, b, c = ops.ptrs()
    s = torch.cuda.current_stream()
    sh = s.cuda_stream

    def run():
        if plan is None:
            rc = cosma.cosma_gemm(m, n, k, a, k, b, n, c, n, dtype, sh)
        else:
            rc = cosma.cosma_gemm_planned(m, n, k, a, k, b, n, c, n, dtype, plan, sh)
        if rc != 0:
            raise cosma.CosmaError(rc, "time_plan")

    run()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record(s)
        run()
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    return float(np.median(ts))


def candidates(m, n, k, dtype, max_ws_bytes):
    out = []
    for c in range(cosma.COSMA_MLP_OUT):
        p = cosma.cosma_plan_candidate(m, n, k, dtype, c)
        if p is not None and p.workspace_bytes <= max_ws_bytes:
            out.append((c, p))
    return out


_PLAN_KEY = ("tile_m", "tile_n", "k_block", "pk", "order", "ctas", "pm", "pn")


def analytic_candidate(m, n, k, dtype, cands):
    """Index of the candidate that is the analytic plan, or None when the
    analytic plan lies outside the candidate set."""
    pa = cosma.cosma_plan_query(m, n, k, dtype, cosma.COSMA_SELECT_ANALYTIC)
    want = tuple(getattr(pa, f) for f in _PLAN_KEY)
    for c, p in cands:
        if tuple(getattr(p, f) for f in _PLAN_KEY) == want:
            return c
    return None


def _load_rows(path):
    rows = []
    if path and os.path.exists(path):
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line:
                    rows.append(json.loads(line))
    return rows


def collect(path, shapes, dtype=cosma.COSMA_BF16, cap_bytes=16e9, max_ws_bytes=24e9, reps=3,
            time_budget_s=None, log=None):
    """Times all applicable candidates of each shape; returns the rows of `path`."""
    done = {(r["m"], r["n"], r["k"], r["dtype"], r["cand"]) for r in _load_rows(path)}
    ops = Operands(dtype, cap_bytes)
    t0 = time.time()
    with open(path, "a") as f:
        for (m, n, k) in shapes:
            if time_budget_s and time.time() - t0 > time_budget_s:
                break
            for c, p in candidates(m, n, k, dtype, max_ws_bytes):
                key = (m, n, k, dtype, c)
                if key in done:
                    continue
                sec = time_plan(m, n, k, dtype, p, ops, reps)
                f.write(json.dumps({"m": m, "n": n, "k": k, "dtype": dtype, "cand": c,
                                    "seconds": sec}) + "\n")
                done.add(key)
            f.flush()
            if log:
                log(f"collected {m}x{n}x{k}")
    del ops
    return _load_rows(path)


def is_calibration(m, n, k, dtype):
    """One shape in five (by a hash of the shape) is kept out of training and used
    to calibrate the selector's per-dtype margin."""
    h = (int(m) * 73856093) ^ (int(n) * 19349663) ^ (int(k) * 83492791) ^ int(dtype)
    return h % 5 == 0


# Margins (log2 seconds) the calibration chooses from; inf: keep the analytic plan.
MARGINS = (0.05, 0.1, 0.15, 0.2, 0.3, 0.5, 1.0, math.inf)


def calibrate_margin(rows, dtype, max_ws_bytes=24e9):
    """The margin (from MARGINS) whose learned choices have the least mean regret
    on the calibration shapes of `rows` (every candidate of a shape timed), ties
    to the larger margin; shapes whose analytic plan is not a timed candidate are
    skipped (the selector keeps the analytic plan there anyway).  Uses the
    installed network.  Returns (margin, {margin: mean regret}, shapes used)."""
    by = {}
    for r in rows:
        if r["dtype"] == dtype and is_calibration(r["m"], r["n"], r["k"], dtype):
            by.setdefault((r["m"], r["n"], r["k"]), {})[r["cand"]] = r["seconds"]
    shapes = sorted(by)
    if not shapes:
        return 0.05, {}, 0
    _, preds = cosma.cosma_selector_predict(shapes, dtype)
    regrets = {mg: [] for mg in MARGINS}
    used = 0
    for (m, n, k), pred in zip(shapes, preds):
        times = by[(m, n, k)]
        ca = analytic_candidate(m, n, k, dtype, candidates(m, n, k, dtype, max_ws_bytes))
        if ca is None or ca not in times:
            continue
        used += 1
        best_t = min(times.values())
        b = min(times, key=lambda c: pred[c])
        for mg in MARGINS:
            choice = b if pred[b] < pred[ca] - mg else ca
            regrets[mg].append(times[choice] / best_t - 1.0)
    if not used:
        return 0.05, {}, 0
    mean = {mg: float(np.mean(v)) for mg, v in regrets.items()}
    lo = min(mean.values())
    pick = max(mg for mg in MARGINS if mean[mg] <= lo + 1e-12)
    return pick, mean, used


def features(rows):
    X = np.array([cosma.cosma_selector_features(r["m"], r["n"], r["k"], r["dtype"]) for r in rows],
                 dtype=np.float32)
    cand = np.array([r["cand"] for r in rows], dtype=np.int32)
    y = np.log2(np.array([r["seconds"] for r in rows], dtype=np.float64))
    return X, cand, y


def init_params(seed):
    """He-uniform initial weights from the shared generator, zero biases."""
    import cosma_inputs as ci
    IN, H, OUT = cosma.COSMA_MLP_IN, cosma.COSMA_MLP_HIDDEN, cosma.COSMA_MLP_OUT
    parts = []
    for j, (fo, fi) in enumerate([(H, IN), (H, H), (OUT, H)]):
        lim = math.sqrt(6.0 / fi)
        e = np.arange(fo * fi)
        w = lim * ci.entries(e, np.zeros(fo * fi), 1, "uniform", "f64", seed, 30 + j)
        parts += [w, np.zeros(fo)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == cosma.COSMA_MLP_PARAMS
    return p


def destandardize(params, mu, sigma):
    """The same network with outputs in log2 seconds instead of standardised
    units (the last layer scaled by sigma, shifted by mu): the form the library's
    selector reads, so its margin has a fixed meaning."""
    IN, H, OUT = cosma.COSMA_MLP_IN, cosma.COSMA_MLP_HIDDEN, cosma.COSMA_MLP_OUT
    p = np.array(params, dtype=np.float64)
    w3 = H * IN + H + H * H + H   # start of the last layer's weights
    p[w3:w3 + OUT * H] *= sigma
    p[w3 + OUT * H:w3 + OUT * H + OUT] = p[w3 + OUT * H:w3 + OUT * H + OUT] * sigma + mu
    return p.astype(np.float32)


def train(X, cand, y, epochs=300, batch=256, lr=2e-3, seed=0, checkpoint=None, log=None):
    """Adam on the library's MLP kernels.  Targets are standardised log2 times.
    Returns (params, history of epoch losses, (mu, sigma))."""
    import torch
    mu, sigma = float(np.mean(y)), float(np.std(y) + 1e-9)
    t = ((y - mu) / sigma).astype(np.float32)
    N = X.shape[0]
    dev = "cuda"
    Xd = torch.from_numpy(X).to(dev)
    cd = torch.from_numpy(cand).to(dev)
    td = torch.from_numpy(t).to(dev)
    start_epoch, step = 0, 0
    p = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    hist = []
    if checkpoint and os.path.exists(checkpoint):
        ck = np.load(checkpoint)
        p.copy_(torch.from_numpy(ck["params"]))
        m.copy_(torch.from_numpy(ck["m"]))
        v.copy_(torch.from_numpy(ck["v"]))
        start_epoch, step = int(ck["epoch"]) + 1, int(ck["step"])
        hist = list(ck["hist"])
    g = torch.zeros_like(p)
    loss = torch.zeros(1, device=dev)
    sh = torch.cuda.current_stream().cuda_stream
    perm_rng = np.random.default_rng(seed)
    for _ in range(start_epoch):  # replay the permutation stream for a resumed run
        perm_rng.permutation(N)
    for ep in range(start_epoch, epochs):
        perm = torch.from_numpy(perm_rng.permutation(N).astype(np.int64)).to(dev)
        Xs, cs, ts = Xd[perm].contiguous(), cd[perm].contiguous(), td[perm].contiguous()
        tot = 0.0
        nb = 0
        for s0 in range(0, N, batch):
            b = min(batch, N - s0)
            rc = cosma.cosma_mlp_loss_grad(b, Xs[s0:].data_ptr(), cs[s0:].data_ptr(),
                                           ts[s0:].data_ptr(), p.data_ptr(), g.data_ptr(),
                                           loss.data_ptr(), sh)
            if rc != 0:
                raise cosma.CosmaError(rc, "cosma_mlp_loss_grad")
            step += 1
            rc = cosma.cosma_mlp_adam(p.numel(), p.data_ptr(), g.data_ptr(), m.data_ptr(),
                                      v.data_ptr(), step, lr, 0.9, 0.999, 1e-8, sh)
            if rc != 0:
                raise cosma.CosmaError(rc, "cosma_mlp_adam")
            tot += float(loss.item()) * b
            nb += b
        hist.append(tot / max(nb, 1))
        if checkpoint:
            np.savez(checkpoint, params=p.cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(),
                     epoch=ep, step=step, hist=np.array(hist))
        if log and (ep % 50 == 0 or ep == epochs - 1):
            log(f"epoch {ep} loss {hist[-1]:.4f}")
    return p.cpu().numpy(), hist, (mu, sigma)


def evaluate(shapes, dtype=cosma.COSMA_BF16, cap_bytes=16e9, max_ws_bytes=24e9, reps=3,
             log=None):
    """Exhaustive timing on shapes; returns per-shape records with the best
    candidate, the learned pick (installed selector; -1 = the analytic plan) and
    the analytic plan.  Where the analytic plan is a candidate, its time is that
    candidate's measurement, so equal choices have equal times."""
    best_l, _ = cosma.cosma_selector_predict(shapes, dtype)
    ops = Operands(dtype, cap_bytes)
    recs = []
    for (m, n, k), pick in zip(shapes, best_l):
        cands = candidates(m, n, k, dtype, max_ws_bytes)
        times = {}
        for c, p in cands:
            times[c] = time_plan(m, n, k, dtype, p, ops, reps)
        if not times:
            continue
        t_best = min(times.values())
        ca = analytic_candidate(m, n, k, dtype, cands)
        t_ana = times[ca] if ca is not None else time_plan(m, n, k, dtype, None, ops, reps)
        t_sel = t_ana if pick < 0 or pick == ca else times.get(pick, t_ana)
        recs.append({"m": m, "n": n, "k": k, "dtype": dtype, "best": min(times, key=times.get),
                     "pick": pick, "analytic": -1 if ca is None else ca,
                     "t_best": t_best, "t_sel": t_sel, "t_analytic": t_ana,
                     "regret_sel": t_sel / t_best - 1.0, "regret_analytic": t_ana / t_best - 1.0})
        if log:
            log(f"eval {m}x{n}x{k} regret sel {recs[-1]['regret_sel']:.3f} "
                f"analytic {recs[-1]['regret_analytic']:.3f}")
    del ops
    return recs


SHIPPED_PARAMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                              "selector_gb300.npy")


def tune_grouped(As, Bs, Cs, dtype, tiles=None, reps=3):
    """Autotune the grouped launch for this group of products: time
    cosma_gemm_grouped (CUDA events, best of `reps`) with each tile width (bf16:
    128 x 128 and 128 x 256 C tiles, and 256 x 256 tiles on CTA pairs (512); f32:
    64 and 128), the library's tables for
    a width being built by an untimed first call; set the fastest as the
    library's grouped_tile and return (tile, {tile: milliseconds})."""
    import torch
    if tiles is None:
        tiles = (128, 256, 512) if dtype in ("bf16", cosma.COSMA_BF16) else (64, 128)
    cfg = cosma.cosma_get_config()

    def use(tile):
        rc = cosma.cosma_init(cfg.delta, cfg.selector, cfg.emu_slices, cfg.emu_slice_bits,
                              cfg.wait_limit, tile)
        if rc != cosma.COSMA_OK:
            raise cosma.CosmaError(rc, "cosma_init")

    times = {}
    for t in tiles:
        use(t)
        cosma.gemm_grouped(As, Bs, Cs, dtype)
        torch.cuda.synchronize()
        best = math.inf
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            cosma.gemm_grouped(As, Bs, Cs, dtype)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        times[t] = best
    choice = min(times, key=times.get)
    use(choice)
    return choice, times


def install(params_path=None, log2_lo=8.0, log2_hi=16.0, dtypes=None):
    """Installs trained selector weights saved by main() (an .npy vector of
    log2-second outputs, with its per-dtype margins from <stem>_margins.json when
    present); by default the weights shipped with the package, trained on a GB300
    on all four dtypes.  dtypes: restrict the network to these (None: every
    dtype)."""
    path = params_path or SHIPPED_PARAMS
    p = np.load(path).astype(np.float32)
    rc = cosma.cosma_selector_set(p, log2_lo, log2_hi)
    if rc != 0:
        raise cosma.CosmaError(rc, "cosma_selector_set")
    mpath = os.path.splitext(path)[0] + "_margins.json"
    if os.path.exists(mpath):
        with open(mpath) as f:
            for name, mg in json.load(f).items():
                rc = cosma.cosma_selector_margin(name, math.inf if mg is None else mg)
                if rc != 0:
                    raise cosma.CosmaError(rc, "cosma_selector_margin")
    if dtypes is not None:
        rc = cosma.cosma_selector_restrict(dtypes)
        if rc != 0:
            raise cosma.CosmaError(rc, "cosma_selector_restrict")


def parser():
    import argparse
    ap = argparse.ArgumentParser(description="collect timings, train the selector, report regret")
    ap.add_argument("--out", required=True)
    ap.add_argument("--dtypes", default="bf16,f32,f64,f64_emu_bf16")
    ap.add_argument("--train-shapes", type=int, default=4000, help="per dtype, budget permitting")
    ap.add_argument("--test-shapes", type=int, default=500, help="held out, over all dtypes")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--budget-scale", type=float, default=1.0,
                    help="scales every dtype's collection budget")
    ap.add_argument("--eval-budget-s", type=float, default=600, help="over all dtypes")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-collect", action="store_true",
                    help="train on the timing files already in --out")
    ap.add_argument("--collect-dtypes", default=None,
                    help="collect fresh timings for these dtypes only (comma-separated) and "
                         "train on the files already in --out for the others")
    ap.add_argument("--eval-only", metavar="PARAMS",
                    help="install these weights (and their margins) and only evaluate")
    return ap


def _summary(recs):
    rs = np.array([r["regret_sel"] for r in recs])
    ra = np.array([r["regret_analytic"] for r in recs])
    if not len(rs):
        return {"test_shapes": 0}
    dev = [r for r in recs if r["pick"] >= 0 and r["pick"] != r["analytic"]]
    return {
        "test_shapes": len(recs),
        "median_regret_learned": float(np.median(rs)),
        "mean_regret_learned": float(np.mean(rs)),
        "p90_regret_learned": float(np.percentile(rs, 90)),
        "median_regret_analytic": float(np.median(ra)),
        "mean_regret_analytic": float(np.mean(ra)),
        "p90_regret_analytic": float(np.percentile(ra, 90)),
        "learned_differs_from_analytic": len(dev),
        "mean_gain_where_it_differs": float(np.mean([r["t_analytic"] / r["t_sel"] - 1.0
                                                     for r in dev])) if dev else 0.0,
        "learned_exact_best_fraction": float(np.mean([
            (r["pick"] if r["pick"] >= 0 else r["analytic"]) == r["best"] for r in recs])),
    }


def _evaluate_all(a, dts):
    """Held-out shapes of every dtype, timed within the evaluation budget;
    records also written to <out>/eval.jsonl."""
    per = max(1, a.test_shapes // len(dts))
    recs, t_eval = [], {}
    for dt in dts:
        test = random_shapes(per, seed=200 + a.seed + 1000 * dt, dtype=dt,
                             max_flops=TUNE[dt]["max_flops"])
        t0 = time.time()
        for sh in test:
            if time.time() - t0 > a.eval_budget_s / len(dts):
                break
            recs += evaluate([sh], dt, reps=3)
        t_eval[dt] = time.time() - t0
    with open(os.path.join(a.out, "eval.jsonl"), "w") as f:
        for r in recs:
            f.write(json.dumps(r) + "\n")
    return recs, t_eval


def main(argv=None):
    import torch
    a = parser().parse_args(argv)
    os.makedirs(a.out, exist_ok=True)
    torch.cuda.set_device(0)
    cosma.load()
    log = lambda s: print(s, flush=True)  # noqa: E731
    dts = [cosma.DTYPES[d] for d in a.dtypes.split(",")]
    names = {v: k for k, v in cosma.DTYPES.items() if k in a.dtypes.split(",")}
    if a.eval_only:
        install(a.eval_only)
        recs, t_eval = _evaluate_all(a, dts)
        summary = {"params": os.path.basename(a.eval_only),
                   "per_dtype": {names[dt]: _summary([r for r in recs if r["dtype"] == dt])
                                 for dt in dts},
                   "all": _summary(recs),
                   "seconds": {"eval": {names[d]: v for d, v in t_eval.items()}}}
        with open(os.path.join(a.out, "summary.json"), "w") as f:
            json.dump(summary, f, indent=1)
        print(json.dumps(summary), flush=True)
        return 0
    rows, t_collect = [], {}
    for dt in dts:
        shapes = random_shapes(a.train_shapes, seed=100 + a.seed + 1000 * dt, dtype=dt,
                               max_flops=TUNE[dt]["max_flops"])
        t0 = time.time()
        path = os.path.join(a.out, f"timings_{dt}.jsonl")
        fresh = not a.no_collect and (a.collect_dtypes is None or
                                      names[dt] in a.collect_dtypes.split(","))
        rows += (collect(path, shapes, dt, time_budget_s=TUNE[dt]["budget_s"] * a.budget_scale,
                         reps=3) if fresh else _load_rows(path))
        t_collect[dt] = time.time() - t0
        log(f"dtype {dt}: {len(rows)} rows so far")
    train_rows = [r for r in rows if not is_calibration(r["m"], r["n"], r["k"], r["dtype"])]
    X, c, y = features(train_rows)
    t0 = time.time()
    p, hist, (mu, sigma) = train(X, c, y, epochs=a.epochs, seed=a.seed,
                                 checkpoint=os.path.join(a.out, "checkpoint.npz"), log=log)
    t_train = time.time() - t0
    p = destandardize(p, mu, sigma)
    np.save(os.path.join(a.out, "selector_params.npy"), p)
    rc = cosma.cosma_selector_set(p, math.log2(256), math.log2(65536))
    if rc != 0:
        raise cosma.CosmaError(rc, "cosma_selector_set")
    margins, calib = {}, {}
    for dt in dts:
        mg, table, used = calibrate_margin(rows, dt)
        cosma.cosma_selector_margin(dt, mg)
        margins[names[dt]] = None if math.isinf(mg) else mg
        calib[names[dt]] = {"margin": margins[names[dt]], "shapes": used,
                            "mean_regret_by_margin": {str(k): v for k, v in table.items()}}
        log(f"dtype {dt}: margin {mg} from {used} calibration shapes")
    with open(os.path.join(a.out, "selector_params_margins.json"), "w") as f:
        json.dump(margins, f, indent=1)
    recs, t_eval = _evaluate_all(a, dts)
    summary = {
        "train_rows": len(train_rows), "calibration_rows": len(rows) - len(train_rows),
        "margins": calib,
        "train_rows_per_dtype": {names[dt]: sum(r["dtype"] == dt for r in train_rows)
                                 for dt in dts},
        "epochs": a.epochs, "final_loss": hist[-1] if hist else None,
        "per_dtype": {names[dt]: _summary([r for r in recs if r["dtype"] == dt]) for dt in dts},
        "all": _summary(recs),
        "seconds": {"collect": {names[d]: v for d, v in t_collect.items()}, "train": t_train,
                    "eval": {names[d]: v for d, v in t_eval.items()}},
        "target_standardisation": {"mu": mu, "sigma": sigma},
        "max_flops": {names[dt]: TUNE[dt]["max_flops"] for dt in dts},
    }
    with open(os.path.join(a.out, "summary.json"), "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary), flush=True)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
