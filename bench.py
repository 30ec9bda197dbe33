#!/usr/bin/env python3
"""Benchmark of the GEMM hot path through the C ABI (one JSON line on rank 0).

A step is one C = A B on the chosen workload through cosma_gemm: plan
(FindSeqSchedule, ParallelizeSched/FitRanks), staged main loop, Reduce when the
plan splits k, and -- for the emulated dtype -- slice extraction and
recombination.  Inputs are generated on the device by the shared seeded
generator before the timed region and are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload square]
                  [--dtype f64_emu_bf16|f64|f32|bf16|f32_emu_tf32] [--impl reference]

Under torchrun each rank runs its own replica of the workload (the path needs
no exchange between GPUs): value = all ranks' flops / max-over-ranks time.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TFLOP/s and HBM bytes / I/O lower bound; split-BF16 vs native FP64 at equal error"
WORKLOADS = {
    "square": (16384, 16384, 16384),
    "largeK": (4096, 4096, 1 << 20),
    "largeM": (1 << 20, 4096, 4096),
    "flat": (65536, 65536, 1024),
    "flat16k": (16384, 16384, 1024),   # the flat family at profiling size
    "emu8192": (8192, 8192, 8192),
    "4096": (4096, 4096, 4096),
    "512": (512, 512, 512),
    "grouped512": None,   # 512 problems, dims log-uniform in [64, 4096], seed 1
}
DEFAULT_DTYPE = "f64_emu_bf16"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="square", choices=list(WORKLOADS))
    ap.add_argument("--dtype", default=DEFAULT_DTYPE,
                    choices=["f64", "f32", "bf16", "f64_emu_bf16", "f32_emu_tf32"])
    ap.add_argument("--impl", default="cosma", choices=["cosma", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-native", action="store_true")
    ap.add_argument("--grouped-tile", type=int, default=0,
                    help="grouped workload: this C tile width instead of the autotuner's "
                         "choice (profiler runs, whose timings mislead the autotuner)")
    return ap.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


# FP64 / FP32 FMA peaks of GB300 (dense, whole GPU), derived from the SM count,
# the FMA lanes per SM and the maximum SM clock: 152 SMs x 2070 MHz x
# (FP64: 2 FMA/clk/SM -> 1.26 TFLOP/s; FP32: 128 FMA/clk/SM -> 80.5 TFLOP/s).
def _alu_peak_tflops(dtype, sms):
    lanes = {"f64": 2, "f32": 128}[dtype]
    return sms * 2070e6 * lanes * 2 / 1e12


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel, from one ncu capture of exactly this workload and kernel
# version; absent entries are reported as null.
DRAM_TRAFFIC = {
    ("square", "bf16"): 10.25e9 + 1.07e9,     # tc_gemm_kernel<256,4,A K,B MN>, tensor-store C
    ("flat", "bf16"): 4.30e9 + 17.15e9,       # same kernel, 16 GB of f32 C
    ("4096", "f32"): 0.328e9 + 0.109e9,       # simt_f32_kernel<128,4,256>, pk = 2, f32x2 FMAs
    ("4096", "f64"): 0.969e9 + 0.133e9,       # simt_gemm_kernel<double,64,64,8,4,4>
    ("grouped512", "bf16"): 2.21e9 + 2.02e9,    # grouped_tc_kernel<256,4> (tile 256)
    ("grouped512", "bf16", 512): 2.122e9 + 2.021e9,  # grouped_pair_kernel (tile 512)
    # emu_pair_kernel<256>: the lock-step schedule captured under a plain cluster
    # launch (COSMA_EMU_LOCKSTEP=2; ncu cannot launch the cooperative one); 8192^3
    # is the mean of four captures of this kernel version (reads 43.3-55.6 GB),
    # 16384^3 8 x that (4096^3 -> 8192^3 grew 8.05x for 8x the work)
    ("emu8192", "f64_emu_bf16"): 49.09e9 + 3.40e9,
    ("square", "f64_emu_bf16"): 8 * (49.09e9 + 3.40e9),
    ("flat16k", "f64_emu_bf16"): 13.55e9 + 6.24e9,   # from the --set full capture
    # tf32x3_gemm_kernel: lock-step ticks under a plain launch (COSMA_TF32_LOCKSTEP=2)
    ("square", "f32_emu_tf32"): 53.16e9 + 1.07e9,
}


# Entries above that are scaled from a smaller capture, and how.
DRAM_SCALED = {
    ("square", "f64_emu_bf16"): "; 8 x the mean of four 8192^3 captures of the same "
                                "kernel (DRAM bytes grew 8.05x from 4096^3 to 8192^3 for "
                                "8x the work in an earlier build)",
}


def io_report(m, n, k, dtype, plan, traffic, l2_bytes, sms, smem_per_sm):
    """Planned L2->SM words against Theorem 1 at one SM's S, and DRAM bytes
    against Theorem 1 at the chip's fast memory (L2 + all SMs) and against the
    compulsory bytes."""
    w_in = {"f64": 8, "f32": 4, "bf16": 2, "f64_emu_bf16": 2, "f32_emu_tf32": 4}[dtype]
    w_out = {"f64": 8, "f32": 4, "bf16": 4, "f64_emu_bf16": 8, "f32_emu_tf32": 4}[dtype]
    reg_or_tmem = 262144
    s_chip = (l2_bytes + sms * (smem_per_sm + reg_or_tmem)) / w_in
    passes = 1  # times the operands are read over: slice pairs, or TF32 parts
    compulsory = w_in * (m * k + k * n) + w_out * m * n
    if dtype == "f64_emu_bf16":
        slices = 6
        passes = slices * (slices + 1) // 2
        compulsory = w_in * slices * (m * k + k * n) + w_out * m * n
    if dtype == "f32_emu_tf32":
        # hi and lo parts of both operands: read as one product of inner dimension
        # 2k ([A_h A_l] times [B_h; B_l]), of which three of the four blocks are used
        passes = 2
        compulsory = w_in * 2 * (m * k + k * n) + w_out * m * n
    thm1_chip_words = passes * 2.0 * m * n * k / math.sqrt(s_chip) + m * n
    out = {"S_sm_words": plan.fast_words, "S_chip_words": s_chip,
           "l2_to_sm_words_planned": plan.io_words * passes,
           "theorem1_words_at_S_sm": passes * (plan.bound_words - m * n) + m * n,
           "dram_bytes_per_launch": traffic,
           "theorem1_bytes_at_S_chip": thm1_chip_words * w_in,
           "compulsory_bytes": compulsory,
           "operand_passes_per_call": passes}
    out["ratio_l2_sm"] = out["l2_to_sm_words_planned"] / out["theorem1_words_at_S_sm"]
    if traffic:
        out["ratio_dram_vs_theorem1_chip"] = traffic / out["theorem1_bytes_at_S_chip"]
        out["ratio_dram_vs_compulsory"] = traffic / compulsory
    return out


def workload_config(name, m, n, k, dtype):
    w = {"f64": 8, "f32": 4, "bf16": 2, "f64_emu_bf16": 8, "f32_emu_tf32": 4}[dtype]
    return {"workload": f"{name} m={m} n={n} k={k} {dtype} uniform[-1,1) seed 0",
            "m": m, "n": n, "k": k, "operands": "row-major, device-generated (Philox4x32-10)",
            "l2": "inputs larger than L2" if (m * k + k * n) * w > 130e6 else "inputs fit in L2"}


def combine_ranks(local_ms, flops_per_step, steps, world, dist=None, device=None):
    """Whole-job throughput: the slowest rank's timed region (max over ranks)
    against all ranks' work.  Returns (max_ms, TFLOP/s)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, world * flops_per_step * steps / (max_ms * 1e-3) / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.dev_id = dev_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        load = [s for s, p in zip(sm, power) if p > 200] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def _smi_id(torch, dev):
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        s = str(uuid)
        return s if s.startswith("GPU-") else "GPU-" + s
    return str(dev)


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline leg and the reference arm)


def oracle_sample(m, n, k, target_s, kind="uniform", gen="f64", seed=0, keep=False):
    """Time the oracle's plain product on an r x r corner of C (full k) sized
    to about target_s seconds.  Returns (flop/s, seconds, rows[, block])."""
    import numpy as np
    import cosma_inputs as ci
    from oracle import gemm as og

    def operand(x):
        if gen == "bf16":
            x = x.float().numpy()
        return np.asarray(x, dtype=np.float64)

    r = 32
    while True:
        A = operand(ci.rows(np.arange(r), k, kind, gen, seed, ci.STREAM_A))
        B = np.ascontiguousarray(operand(ci.cols(np.arange(r), k, n, kind, gen, seed,
                                                 ci.STREAM_B)).T)
        t0 = time.perf_counter()
        block = og.gemm(A, B, "naive")
        dt = time.perf_counter() - t0
        if dt >= target_s or r >= min(m, n):
            out = (2.0 * r * r * k / dt, dt, r)
            return out + (block,) if keep else out
        grow = math.sqrt(max(target_s / max(dt, 1e-3), 1.0))
        r = int(min(min(m, n), max(r + 1, r * min(grow, 4.0))))


def step_stats(step_ms):
    """Median, minimum and a 95 % confidence interval (Student t) of the mean of
    the timed steps' CUDA-event times."""
    n = len(step_ms)
    mean = sum(step_ms) / n
    out = {"median_ms": statistics.median(step_ms), "min_ms": min(step_ms), "mean_ms": mean}
    if n > 1:
        t975 = {2: 12.706, 3: 4.303, 4: 3.182, 5: 2.776, 6: 2.571, 7: 2.447, 8: 2.365,
                9: 2.306, 10: 2.262}.get(n, 1.96 if n > 30 else 2.23)
        half = t975 * statistics.stdev(step_ms) / math.sqrt(n)
        out["ci95_ms"] = [mean - half, mean + half]
    return out


def host_info():
    """Host cores and CPU model, for the CPU timings."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def tiled_sample(A_dev, B_dev, target_s):
    """Time the sequential schedule of Sec. 5.2 on the host cores: an
    r x r corner of C (full k) of the workload's own operands (their leading
    rows / columns copied from the device), a x b tiles from FindSeqSchedule at
    S = 32768 doubles (256 KB, a core's cache), tiles over all OpenMP threads;
    r is sized from one probe to take about target_s seconds.  Returns
    (flop/s, seconds, r, threads, a, b)."""
    import numpy as np
    from oracle import bounds
    from oracle import gemm as og

    m, k = A_dev.shape
    n = B_dev.shape[1]
    a, b = bounds.find_seq_schedule(32768)
    # probe with about four tiles per core, so the probe's rate is the run's
    r = min(a * int(math.ceil(math.sqrt(4 * (os.cpu_count() or 1)))), m, n)
    for attempt in range(2):
        A = np.ascontiguousarray(A_dev[:r].double().cpu().numpy())
        B = np.ascontiguousarray(B_dev[:, :r].double().cpu().numpy())
        t0 = time.perf_counter()
        _, used = og.tiled(A, B, a, b)
        dt = time.perf_counter() - t0
        if attempt == 1 or dt >= target_s or r >= min(m, n):
            break
        r = int(min(min(m, n), r * math.sqrt(target_s / max(dt, 1e-3))))
    return 2.0 * r * r * k / dt, dt, r, used, a, b


GROUPED_WORKLOAD = ("grouped: 512 independent products, m,n,k log-uniform in [64,4096] "
                    "seed 1")


def grouped_oracle_sample(dims, target_s):
    """Time the oracle's plain product over the first problems of a grouped
    workload for about target_s seconds (a problem above 3e8 multiply-adds
    contributes the 64 x 64 leading corner of its C, full k; input generation
    is inside the time).  Returns (flop, seconds, problems)."""
    import numpy as np
    import cosma_inputs as ci
    from oracle import gemm as og
    t0 = time.perf_counter()
    done, i = 0.0, 0
    while time.perf_counter() - t0 < target_s and i < len(dims):
        m, n, k = (int(x) for x in dims[i])
        A = np.asarray(ci.matrix(m, k, "uniform", "f32", 1000 + i, ci.STREAM_A), np.float64)
        B = np.asarray(ci.matrix(k, n, "uniform", "f32", 1000 + i, ci.STREAM_B), np.float64)
        if m * n * k > 3e8:
            A, B = A[:64], B[:, :64]
        og.gemm(A, B, "naive")
        done += 2.0 * A.shape[0] * B.shape[1] * k
        i += 1
    return done, time.perf_counter() - t0, i


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    dtype = args.dtype
    vals, secs = [], []
    if args.workload == "grouped512":
        import cosma_inputs as ci
        dims = ci.grouped_dims(512, seed=1)
        count = 0
        for i in range(args.warmup + args.steps):
            fl, dt, count = grouped_oracle_sample(dims, 8.0 if i >= args.warmup else 2.0)
            if i >= args.warmup:
                vals.append(fl / dt)
                secs.append(dt)
        sample = (f"oracle naive loop over the first {count} problems (>3e8 MACs: 64x64 "
                  "corner), incl. input generation")
        config = {"workload": GROUPED_WORKLOAD, "l2": "inputs larger than L2"}
        ms_per_step = statistics.median(secs) * 1e3
        value = statistics.median(vals) / 1e12
    else:
        m, n, k = WORKLOADS[args.workload]
        gen = "f32" if dtype in ("f32", "f32_emu_tf32") else "f64"
        rows = None
        for i in range(args.warmup + args.steps):
            fl, dt, rows = oracle_sample(m, n, k, 8.0 if i >= args.warmup else 2.0, gen=gen)[:3]
            if i >= args.warmup:
                vals.append(fl)
        value = statistics.median(vals) / 1e12
        sample = f"oracle naive FP64 loop on the {rows}x{rows} leading block of C, full k={k}"
        config = workload_config(args.workload, m, n, k, dtype)
        ms_per_step = 2.0 * rows * rows * k / (value * 1e12) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------


def run_grouped(args):
    """512 independent products in one persistent grouped launch, replayed from a
    CUDA graph; compared with one cosma_gemm launch per product."""
    import numpy as np
    import torch
    from paper_1908_09606_gb300 import cosma
    from cosma_inputs import device as cid
    import cosma_inputs as ci
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    cosma.load()
    dtype = "bf16" if args.dtype not in ("f32", "bf16") else args.dtype
    g = "bf16" if dtype == "bf16" else "f32"
    tdt = torch.bfloat16 if g == "bf16" else torch.float32
    dims = ci.grouped_dims(512, seed=1)
    # Row pitches padded to 16 bytes (B loaded as it is, C written by tensor stores).
    pad = 8 if g == "bf16" else 4
    rup = lambda x, r: -(-int(x) // r) * r
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(dims):
        A = torch.empty((m, rup(k, pad)), dtype=tdt, device="cuda")[:, :k]
        B = torch.empty((k, rup(n, pad)), dtype=tdt, device="cuda")[:, :n]
        cid.fill(A, "uniform", g, 1000 + i + 100000 * rank, ci.STREAM_A)
        cid.fill(B, "uniform", g, 1000 + i + 100000 * rank, ci.STREAM_B)
        As.append(A)
        Bs.append(B)
        Cs.append(torch.empty((m, rup(n, 4)), dtype=torch.float32, device="cuda")[:, :n])
    flops = float((2 * dims.prod(axis=1)).sum())
    # tile width by the autotuner (eager launches, before the graph is captured)
    from paper_1908_09606_gb300 import autotune
    tile, tile_ms = autotune.tune_grouped(
        As, Bs, Cs, dtype, tiles=(args.grouped_tile,) if args.grouped_tile else None)
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        cosma.gemm_grouped(As, Bs, Cs, dtype)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cosma.gemm_grouped(As, Bs, Cs, dtype)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(_smi_id(torch, local))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    reps = 20  # graph replays per step: one replay is ~1 TFLOP
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    l0 = cosma.cosma_launch_count()
    evs[0].record(stream)
    for i in range(args.steps):
        for _ in range(reps):
            graph.replay()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms, value = combine_ranks(sum(evs[i].elapsed_time(evs[i + 1])
                                        for i in range(args.steps)),
                                    flops * reps, args.steps, world, dist, "cuda")
    replay_ms = total_ms / (args.steps * reps)
    # library kernels per replay: the grouped prep (bf16) and the grouped GEMM
    per_replay = 2 if dtype == "bf16" else 1
    launches = per_replay * reps * args.steps
    # dominant kernel time from an eager, profiled call
    cosma.cosma_profile_read()
    cosma.cosma_profile_enable(True)
    for _ in range(3):
        cosma.gemm_grouped(As, Bs, Cs, dtype)
    torch.cuda.synchronize()
    cosma.cosma_profile_enable(False)
    kms, kn = cosma.cosma_profile_read()
    kms /= max(kn, 1)
    # one launch per product, same operands
    code = cosma.DTYPES[dtype]
    sh = stream.cuda_stream

    def per_gemm():
        for A, B, C in zip(As, Bs, Cs):
            m, k = A.shape
            n = B.shape[1]
            rc = cosma.cosma_gemm(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                  C.data_ptr(), C.stride(0), code, sh)
            if rc != 0:
                raise cosma.CosmaError(rc, "per-gemm baseline")
    per_gemm()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        per_gemm()
    e1.record(stream)
    torch.cuda.synchronize()
    pg_ms = e0.elapsed_time(e1) / 3
    peaks, peak_src = _peaks()
    if dtype == "bf16":
        kname = {512: "grouped_pair_kernel", 256: "grouped_tc_kernel<256,4>",
                 128: "grouped_tc_kernel<128,6>"}.get(tile, "grouped_tc_kernel")
        roof = {"kernel": kname, "bound": "tensor",
                "peak": peaks.get("bf16_tflops_sustained", 1700.0),
                "peak_source": f"bf16_tflops_sustained of {peak_src} peaks"}
    else:
        roof = {"kernel": "grouped_f32_kernel", "bound": "alu",
                "peak": _alu_peak_tflops("f32", torch.cuda.get_device_properties(local)
                                         .multi_processor_count),
                "peak_source": "derived: SMs x 128 FMA/clk x 2 x 2070 MHz"}
    roof.update({"achieved": flops / (kms * 1e-3) / 1e12, "unit": "TFLOP/s",
                 "algorithmic": "sum of 2mnk over the 512 products per launch",
                 "kernel_ms": kms,
                 "traffic": DRAM_TRAFFIC.get(("grouped512", dtype, tile)
                                             if tile == 512 else ("grouped512", dtype))
                 if dtype != "bf16" or tile in (256, 512) else None})
    roof["frac"] = roof["achieved"] / roof["peak"]
    # e2e: operands copied in from pinned host memory, one result read back
    Ah = [a.cpu().pin_memory() for a in As]
    Bh = [b.cpu().pin_memory() for b in Bs]
    Ch = [torch.empty(c.shape, dtype=c.dtype, pin_memory=True) for c in Cs]
    e0.record(stream)
    for A, B, a, b in zip(As, Bs, Ah, Bh):
        A.copy_(a, non_blocking=True)
        B.copy_(b, non_blocking=True)
    graph.replay()
    for C, c in zip(Cs, Ch):
        c.copy_(C, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1)
    esz = 2 if dtype == "bf16" else 4
    e2e = {"value": world * flops / (ems * 1e-3) / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": int(sum(a.numel() + b.numel() for a, b in zip(As, Bs)) * esz),
           "d2h_bytes_per_step": int(sum(c.numel() for c in Cs) * 4), "steps": 1}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        done, dt, i = grouped_oracle_sample(dims, 12.0)
        cpu = {"value": done / dt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle naive loop over the first {i} problems "
                         f"(>3e8 MACs: 64x64 corner), {dt:.1f} s incl. input generation"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": dtype, "data": "synthetic",
                "config": {"workload": GROUPED_WORKLOAD + ", one persistent launch replayed "
                                       f"from a CUDA graph ({reps} replays per step)",
                           "flops_per_replay": flops, "replay_ms": replay_ms,
                           "pitches": "rows padded to 16 bytes",
                           "l2": "inputs larger than L2",
                           "autotuned_tile": {"chosen": tile,
                                              "eager_ms": {str(t): v for t, v in tile_ms.items()}}},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks,
                "one_launch_per_gemm": {"value": flops / (pg_ms * 1e-3) / 1e12,
                                        "unit": "TFLOP/s", "ms": pg_ms,
                                        "grouped_speedup": pg_ms / replay_ms}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "grouped512":
        return run_grouped(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1908_09606_gb300 import cosma
    from cosma_inputs import device as cid
    import cosma_inputs as ci
    cosma.load()

    m, n, k = WORKLOADS[args.workload]
    dtype = args.dtype
    code = cosma.DTYPES[dtype]
    gen = {"f64": "f64", "f32": "f32", "bf16": "bf16", "f64_emu_bf16": "f64",
           "f32_emu_tf32": "f32"}[dtype]
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[gen]
    out_dt = torch.float32 if dtype in ("f32", "bf16", "f32_emu_tf32") else torch.float64
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    A = torch.empty((m, k), dtype=tdt, device=dev)
    B = torch.empty((k, n), dtype=tdt, device=dev)
    C = torch.empty((m, n), dtype=out_dt, device=dev)
    cid.fill(A, "uniform", gen, seed=rank, stream_id=ci.STREAM_A)
    cid.fill(B, "uniform", gen, seed=rank, stream_id=ci.STREAM_B)
    plan = cosma.cosma_plan_query(m, n, k, code)

    def step():
        rc = cosma.cosma_gemm(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, code, sh)
        if rc != 0:
            raise cosma.CosmaError(rc, "cosma_gemm")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = cosma.cosma_stream_status(sh)
    if st != 0:
        raise cosma.CosmaError(st, "device status after warm-up")

    sampler = ClockSampler(_smi_id(torch, local))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = cosma.cosma_launch_count()
    cosma.cosma_profile_read()          # drop anything recorded before
    cosma.cosma_profile_enable(True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = cosma.cosma_launch_count() - launches0
    cosma.cosma_profile_enable(False)
    kern_total_ms, kern_n = cosma.cosma_profile_read()
    clocks = sampler.stop()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    flops = 2.0 * m * n * k
    total_ms, value = combine_ranks(sum(step_ms), flops, args.steps, world, dist, dev)
    st = cosma.cosma_stream_status(sh)
    if st != 0:
        raise cosma.CosmaError(st, "device status after timed region")

    # Roofline of the dominant kernel, timed by the library's event pair around it.
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    kern_ms = kern_total_ms / max(kern_n, 1)
    cfg_lib = cosma.cosma_get_config()
    slices = cfg_lib.emu_slices or 6
    pairs = slices * (slices + 1) // 2
    if dtype in ("f64", "f32"):
        roof = {"kernel": "simt_f32_kernel" if dtype == "f32" else "simt_gemm_kernel<double>",
                "bound": "alu",
                "achieved": flops / (kern_ms * 1e-3) / 1e12,
                "peak": _alu_peak_tflops(dtype, sms), "unit": "TFLOP/s",
                "peak_source": "derived: SMs x FMA lanes/clk x 2 x 2070 MHz",
                "algorithmic": "2mnk flop per launch"}
    elif dtype == "f32_emu_tf32":
        # tf32 peak: the measured bf16 peak x the nominal tf32 / bf16 ratio (1.1 / 2.25)
        roof = {"kernel": "tf32x3_gemm_kernel", "bound": "tensor",
                "achieved": 3 * flops / (kern_ms * 1e-3) / 1e12,
                "peak": peaks.get("bf16_tflops_sustained", 1700.0) * 1.1 / 2.25,
                "unit": "TFLOP/s",
                "peak_source": f"bf16_tflops_sustained of {peak_src} peaks x 1.1/2.25 "
                               "(nominal dense tf32 / bf16)",
                "algorithmic": "3 part products x 2mnk tf32 flop per launch"}
    else:
        work = flops * (pairs if dtype == "f64_emu_bf16" else 1)
        if dtype == "f64_emu_bf16":
            kname = (f"emu_pair_kernel<{plan.tile_n}>" if plan.tile_m == 256
                     else "emu_gemm_kernel")
        else:
            kname = "tc_gemm_kernel"
        roof = {"kernel": kname,
                "bound": "tensor", "achieved": work / (kern_ms * 1e-3) / 1e12,
                "peak": peaks.get("bf16_tflops_sustained", 1700.0), "unit": "TFLOP/s",
                "peak_source": f"bf16_tflops_sustained of {peak_src} peaks",
                "algorithmic": (f"{pairs} slice-pair products x 2mnk bf16 flop per launch"
                                if dtype == "f64_emu_bf16" else "2mnk flop per launch")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = DRAM_TRAFFIC.get((args.workload, dtype))
    if roof["kernel"].startswith("emu_pair_kernel"):
        roof["traffic_note"] = (
            "ncu cannot launch the cooperative cluster kernel: traffic is the same lock-step "
            "schedule captured under a plain cluster launch (COSMA_EMU_LOCKSTEP=2)"
            + (DRAM_SCALED.get((args.workload, dtype), "")) if roof["traffic"] is not None else
            "null: no capture of this workload's lock-step schedule")
    if roof["kernel"] == "tf32x3_gemm_kernel" and roof["traffic"] is not None:
        roof["traffic_note"] = ("captured with the lock-step ticks under a plain launch "
                                "(COSMA_TF32_LOCKSTEP=2); the bench launches cooperatively")
    roof["kernel_ms"] = kern_ms
    roof["kernel_launches_timed"] = kern_n

    # Native FP64 on the same operands, for "split-BF16 vs native FP64".
    native = None
    if dtype == "f64_emu_bf16" and not args.no_native:
        Cn = torch.empty_like(C)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = cosma.cosma_gemm(m, n, k, A.data_ptr(), k, B.data_ptr(), n, Cn.data_ptr(), n,
                              cosma.COSMA_F64, sh)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise cosma.CosmaError(rc, "native f64")
        nms = e0.elapsed_time(e1)
        native = {"value": flops / (nms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms": nms,
                  "speedup_of_emulated": (flops / (nms * 1e-3) / 1e12) and value /
                  (flops / (nms * 1e-3) / 1e12)}

    # End-to-end through the C ABI with HOST buffers: cosma_gemm_host copies the
    # page-locked operands in and the product out itself, every step.
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty((m, k), dtype=tdt, pin_memory=True)
        Bh = torch.empty((k, n), dtype=tdt, pin_memory=True)
        Ch = torch.empty((m, n), dtype=out_dt, pin_memory=True)
        Ah.copy_(A)
        Bh.copy_(B)
        torch.cuda.synchronize()

        def host_step():
            rc = cosma.cosma_gemm_host(m, n, k, Ah.data_ptr(), k, Bh.data_ptr(), n,
                                       Ch.data_ptr(), n, code, sh)
            if rc != 0:
                raise cosma.CosmaError(rc, "cosma_gemm_host")

        for _ in range(2):  # sizes the library's device staging (outside the timed region)
            host_step()
        torch.cuda.synchronize()
        # this box's page-locked copy rates (1 GiB each way), context for the e2e figure
        nb = min(Ah.numel(), (1 << 30) // Ah.element_size())
        src_h, dst_d = Ah.view(-1)[:nb], A.view(-1)[:nb].clone()
        rates = {}
        for name, fn in (("h2d", lambda: dst_d.copy_(src_h, non_blocking=True)),
                         ("d2h", lambda: src_h.copy_(dst_d, non_blocking=True))):
            fn()
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record()
            fn()
            c1.record()
            torch.cuda.synchronize()
            rates[name] = nb * Ah.element_size() / (c0.elapsed_time(c1) * 1e-3) / 1e9
        del dst_d
        e_steps = max(1, min(args.steps, 5))
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(e_steps + 1)]
        if world > 1:
            dist.barrier()
        evs[0].record(stream)
        for i in range(e_steps):
            host_step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        e0, e1 = evs[0], evs[-1]
        per_call = [round(evs[i].elapsed_time(evs[i + 1]), 2) for i in range(e_steps)]
        rows = slice(0, m, max(1, m // 64))
        diff = float((Ch[rows].double() - C[rows].cpu().double()).abs().max())
        ems = e0.elapsed_time(e1)
        # one more call, outside the timed region, with the library's phase events on
        phases = None
        if hasattr(cosma, "cosma_profile_host"):
            cosma.cosma_profile_enable(True)
            try:
                host_step()
                phases = {kk: (round(v, 2) if isinstance(v, float) else v)
                          for kk, v in cosma.cosma_profile_host().items()}
            finally:
                cosma.cosma_profile_enable(False)
                cosma.cosma_profile_read()
            torch.cuda.synchronize()
        tt = torch.tensor([ems], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ems = float(tt.item())
        esz = A.element_size()
        e2e = {"value": world * flops * e_steps / (ems * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": (m * k + k * n) * esz,
               "d2h_bytes_per_step": m * n * C.element_size(), "steps": e_steps,
               "api": "cosma_gemm_host (page-locked host A, B, C)",
               "copy_gbs": {kk: round(v, 1) for kk, v in rates.items()},
               "per_call_ms": per_call,
               "phases_ms": phases,
               "max_abs_diff_vs_device_path": diff}
        del Ah, Bh, Ch

    # CPU baseline: the oracle on a bounded block of the same product; its values
    # also give the error of the GPU results on that block.
    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import numpy as np
        from oracle import gemm as og
        gen_o = gen
        fl, dt, rows, ref = oracle_sample(m, n, k, 12.0, gen=gen_o, seed=rank, keep=True)
        cpu = {"value": fl / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle naive FP64 loop, {rows}x{rows} leading block of C, "
                         f"full k={k}, {dt:.1f} s"}
        got = C[:rows, :rows].double().cpu().numpy()
        errors = {"block": f"{rows}x{rows}", "this_path": og.normwise_rel_error(got, ref)}
        # the paper's tiled schedule on all host cores, beside the naive oracle
        fl1, dt1, r1, used1, ta1, tb1 = tiled_sample(A, B, 6.0)
        cpu["tiled_all_cores"] = {
            "value": fl1 / 1e12, "unit": "TFLOP/s", "cores": used1,
            "sample": f"Sec. 5.2 tiled schedule on the host: {ta1}x{tb1} C blocks over {used1} OpenMP "
                      f"threads, {r1}x{r1} leading block of C, full k={k}, {dt1:.1f} s"}
        cpu["host"] = host_info()
        if native is not None:
            errors["native_f64"] = og.normwise_rel_error(
                Cn[:rows, :rows].double().cpu().numpy(), ref)
            errors["tolerance_emulated"] = 1e-12

    props = torch.cuda.get_device_properties(local)
    smem_sm = getattr(props, "shared_memory_per_multiprocessor", 233472)
    if rank == 0:
        cfg = workload_config(args.workload, m, n, k, dtype)
        cfg["plan"] = {kk: (round(v, 6) if isinstance(v, float) else v)
                       for kk, v in plan.as_dict().items()}
        cfg["plan"]["kernel"] = cosma.KERNELS.get(plan.kernel, plan.kernel)
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16",
                          "f64_emu_bf16": "bf16 slices -> f64",
                          "f32_emu_tf32": "tf32 parts -> f32"}[dtype],
                "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "step_stats": step_stats(step_ms),
                "native_f64": native, "error_vs_oracle": errors,
                "io": io_report(m, n, k, dtype, plan, roof["traffic"],
                                props.L2_cache_size, props.multi_processor_count,
                                smem_sm)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
