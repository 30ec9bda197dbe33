#!/usr/bin/env python3
"""Benchmark of the GEMM hot path through the C ABI (one JSON line on rank 0).

A step is one C = A B on the chosen workload through cosma_gemm: plan
(FindSeqSchedule, ParallelizeSched/FitRanks), staged main loop, Reduce when the
plan splits k, and -- for the emulated dtype -- slice extraction and
recombination.  Inputs are generated on the device by the shared seeded
generator before the timed region and are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload square]
                  [--dtype f64_emu_bf16|f64|f32|bf16] [--impl reference]

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
    "emu8192": (8192, 8192, 8192),
    "4096": (4096, 4096, 4096),
    "512": (512, 512, 512),
}
DEFAULT_DTYPE = "f64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="square", choices=list(WORKLOADS))
    ap.add_argument("--dtype", default=DEFAULT_DTYPE,
                    choices=["f64", "f32", "bf16", "f64_emu_bf16"])
    ap.add_argument("--impl", default="cosma", choices=["cosma", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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


def workload_config(name, m, n, k, dtype):
    return {"workload": f"{name} m={m} n={n} k={k} {dtype} uniform[-1,1) seed 0",
            "m": m, "n": n, "k": k, "operands": "row-major, device-generated (Philox4x32-10)",
            "l2": "inputs larger than L2" if (m * k + k * n) * 2 > 130e6 else "inputs fit in L2"}


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


def oracle_sample(m, n, k, target_s, kind="uniform", gen="f64"):
    """Time the oracle's plain product on an r x r corner of C (full k) sized
    to about target_s seconds.  Returns (flop/s, seconds, rows)."""
    import numpy as np
    import cosma_inputs as ci
    from oracle import gemm as og
    r = 32
    while True:
        A = np.asarray(ci.rows(np.arange(r), k, kind, gen, 0, ci.STREAM_A), dtype=np.float64)
        B = np.asarray(ci.cols(np.arange(r), k, n, kind, gen, 0, ci.STREAM_B), dtype=np.float64).T
        B = np.ascontiguousarray(B)
        t0 = time.perf_counter()
        og.gemm(A, B, "naive")
        dt = time.perf_counter() - t0
        if dt >= target_s or r >= min(m, n):
            return 2.0 * r * r * k / dt, dt, r
        grow = math.sqrt(max(target_s / max(dt, 1e-3), 1.0))
        r = int(min(min(m, n), max(r + 1, r * min(grow, 4.0))))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    m, n, k = WORKLOADS[args.workload]
    dtype = args.dtype
    gen = "f32" if dtype == "f32" else "f64"
    vals = []
    rows = None
    for i in range(args.warmup + args.steps):
        fl, dt, rows = oracle_sample(m, n, k, 8.0 if i >= args.warmup else 2.0, gen=gen)
        if i >= args.warmup:
            vals.append(fl)
    value = statistics.median(vals) / 1e12
    sample = f"oracle naive FP64 loop on the {rows}x{rows} leading block of C, full k={k}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 2.0 * rows * rows * k / (value * 1e12) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, m, n, k, dtype),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

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
    gen = {"f64": "f64", "f32": "f32", "bf16": "bf16", "f64_emu_bf16": "f64"}[dtype]
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[gen]
    out_dt = torch.float32 if dtype in ("f32", "bf16") else torch.float64
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
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = cosma.cosma_launch_count() - launches0
    clocks = sampler.stop()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    flops = 2.0 * m * n * k
    value = world * flops * args.steps / (total_ms * 1e-3) / 1e12
    st = cosma.cosma_stream_status(sh)
    if st != 0:
        raise cosma.CosmaError(st, "device status after timed region")

    # Roofline of the dominant kernel: one launch per step unless k is split.
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    kern_ms = statistics.mean(step_ms)
    if dtype in ("f64", "f32"):
        peak = _alu_peak_tflops(dtype, sms)
        roof = {"bound": "alu", "achieved": flops / (kern_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": "derived: SMs x FMA lanes x 2 x max clock"}
    else:
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "tensor", "achieved": flops / (kern_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": f"bf16 sustained, {peak_src}"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["kernel_launches_per_step"] = 1 + (1 if plan.pk > 1 else 0)

    # End-to-end through the public API from pinned host buffers.
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty((m, k), dtype=tdt, pin_memory=True)
        Bh = torch.empty((k, n), dtype=tdt, pin_memory=True)
        Ch = torch.empty((m, n), dtype=out_dt, pin_memory=True)
        Ah.copy_(A)
        Bh.copy_(B)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        e0.record(stream)
        for _ in range(e_steps):
            A.copy_(Ah, non_blocking=True)
            B.copy_(Bh, non_blocking=True)
            step()
            Ch.copy_(C, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        tt = torch.tensor([ems], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ems = float(tt.item())
        esz = A.element_size()
        e2e = {"value": world * flops * e_steps / (ems * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": (m * k + k * n) * esz,
               "d2h_bytes_per_step": m * n * C.element_size(), "steps": e_steps}
        del Ah, Bh, Ch

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        fl, dt, rows = oracle_sample(m, n, k, 12.0, gen="f32" if dtype == "f32" else "f64")
        cpu = {"value": fl / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle naive FP64 loop, {rows}x{rows} leading block of C, "
                         f"full k={k}, {dt:.1f} s"}

    if rank == 0:
        cfg = workload_config(args.workload, m, n, k, dtype)
        cfg["plan"] = {kk: (round(v, 6) if isinstance(v, float) else v)
                       for kk, v in plan.as_dict().items()}
        cfg["plan"]["kernel"] = cosma.KERNELS.get(plan.kernel, plan.kernel)
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16",
                          "f64_emu_bf16": "bf16 slices -> f64"}[dtype],
                "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "io": {"l2_to_sm_words_planned": plan.io_words,
                       "theorem1_words_at_S": plan.bound_words,
                       "ratio": plan.io_words / plan.bound_words,
                       "S_words": plan.fast_words}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
