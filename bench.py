#!/usr/bin/env python
"""Throughput of fast adaptive bilateral filtering (Algorithm 1) on GB300.

One step = one fabf_filter call (the fused CUDA kernel) over one synthetic
1920x1080 image: box radius w = 20, degree N = 5, theta = f + zeta (zeta a
smooth field in [-20, 20]), sigma a smooth field in [5, 60], FP64 -- the
reference point (N = 5, w = 20) of the 1920x1080 sweep.  Inputs are resident
in HBM and rotate over 8 slots (8 x 34 MB > the 126 MB L2), so every step
reads cold inputs.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the
plain C implementation of Algorithm 1) on a bounded sample of the same
workload instead.  With N > 1 GPUs (torchrun) every rank filters its own
images (replicas; the method needs no exchange between GPUs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H_, W_, WR, NDEG = 1080, 1920, 20, 5
N_BLOBS = 200
METRIC = "FABF Mpix/s (N=5,w=20) & % of roofline vs plain FP64 form; served p50/p99 ms"
WORKLOAD = ("1920x1080 uint8 synthetic (200 blobs, 4 step edges, noise 10), box w=20, N=5, "
            "theta=f+zeta (zeta in [-20,20]), sigma in [5,60]")
# DRAM bytes (read + write) per launch of the fused FP64 kernel on this
# workload, from the ncu capture in profiles/ (scaled from 4096x4096 by pixel
# count); set to None whenever the kernel changes until it is re-captured.
NCU_TRAFFIC_BYTES = 30.8e6
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
FP64_FLOP_PER_SM_CLK = 4.0        # 2 DFMA per clock per SM (nominal 1.25 TFLOP/s FP64)


def fp64_flops_per_pixel(N: int) -> float:
    """Algorithmic FP64 work of one non-flat pixel (FMA = 2, div/sqrt = 1,
    erf/erfc/exp = 20 each): mu (N+1 div), fit 2(N+1)^2, t0 and lambda 5,
    I_0 and I_1 with 2 erf + 2 exp 95, recursion 4N, T1/T2 4(N+1), ratio 3."""
    return (N + 1) + 2 * (N + 1) ** 2 + 5 + 95 + 4 * N + 4 * (N + 1) + 3


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_slot_inputs(n_distinct: int, seed0: int):
    from paper_1811_02308_gb300 import synth
    return [synth.make_inputs(H_, W_, seed0 + i, n_blobs=N_BLOBS, zeta_range=(-20, 20),
                              sigma_range=(5, 60)) for i in range(n_distinct)]


def run_oracle_sample(inp, n_pix: int, seed: int):
    import oracle
    f, th, s = inp
    rng = np.random.default_rng(seed)
    ys = rng.integers(0, H_, n_pix)
    xs = rng.integers(0, W_, n_pix)
    t = time.perf_counter()
    oracle.fabf_pixels(f, th, s, WR, NDEG, ys, xs)
    return time.perf_counter() - t


def cpu_baseline(inp, target_s: float = 12.0):
    """The oracle as it stands, one host thread, on a bounded pixel sample."""
    import oracle
    oracle.build()
    t = run_oracle_sample(inp, 500, 1)
    n = int(min(2_000_000, max(500, 500 * target_s / max(t, 1e-6))))
    t = run_oracle_sample(inp, n, 2)
    return {"value": n / t / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": "%d random pixels of the 1920x1080 w=20 N=5 workload, %.1f s, 1 thread"
                      % (n, t)}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    inp = make_slot_inputs(1, 1000)[0]
    t = run_oracle_sample(inp, 300, 3)
    per_step_s = 4.0
    n_pix = int(max(300, 300 * per_step_s / max(t, 1e-6)))
    for i in range(args.warmup):
        run_oracle_sample(inp, max(50, n_pix // 20), 10 + i)
    ts = [run_oracle_sample(inp, n_pix, 100 + i) for i in range(args.steps)]
    tot = sum(ts)
    value = n_pix * args.steps / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_pixels_per_step": n_pix},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": "%d random pixels per step, 1 thread" % n_pix},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fabf", choices=["fabf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per launch of the fused kernel from an ncu capture")
    ap.add_argument("--profile", default=None, metavar="HxW",
                    help="profiling case: one input of this size, no end-to-end or CPU legs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)

    import torch

    from paper_1811_02308_gb300 import build, fabf
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    ctx = fabf.Context(device=local)
    dev = torch.device("cuda", local)

    global H_, W_
    n_distinct, n_slots = 4, 8
    if args.profile:
        H_, W_ = (int(v) for v in args.profile.lower().split("x"))
        n_distinct, n_slots = 1, 1
        args.no_cpu_baseline = True
    host = make_slot_inputs(n_distinct, 1000 + 17 * rank)
    slots = []
    for i in range(n_slots):
        f, th, s = host[i % n_distinct]
        slots.append((torch.from_numpy(f).to(dev), torch.from_numpy(th).to(dev),
                      torch.from_numpy(s).to(dev),
                      torch.empty((H_, W_), dtype=torch.float64, device=dev)))
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step(i):
        f, th, s, out = slots[i % n_slots]
        rc = fabf.load().fabf_filter(ctx.handle, f.data_ptr(), th.data_ptr(), s.data_ptr(), H_, W_,
                                     W_, WR, NDEG, out.data_ptr(), 1, sh)
        if rc != 0:
            raise fabf.FabfError(rc, "fabf_filter")

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    st, _ = fabf.fabf_get_status(ctx, sh)
    if st != 0:
        raise RuntimeError("warm-up status %d" % st)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        t_all0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step(i)
            ev[i][1].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    total_ms = t_all0.elapsed_time(t_all1)
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    st, nfb = fabf.fabf_get_status(ctx, sh)
    npix = H_ * W_
    value = ws * npix * args.steps / (total_ms / 1e3) / 1e6

    if args.profile:
        print(json.dumps({"profile": args.profile, "ms_per_step": total_ms / args.steps,
                          "status": st}), flush=True)
        ctx.close()
        return 0
    # end to end through the C ABI with pinned host buffers (copies inside)
    f, th, s = host[0]
    hf = torch.from_numpy(f).pin_memory()
    hth = torch.from_numpy(th).pin_memory()
    hs = torch.from_numpy(s).pin_memory()
    hout = torch.empty((H_, W_), dtype=torch.float64).pin_memory()
    lib = fabf.load()

    def e2e_call():
        rc = lib.fabf_filter(ctx.handle, hf.data_ptr(), hth.data_ptr(), hs.data_ptr(), H_, W_, W_, WR,
                             NDEG, hout.data_ptr(), 1, sh)
        if rc != 0:
            raise fabf.FabfError(rc, "fabf_filter (host buffers)")

    for _ in range(3):
        e2e_call()
    n_e2e = max(5, min(50, args.steps // 4))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_call()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e = {"value": ws * npix / e2e_s / 1e6, "unit": "Mpix/s",
           "h2d_bytes_per_step": npix * (1 + 4 + 4), "d2h_bytes_per_step": npix * 8}

    flops = fp64_flops_per_pixel(NDEG) * npix
    achieved = flops / (kern_ms / 1e3) / 1e12
    peak = SM_COUNT * SM_MAX_MHZ * 1e6 * FP64_FLOP_PER_SM_CLK / 1e12
    roofline = {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": args.traffic_bytes if args.traffic_bytes is not None else NCU_TRAFFIC_BYTES,
                "peak_source": "nominal FP64 (152 SM x 4 flop/clk x 2070 MHz)",
                "flops_per_pixel": fp64_flops_per_pixel(NDEG),
                "kernel_ms": kern_ms, "hbm_bytes_per_pixel": 17}
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H_, "W": W_, "w": WR, "N": NDEG,
                       "precision": "fp64", "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs rotate over 8 slots of 34 MB (> 126 MB L2)"},
            "roofline": roofline, "e2e": e2e, "clocks": clk.summary(), "gpu_launches": args.steps,
            "status": st, "fallback_pixels": nfb}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(host[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
