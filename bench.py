#!/usr/bin/env python3
"""Benchmark of the ILE hot path on one GB300 (or N independent replicas).

Workload: the single large solve — 3 detectors (H1, L1, V1), all 21 modes with
2 <= l <= 4, Q at 16384 Hz over 0.2 s (3277 samples), 1001 time bins over
+-50 ms, SNR-20 synthetic injection with noise, 1e6 extrinsic samples per step.
A step is one full pass of the hot path: draw 1e6 samples from the adaptive
sampling prior -> sort by sky cell -> time-marginalised ln L (float32 bulk,
float64 delays and sums) -> ln Z / n_eff / n_ESS reduction -> histogram
adaptation.  Metric: ln L sample-evaluations per second (each evaluation
includes the full 1001-bin time marginalisation).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent solve (its own intrinsic
point); value = samples of all ranks / the slowest rank's time ("weak").
`--impl reference` times the FP64 CPU oracle (the reference arm of this
project) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ile_synth as S  # noqa: E402

METRIC = "ILE lnL sample-evals/s"
UNIT = "sample-evals/s"
N_SAMPLES = 1_000_000
FP32_LANES_PER_SM = 128
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
PROFILE = os.path.join(ROOT, "profiles", "lnl_tc_single_large.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2505_11655_gb300", "csrc", "k_tile_tc.cu")


def workload_config(prob, n):
    return {
        "workload": "single large solve: 3 detectors (H1,L1,V1), 21 modes (l=2..4), Q 16384 Hz x 0.2 s, "
                    "1001 time bins over +-50 ms, SNR 20 + noise, 1e6 samples per step, FP32 path",
        "n_det": prob.n_det, "n_modes": prob.n_modes, "fs_hz": prob.fs, "n_q": prob.n_q, "n_t": prob.n_t,
        "samples_per_step": n, "step": "draw + sky sort + lnL/time marginal + lnZ reduce + adapt",
        "l2": "flushed between timed steps (256 MiB write)",
    }


def flops_per_sample(prob):
    """Algorithmic FP32 work of one time-marginalised sample evaluation:
    K (4 M T_w + 3 n_t) + 8 K M^2 + 3 n_t with T_w = (t_hi - t_lo) fs + 2."""
    K, M, nt = prob.n_det, prob.n_modes, prob.n_t
    tw = (prob.t_hi - prob.t_lo) * prob.fs + 2
    return K * (4 * M * tw + 3 * nt) + 8 * K * M * M + 3 * nt


def fp32_peak_tflops():
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def profile_traffic():
    """dram bytes per launch of the tiled likelihood kernel from the committed ncu
    summary, or None if the kernel source changed since it was captured."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"k_lnl_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    cur = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    return float(m.group(1)) if cur == h.group(1) else None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(prob, budget_s=12.0):
    """The FP64 oracle, as it stands, timed on this host's cores on a bounded
    sample of the same step (draw + lnL + reduce + adapt)."""
    import oracle
    oracle.build()
    P = oracle.Problem(prob)

    def step(n, it):
        sm = oracle.Sampler(n_bins=64, seed=1)
        t0 = time.perf_counter()
        th, lr, bins = sm.draw(n, it=it)
        ll = oracle.lnL(P, th)
        lnw = ll + lr
        oracle.reduce(lnw)
        sm.adapt(bins, lnw)
        return time.perf_counter() - t0

    t_small = step(500, 0)
    n = int(max(500, min(2_000_000, 500 * budget_s / max(t_small, 1e-6))))
    dt = step(n, 1)
    return {"value": n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} samples of the same workload (one draw+lnL+reduce+adapt pass), {dt:.1f} s"}


def emit(obj):
    print(json.dumps(obj), flush=True)


def run_reference(args, rank):
    if rank != 0:
        return
    prob = S.single_large_problem(point=0)
    import oracle
    oracle.build()
    P = oracle.Problem(prob)
    sm = oracle.Sampler(n_bins=64, seed=1)
    # size each step so that warm-up + timed steps take about two minutes
    t0 = time.perf_counter()
    th, lr, bins = sm.draw(400, it=0)
    oracle.lnL(P, th)
    per = (time.perf_counter() - t0) / 400
    n = int(max(200, min(N_SAMPLES, 120.0 / max(1, args.steps + args.warmup) / max(per, 1e-9))))
    times = []
    for g in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        th, lr, bins = sm.draw(n, it=g)
        ll = oracle.lnL(P, th)
        lnw = ll + lr
        oracle.reduce(lnw)
        sm.adapt(bins, lnw)
        dt = time.perf_counter() - t0
        if g >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = n * len(times) / tot
    cores = oracle.num_threads()
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": dict(workload_config(prob, n), reference="FP64 CPU oracle (oracle/ile_oracle.c), OpenMP"),
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"{n} samples per step of the same workload"},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2505_11655_gb300 as G

    torch.cuda.set_device(local_rank)
    G.load(build_if_missing=True)
    n = args.samples
    prob = S.single_large_problem(point=rank)
    stream = torch.cuda.Stream()
    ile = G.ILE(prob, precision=G.RIFT_FP32, max_samples=n, n_bins=64, seed=1 + rank, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ile.adapt(1, n)
    barrier()
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        gpu_id = None
    clk = Clocks(gpu_id)
    clk.start()
    step_ms, lnl_ms = [], []
    l0 = ile.kernel_launches()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ile.adapt(1, n)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        lnl_ms.append(r["time_ms"][1])
    launches = ile.kernel_launches() - l0
    barrier()
    clocks = clk.stop()
    total = sum(step_ms)
    if world > 1:
        t = torch.tensor([total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    value = n * args.steps * world / (total / 1e3)

    # end to end through the public API with host buffers: Q, U, V uploaded from
    # pinned memory and the result record read back inside the timed region
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k), np.complex128)).pin_memory().numpy()
           for k in ("Q", "U", "V")}
    h2d = sum(a.nbytes for a in pin.values())
    d2h = 4 + 8 * 6 + 8 * 8   # status word, pooled record, one iteration record
    e2e_t = []
    for _ in range(0 if args.quick else min(args.steps, 5)):
        barrier()
        t0 = time.perf_counter()
        ile.set_overlaps(pin["Q"], pin["U"], pin["V"])
        ile.adapt(1, n)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_t) if e2e_t else float("nan")
    if world > 1:
        t = torch.tensor([e2e_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = n * len(e2e_t) * world / e2e_total if e2e_t else None

    fps = flops_per_sample(prob)
    lnl_avg = statistics.mean(lnl_ms)
    achieved = fps * n / (lnl_avg / 1e3) / 1e12
    peak = fp32_peak_tflops()
    traffic = profile_traffic()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(prob, n),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "lnl_tc_kernel", "kernel_ms": lnl_avg,
                     "peak_basis": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (unit counts x max clock)",
                     "flops_per_sample": fps},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clocks,
        "lnZ_last": r["lnZ"], "n_eff_last": r["n_eff"],
    }
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.quick):
        out["cpu_baseline"] = cpu_baseline(prob)
    ile.close()
    if rank == 0:
        emit(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--samples", type=int, default=N_SAMPLES, help="samples per step (profiling cases only)")
    ap.add_argument("--quick", action="store_true", help="skip the end-to-end and CPU-baseline legs (profiling)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
