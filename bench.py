#!/usr/bin/env python3
"""Benchmark of the ILE hot path on one GB300 (or N independent replicas).

Workload: the single large solve — 3 detectors (H1, L1, V1), all 21 modes with
2 <= l <= 4, Q at 16384 Hz over 0.2 s (3277 samples), 1001 time bins over
+-50 ms, SNR-20 synthetic injection with noise, 1e6 extrinsic samples per step.
A step is one full pass of the hot path: draw 1e6 samples from the adaptive
sampling prior -> sort by sky cell -> time-marginalised ln L (float32 bulk,
float64 delays and sums) -> ln Z / n_eff / n_ESS reduction -> histogram
adaptation.  Metric: ln L sample-evaluations per second (each evaluation
includes the full 1001-bin time marginalisation).  The same line carries the rest of
the metric: a "batched" block (512 uneven solves as one CUDA graph: solves/s) and a
"serving" block (a Poisson stream of solves: solves/s, p50/p99 latency), each with a
fixed subset of its solves also run one at a time through the plain FP64 GPU path (the
same requests on both arms) and the |d ln Z| of the served results against it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent solve (its own intrinsic
point); value = samples of all ranks / the slowest rank's time ("weak").
`--impl reference` times the FP64 CPU oracle (the reference arm of this
project) on bounded samples of the same workload.

Other workloads (one JSON line each, same keys):
  --workload batched   512 uneven solves (1-3 detectors, 2-21 modes, 1e4-1e6
                       samples, 3 adaptive iterations each) as one CUDA graph;
                       solves/s against sequential FP32 and FP64 solves
  --workload high_snr  SNR-150 realisable injection, q=20-like mode hierarchy:
                       10 adaptive iterations x 1e6 samples in RIFT_MIXED, n_eff
                       per iteration, error of FP32 and MIXED against the FP64 path
  --workload serving   Poisson stream of solves of four sizes through rift_srv_*:
                       p50/p99 latency and solves/s against sequential FP64
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
# DRAM bytes of one 1e6-sample launch of the tensor-core likelihood kernel (a 2e5-sample
# ncu capture scaled by the samples, profiles/lnl_tc_single_large.md), keyed by the SHA-256
# of the tensor-core kernel's and the correction's sources; null for any other source.
TRAFFIC_SOURCES = [os.path.join(ROOT, "paper_2505_11655_gb300", "csrc", f) for f in ("k_tile_tc.cu", "k_fixup.cu")]
TRAFFIC_BY_SOURCE = {
    "3e98ac2b2f6e30de16cf5dde8c8e0c1c184a69bbe778eea4e7a9c189816e4061": 5.98e7,
    "02d8362c4117749bf193a68eea6c4ee9c70af5751d9d82631086b1437d6f8777": 5.97e7,
    "a1a0f3fa500f237d67cded3cf3f47eaac17dae8af6c99f541d525a7f85a14ff1": 6.03e7,
    "70258efe81120ca38cdd3f22b5ffc4ac29c4003ba3fdf3b4467adb6ac9f57fc1": 5.97e7,
}


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


def kernel_traffic():
    """DRAM bytes of one 1e6-sample likelihood stage from the recorded ncu capture, or None
    when the kernels' sources differ from the captured ones."""
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(f, "rb").read())
    return TRAFFIC_BY_SOURCE.get(h.hexdigest())


def measured_peaks():
    """The measured HBM copy and bf16 GEMM rates of this machine (MEASURED_PEAKS.json), else
    fixed fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path)), "of measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def unit_peaks(G):
    """This device's float32 FMA and tcgen05 kind::f16 rates, measured by the library's own
    microbenchmarks (rift_ile_peak_rate) before the timed region."""
    out = {}
    for name, what in (("fp32_fma_tflops", G.RIFT_PEAK_FP32_FMA), ("tc_f16_n128_tflops", G.RIFT_PEAK_TC_F16_N128),
                       ("tc_f16_n256_tflops", G.RIFT_PEAK_TC_F16_N256), ("ex2_tops", G.RIFT_PEAK_EX2),
                       ("fp64_fma_tflops", G.RIFT_PEAK_FP64_FMA)):
        try:
            out[name] = G.rift_ile_peak_rate(what)
        except Exception as e:   # a failed measurement is reported, not hidden
            out[name] = None
            out[name + "_error"] = str(e)
    return out


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
    # the plain configuration (2 detectors, 2 modes, 401 bins) in full: 1e4 samples
    P1 = oracle.Problem(S.plain_fp64_problem())
    sm1 = oracle.Sampler(n_bins=64, seed=1)
    t0 = time.perf_counter()
    th1, lr1, bins1 = sm1.draw(10000)
    oracle.reduce(oracle.lnL(P1, th1) + lr1)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} samples of the same workload (one draw+lnL+reduce+adapt pass), {dt:.1f} s",
            "plain_config_full": {"value": 10000 / dt1, "unit": UNIT,
                                  "sample": f"10000 samples of the plain configuration, {dt1:.2f} s"}}


def emit(obj):
    print(json.dumps(obj), flush=True)


def run_reference_other(args):
    """Reference arm of the batched / high-SNR / serving workloads: the FP64 oracle
    timed on bounded samples of each representative problem (one draw + lnL +
    reduce + adapt pass), converted to the workload's unit by the samples each
    solve evaluates."""
    import oracle
    oracle.build()
    if args.workload == "high_snr":
        items = [(S.high_snr_problem(snr=args.snr), 10, args.samples)]
        unit, metric = "sample-evals/s", "ILE lnL sample-evals/s (high-SNR adaptive, MIXED)"
    elif args.workload == "batched":
        items = [(p, 3, -(-n // 3)) for p, n in (S.batched_problem(i) for i in range(0, args.points, 64))]
        unit, metric = "solves/s", "ILE solves/s (batched uneven solves)"
    else:
        import paper_2505_11655_gb300 as G
        items = [(p, it, n) for _, p, it, n in serving_requests(G, 16)]
        unit, metric = "solves/s", "ILE serving solves/s (p50/p99 latency)"
    per_step = 100.0 / max(1, args.steps + args.warmup) / len(items)
    secs, samples, times = [], 0, []
    for g in range(args.warmup + args.steps):
        t_step, est = 0.0, []
        for j, (p, it, n) in enumerate(items):
            P = oracle.Problem(p)
            sm = oracle.Sampler(n_bins=64, seed=1 + j)
            m = 64
            t0 = time.perf_counter()
            th, lr, bins = sm.draw(m, it=g)
            ll = oracle.lnL(P, th)
            dt0 = time.perf_counter() - t0
            m = int(max(64, min(n, m * per_step / max(dt0, 1e-6))))
            t0 = time.perf_counter()
            th, lr, bins = sm.draw(m, it=g)
            ll = oracle.lnL(P, th)
            oracle.reduce(ll + lr)
            sm.adapt(bins, ll + lr)
            dt = time.perf_counter() - t0
            t_step += dt
            est.append(dt / m * it * n)   # seconds this solve would take
            samples = m
        if g >= args.warmup:
            times.append(t_step)
            secs.append(float(np.mean(est)))
    value = (args.samples * 10 / np.mean(secs)) if unit == "sample-evals/s" else 1.0 / np.mean(secs)
    cores = oracle.num_threads()
    sample = (f"{len(items)} representative problems, about {samples} samples each per step, "
              "scaled to each solve's sample count")
    emit({"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": args.workload, "reference": "FP64 CPU oracle (oracle/ile_oracle.c), OpenMP"},
          "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
          "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_reference(args, rank):
    if rank != 0:
        return
    if args.workload != "single_large":
        run_reference_other(args)
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
    value, total_s = aggregate_over_ranks(n * args.steps, sum(step_ms) / 1e3, world)
    total = 1e3 * total_s

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
    e2e_value = aggregate_over_ranks(n * len(e2e_t), sum(e2e_t), world)[0] if e2e_t else None

    # the overlaps computed on the device from the frequency-domain inputs (the stage the
    # paper runs on the CPU), against uploading precomputed Q, U, V
    pre = None
    if not args.quick:
        wf = prob.meta["waveforms"]
        fin = [np.ascontiguousarray(x) for x in (wf.freqs, wf.h, prob.meta["data"], wf.w)]
        tw, to = [], []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ile.set_waveforms(*fin)
            tw.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            ile.set_overlaps(pin["Q"], pin["U"], pin["V"])
            to.append(time.perf_counter() - t0)
        pre = {"set_waveforms_ms": 1e3 * statistics.median(tw), "set_overlaps_ms": 1e3 * statistics.median(to),
               "n_freq": int(wf.freqs.size), "complex_macs": int(prob.n_det * prob.n_modes * prob.n_q * wf.freqs.size)}
    # the same step with the distance marginalised in every time bin (5-D sampling)
    dm = None
    if not args.quick:
        with G.ILE(prob, precision=G.RIFT_FP32, max_samples=n, n_bins=64, seed=1 + rank, stream=stream,
                   distance_marg=True) as sdm:
            for _ in range(3):   # warm-up, including the adapted class's plan timing (third iteration)
                sdm.adapt(1, n)
            dms, dml = [], []
            for _ in range(3):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rd = sdm.adapt(1, n)
                e1.record(stream)
                e1.synchronize()
                dms.append(e0.elapsed_time(e1))
                dml.append(rd["time_ms"][1])
        dm = {"sample_evals_per_s": n / (statistics.mean(dms) / 1e3), "ms_per_step": statistics.mean(dms),
              "lnl_kernel_ms": statistics.mean(dml), "lnZ": rd["lnZ"], "n_eff": rd["n_eff"],
              "quadrature": "per bin: 2 panels x 10 Gauss-Legendre nodes in ln x (float32)"}
    # the portfolio sampling prior on the same problem and batch, over {histogram, AV} and
    # over {histogram, AV, Gaussian mixture}: per-iteration cost against the histogram
    # sampler's step above
    pfo = pfo3 = None
    if not args.quick:
        def run_pf(members, label):
            with G.ILE(prob, precision=G.RIFT_FP32, max_samples=n, n_bins=64, seed=1 + rank, stream=stream) as spf:
                kw = dict(members=members, p_thr=0.999, n_min_star=1000, gmm_components=4)
                spf.portfolio(2, n, restart=True, **kw)   # warm-up (allocation, kernels)
                torch.cuda.synchronize()
                n_pf = 8
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rp = spf.portfolio(n_pf, n, restart=True, **kw)
                e1.record(stream)
                e1.synchronize()
                pf_ms = e0.elapsed_time(e1)
                pinfo = spf.portfolio_info()
                av_info = spf.av_info()
            return {"iterations": n_pf, "samples_per_iter": n, "ms_per_iter": pf_ms / n_pf,
                    "histogram_ms_per_iter": statistics.mean(step_ms),
                    "sample_evals_per_s": n * n_pf / (pf_ms / 1e3), "lnZ": rp["lnZ"], "sigma_lnZ": rp["sigma_lnZ"],
                    "n_eff": rp["n_eff"], "lnZ_iter": rp["lnZ_iter"], "W_next": pinfo["W_next"],
                    "n_drawn_last": pinfo["n_drawn"], "n_ess_last": pinfo["n_ess"], "av_level": av_info["level"],
                    "av_volume": av_info["V"], "members": label}
        pfo = run_pf(G.RIFT_MEMBER_HIST | G.RIFT_MEMBER_AV,
                     "histogram (64 bins) + adaptive volume (p_thr 0.999, N_min* 1000)")
        pfo3 = run_pf(G.RIFT_MEMBER_HIST | G.RIFT_MEMBER_AV | G.RIFT_MEMBER_GMM,
                      "histogram (64 bins) + adaptive volume (p_thr 0.999, N_min* 1000) + Gaussian mixture (4 "
                      "components)")
    fps = flops_per_sample(prob)
    lnl_avg = statistics.mean(lnl_ms)
    achieved = fps * n / (lnl_avg / 1e3) / 1e12
    mp, basis = measured_peaks()
    peak = float(mp.get("bf16_tflops_sustained", mp.get("bf16_tflops")))
    plan = ile.plan()
    kernel = _lnl_kernel_name(G, plan)
    traffic = kernel_traffic() if plan[0] == G.RIFT_KERNEL_TENSOR else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(prob, n),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel + " + large-term correction (the likelihood stage)",
                     "samples_per_cell": plan[1], "kernel_ms": lnl_avg, "flops_per_sample": fps,
                     "peak_basis": f"dense 16-bit tensor rate {basis} (bf16 GEMM sustained, MEASURED_PEAKS.json; "
                                   "f16 has the same nominal rate), the likelihood stage being timed inside a "
                                   "long step",
                     "note": "achieved = algorithmic flops of the method (the mode contraction, 95% of them, is "
                             "a dense contraction the kernel runs on tcgen05 as a float16 hi/lo split) / the "
                             "likelihood stage's CUDA-event time.  The stage is bound by the per-step drain of "
                             "the accumulators into shared memory and the per-bin gather, not by the tensor "
                             "pipe (profiles/lnl_tc_single_large.md)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clocks,
        "lnZ_last": r["lnZ"], "n_eff_last": r["n_eff"], "precompute": pre, "distance_marg": dm,
        "portfolio": pfo,
        "portfolio_gmm": pfo3,
    }
    if not args.quick:
        up = unit_peaks(G)
        out["roofline"]["unit_peaks_measured"] = up
        if up.get("fp32_fma_tflops"):
            out["roofline"]["algorithmic_vs_fp32_fma"] = achieved / up["fp32_fma_tflops"]
        if up.get("tc_f16_n128_tflops"):
            out["roofline"]["frac_vs_tc_f16_n128_measured"] = achieved / up["tc_f16_n128_tflops"]
        if up.get("ex2_tops"):
            # one exponential per bin in the time marginal (the method's ex2 count)
            ex2_rate = prob.n_t * n / (lnl_avg / 1e3) / 1e12
            out["roofline"]["ex2_tops_achieved"] = ex2_rate
            out["roofline"]["frac_vs_ex2_measured"] = ex2_rate / up["ex2_tops"]
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.quick):
        out["cpu_baseline"] = cpu_baseline(prob)
    ile.close()
    if not (args.quick or args.no_workloads):
        # the rest of the metric: solves/s of the batched workload and solves/s with p50/p99
        # latency of the serving stream, each against the plain FP64 GPU path measured
        # directly on a fixed subset of the same solves
        clk2 = Clocks(gpu_id)
        clk2.start()
        out["batched"] = measure_batched(torch, G, rank, args.points, 2, 5)
        out["serving"] = measure_serving(torch, G, rank, args.requests)
        out["workload_clocks"] = clk2.stop()
    if rank == 0:
        emit(out)


# ======================================================================== other workloads

def _setup(local_rank):
    import torch

    import paper_2505_11655_gb300 as G
    torch.cuda.set_device(local_rank)
    G.load(build_if_missing=True)
    return torch, G


def _lnl_kernel_name(G, plan):
    return {G.RIFT_KERNEL_TENSOR: "lnl_tc_kernel", G.RIFT_KERNEL_CUDA_CORE: "lnl_tile_kernel",
            G.RIFT_KERNEL_FP64: "lnl_fp64_kernel"}[plan[0]]


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def aggregate_over_ranks(units, seconds, world):
    """Whole-job throughput of independent replicas: the units all ranks processed
    divided by the slowest rank's time; returns (value, slowest seconds)."""
    if world == 1:
        return units / seconds, seconds
    import torch
    import torch.distributed as dist
    dev = _reduce_device()
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def rank_points(rank, npts):
    """Intrinsic points of the batched workload on one rank (disjoint across ranks)."""
    return list(range(rank * npts, (rank + 1) * npts))


def _clock_monitor(torch, local_rank):
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        gpu_id = None
    return Clocks(gpu_id)


def _lnz_last_vs_fp64(G, s, prob, n, lnz_last):
    """|d ln Z| of a solve's last iteration against the plain FP64 GPU path on the same
    sample stream: the last batch's theta re-evaluated in float64, reduced the same way."""
    th, lr, ll, lw = s.last_batch(n)
    with G.ILE(prob, precision=G.RIFT_FP64, max_samples=min(n, 1 << 20)) as s64:
        l64 = s64.eval(th)
    x = l64 + lr
    m = float(np.max(x))
    return abs(lnz_last - (m + math.log(float(np.sum(np.exp(x - m)))) - math.log(n)))


def measure_batched(torch, G, rank, npts, warmup, steps, quick=False, fp64_every=32):
    """The batched workload: npts uneven solves (1-3 detectors, 2-21 modes, 1e4-1e6
    samples, 3 adaptive iterations of N/3) as one CUDA graph per step.  Returns solves/s
    and, unless quick, the same solves one at a time in float32, and a fixed subset of the
    points (every fp64_every-th) run both as a batch and one at a time through the plain
    FP64 GPU path (the same requests on both arms, no scaling), with each subset point's
    |d ln Z| against the FP64 path on the same sample stream."""
    pts = [S.batched_problem(i) for i in rank_points(rank, npts)]
    n_iter = 3
    nper = [max(1, -(-n // n_iter)) for _, n in pts]
    solves = [G.ILE(p, precision=G.RIFT_FP32, max_samples=m, n_bins=64, seed=1 + i)
              for i, ((p, _), m) in enumerate(zip(pts, nper))]
    stream = torch.cuda.Stream()
    batch = G.Batch(solves, [n_iter] * npts, nper, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        res, rc = batch.run()
        assert rc == 0, rc
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, rc = batch.run()
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, rc
        step_ms.append(e0.elapsed_time(e1))
    launches = batch.kernel_launches()
    kinds = {}
    for sv in solves:
        k = _lnl_kernel_name(G, sv.plan())
        kinds[k] = kinds.get(k, 0) + 1
    batch.close()
    ms = statistics.mean(step_ms)
    out = {"points": npts, "n_iter": n_iter, "samples_per_step": n_iter * sum(nper), "ms_per_step": ms,
           "solves_per_s": npts / (ms / 1e3), "sample_evals_per_s": n_iter * sum(nper) / (ms / 1e3),
           "steps": steps, "warmup": warmup, "lnl_kernels": kinds, "gpu_launches_per_step": launches,
           "l2": "flushed between timed steps (256 MiB write)"}
    if not quick:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sv, m in zip(solves, nper):
            sv.adapt(n_iter, m)
        out["fp32_one_at_a_time_solves_per_s"] = npts / (time.perf_counter() - t0)
        out["speedup_vs_fp32_one_at_a_time"] = out["solves_per_s"] / out["fp32_one_at_a_time_solves_per_s"]
        sub = list(range(0, npts, fp64_every))
        subsolves = [G.ILE(pts[i][0], precision=G.RIFT_FP32, max_samples=nper[i], n_bins=64, seed=1 + i)
                     for i in sub]
        sb = G.Batch(subsolves, [n_iter] * len(sub), [nper[i] for i in sub], stream=stream)
        sb.run()   # capture; the timed run below replays the graph (the next 3 iterations)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sres, rc = sb.run()
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        sb.close()
        dz = [_lnz_last_vs_fp64(G, sv, pts[i][0], nper[i], r["lnZ_iter"][-1])
              for sv, i, r in zip(subsolves, sub, sres)]
        for sv in subsolves:
            sv.close()
        t64 = 0.0
        for i in sub:
            with G.ILE(pts[i][0], precision=G.RIFT_FP64, max_samples=nper[i], n_bins=64, seed=1 + i) as s64:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s64.adapt(n_iter, nper[i])
                t64 += time.perf_counter() - t0
        out["fp64_subset"] = {
            "points": len(sub), "which": f"every {fp64_every}th point",
            "batched_fp32_solves_per_s": len(sub) / t_b, "fp64_one_at_a_time_solves_per_s": len(sub) / t64,
            "speedup_vs_fp64_one_at_a_time": t64 / t_b,
            "max_abs_dlnZ_vs_fp64": float(max(dz)),
            "dlnZ_basis": "each point's last iteration, its own samples re-evaluated by the FP64 GPU path"}
    for sv in solves:
        sv.close()
    return out


def run_batched(args, rank, world, local_rank):
    """512 uneven solves as one graph per step; solves/s."""
    torch, G = _setup(local_rank)
    clk = _clock_monitor(torch, local_rank)
    clk.start()
    b = measure_batched(torch, G, rank, args.points, args.warmup, args.steps, args.quick, fp64_every=16)
    clocks = clk.stop()
    value, total_s = aggregate_over_ranks(args.points * args.steps, b["ms_per_step"] * args.steps / 1e3, world)
    out = {
        "metric": "ILE solves/s (batched uneven solves)", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched uneven solves: {args.points} points per GPU, detectors 1-3, modes 2-21, "
                               "samples 1e4-1e6 log-uniform, 3 adaptive iterations of N/3, one CUDA graph per step",
                   "l2": b["l2"]},
        "batched": b, "e2e": None, "gpu_launches": b["gpu_launches_per_step"] * args.steps, "clocks": clocks,
    }
    if rank == 0:
        emit(out)


def realisable_high_snr(G, snr=150.0, point=0):
    """SNR-`snr` injection built from this library's own float64 coefficients
    F_k Y_lm at a fixed near-edge-on truth, so that the sampler can converge on it."""
    th_true = np.array([2.2, -0.5, 1.1, 0.7, 1.4, 300.0])
    probe = S.high_snr_problem(snr=snr, point=point)
    with G.ILE(probe, precision=G.RIFT_FP64, max_samples=16) as s:
        c, dt, _ = s.coeffs(th_true[None, :])
    a0 = c[0] * th_true[5] / probe.d_ref
    return S.high_snr_problem(snr=snr, point=point, a0=a0, dt_true=dt[0]), th_true


def run_high_snr(args, rank, world, local_rank):
    """10 adaptive iterations x 1e6 samples in RIFT_MIXED per step."""
    torch, G = _setup(local_rank)
    n, n_iter = args.samples, 10
    prob, th_true = realisable_high_snr(G, snr=args.snr, point=rank)
    stream = torch.cuda.Stream()
    ile = G.ILE(prob, precision=G.RIFT_MIXED, max_samples=n, n_bins=64, seed=1 + rank, stream=stream)
    for _ in range(args.warmup):
        ile.adapt(n_iter, n)
    torch.cuda.synchronize()
    clk = _clock_monitor(torch, local_rank)
    clk.start()
    step_ms, res = [], []
    l0 = ile.kernel_launches()
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ile.adapt(n_iter, n)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        res.append(r)
    launches = ile.kernel_launches() - l0
    clocks = clk.stop()
    value, total_s = aggregate_over_ranks(n * n_iter * args.steps, sum(step_ms) / 1e3, world)
    total = 1e3 * total_s
    r = res[-1]
    # fair draws from the last batch (sample by weight, then time bin by per-bin ln L)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fth, ft, fidx = ile.fair_draws(10000, seed=17)
    fair_ms = 1e3 * (time.perf_counter() - t0)
    # the adaptive-volume integrator on the same problem and budget (10 x n, MIXED)
    av_res = None
    if not args.quick:
        with G.ILE(prob, precision=G.RIFT_MIXED, max_samples=n, n_bins=64, seed=1 + rank, stream=stream) as sav:
            sav.av(2, n, restart=True)   # warm-up (allocation, kernels)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ra = sav.av(n_iter, n, restart=True)
            torch.cuda.synchronize()
            av_ms = 1e3 * (time.perf_counter() - t0)
            info = sav.av_info()
        av_res = {"ms_per_step": av_ms, "sample_evals_per_s": n * n_iter / (av_ms / 1e3), "lnZ": ra["lnZ"],
                  "sigma_lnZ": ra["sigma_lnZ"], "n_eff": ra["n_eff"], "n_eff_iter": ra["n_eff_iter"],
                  "lnZ_iter": ra["lnZ_iter"], "final_level": info["level"], "final_cells": info["n_cells"],
                  "final_volume": info["V"], "p_thr": 0.9999, "n_min_star": 1000}
    # the portfolio on the same problem and budget (10 x n, MIXED): {histogram, AV},
    # {histogram, AV, Gaussian mixture} and the Gaussian mixture alone
    pf_res = {}
    if not args.quick:
        for label, members in (("histogram+av", G.RIFT_MEMBER_HIST | G.RIFT_MEMBER_AV),
                               ("histogram+av+gmm", G.RIFT_MEMBER_HIST | G.RIFT_MEMBER_AV | G.RIFT_MEMBER_GMM),
                               ("gmm", G.RIFT_MEMBER_GMM)):
            with G.ILE(prob, precision=G.RIFT_MIXED, max_samples=n, n_bins=64, seed=1 + rank, stream=stream) as spf:
                spf.portfolio(2, n, members=members, restart=True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rp = spf.portfolio(n_iter, n, members=members, restart=True)
                torch.cuda.synchronize()
                pf_ms = 1e3 * (time.perf_counter() - t0)
                pinfo = spf.portfolio_info()
            pf_res[label] = {"ms_per_step": pf_ms, "sample_evals_per_s": n * n_iter / (pf_ms / 1e3),
                             "lnZ": rp["lnZ"], "sigma_lnZ": rp["sigma_lnZ"], "n_eff": rp["n_eff"],
                             "n_eff_iter": rp["n_eff_iter"], "lnZ_iter": rp["lnZ_iter"], "W_next": pinfo["W_next"],
                             "n_drawn_last": pinfo["n_drawn"], "frozen_last": pinfo["frozen"], "p_thr": 0.9999,
                             "n_min_star": 1000, "gmm_components": 4}
    # error of the last batch against the float64 path (1e-9 parity with the oracle):
    # every sample within 30 of the largest ln w, plus 4096 others
    th, lr, ll, lw = ile.last_batch(n)
    heavy = np.nonzero(lw >= lw.max() - 30.0)[0]
    rest = np.random.default_rng(5).choice(n, 4096, replace=False)
    idx = np.unique(np.concatenate([heavy, rest]))
    with G.ILE(prob, precision=G.RIFT_FP64, max_samples=len(idx)) as s64:
        l64 = s64.eval(th[idx])
    with G.ILE(prob, precision=G.RIFT_FP32, max_samples=len(idx)) as s32:
        l32 = s32.eval(th[idx])

    def lse(x):
        m = x.max()
        return m + math.log(np.exp(x - m).sum())

    def lnz_with(vals):
        lnw = ll + lr
        lnw = lnw.copy()
        lnw[idx] = vals + lr[idx]
        return lse(lnw) - math.log(n)

    ref = lnz_with(l64)
    err = {"mixed": {"max_abs_dlnL_heavy": float(np.max(np.abs(ll[idx] - l64)[np.isin(idx, heavy)])),
                     "abs_dlnZ_last_iter": abs(lnz_with(ll[idx]) - ref)},
           "fp32": {"max_abs_dlnL_heavy": float(np.max(np.abs(l32 - l64)[np.isin(idx, heavy)])),
                    "abs_dlnZ_last_iter": abs(lnz_with(l32) - ref)},
           "reference": "float64 GPU path on the same theta (parity 1e-9 with the FP64 oracle)",
           "samples_compared": int(len(idx)), "heavy_samples": int(len(heavy))}
    ile.close()
    out = {
        "metric": "ILE lnL sample-evals/s (high-SNR adaptive, MIXED)", "value": value, "unit": "sample-evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"high-SNR narrow source: SNR {args.snr:g}, realisable injection (iota 1.4 rad), "
                               "q=20-like hierarchy, 3 detectors, 21 modes, 16384 Hz, 1001 bins, "
                               f"{n_iter} adaptive iterations x {n} samples per step, RIFT_MIXED",
                   "n_iter": n_iter, "samples_per_iter": n, "l2": "inputs (theta 48 MB/iter) exceed L2"},
        "result": {"lnZ": r["lnZ"], "sigma_lnZ": r["sigma_lnZ"], "n_eff": r["n_eff"], "n_ess": r["n_ess"],
                   "lnL_max": r["lnL_max"], "n_eff_iter": r["n_eff_iter"], "lnZ_iter": r["lnZ_iter"]},
        "error_vs_fp64": err,
        "adaptive_volume": av_res,
        "portfolio": pf_res,
        "fair_draws": {"draws": 10000, "ms": fair_ms, "distinct_samples": int(len(np.unique(fidx))),
                       "t_spread_ms": float(1e3 * np.std(ft))},
        "stage_ms_per_step": {"draw_sort": r["time_ms"][0], "lnl_refine": r["time_ms"][1],
                              "reduce_adapt": r["time_ms"][2]},
        "e2e": None, "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0:
        emit(out)


def serving_requests(G, count, seed=17):
    """Request mixture: 40% plain (2 det, 2 modes, 1e4 samples, 1 iteration), 30%
    batched-workload points (3 iterations of N/3), 20% single large (1e6, 1
    iteration), 10% high-SNR (2 iterations x 1e6).  Problems come from a pool of
    distinct seeded points; each request has its own sampler seed."""
    pool = {"plain": [S.plain_fp64_problem(i) for i in range(8)],
            "batched": [S.batched_problem(100 + i) for i in range(32)],
            "large": [S.single_large_problem(i) for i in range(2)],
            "high_snr": [S.high_snr_problem(snr=120.0, point=i) for i in range(2)]}
    rng = np.random.default_rng(seed)
    kinds = rng.choice(["plain", "batched", "large", "high_snr"], size=count, p=[0.4, 0.3, 0.2, 0.1])
    reqs = []
    for i, k in enumerate(kinds):
        j = int(rng.integers(len(pool[k])))
        if k == "plain":
            reqs.append((k, pool[k][j], 1, 10000))
        elif k == "batched":
            p, n = pool[k][j]
            reqs.append((k, p, 3, max(1, -(-n // 3))))
        elif k == "large":
            reqs.append((k, pool[k][j], 1, 1_000_000))
        else:
            reqs.append((k, pool[k][j], 2, 1_000_000))
    return reqs


def _precision(G, kind):
    """Precision of a request: RIFT_MIXED (float64 re-evaluation of the weighted samples)
    for the high-SNR points, whose ln L ~ 1e4 puts float32 rounding above 1e-3; float32
    for the SNR ~20 points, where it meets the 1e-3 bar."""
    return G.RIFT_MIXED if kind == "high_snr" else G.RIFT_FP32


def _serve(G, reqs, rate, budget, slots):
    """Submit `reqs` (all at once if rate is None, else Poisson arrivals at `rate`
    per second); completions with their server-side times."""
    rng = np.random.default_rng(3)
    with G.Server(hbm_budget_bytes=budget, max_slots=slots) as srv:
        t0 = time.perf_counter()
        t_next = 0.0
        got = []
        for i, (k, p, it, n) in enumerate(reqs):
            if rate is not None:
                t_next += rng.exponential(1.0 / rate)
                while True:
                    dt = t0 + t_next - time.perf_counter()
                    if dt <= 0:
                        break
                    got += srv.poll(256, 0)
                    time.sleep(min(dt, 0.002))
            srv.submit(p, it, n, i, precision=_precision(G, k), seed=1 + i)
        got += srv.drain(len(reqs) - len(got))
    return got


def _latency_stats(got):
    lat = np.array([c["t_done_ms"] - c["t_submit_ms"] for c in got])
    span = (max(c["t_done_ms"] for c in got) - min(c["t_submit_ms"] for c in got)) / 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves_per_s": len(got) / span, "span_s": span,
            "failed": int(sum(c["status"] != 0 for c in got))}


def measure_serving(torch, G, rank, n_requests, quick=False, fp64_every=50):
    """The serving stream: n_requests solves of four sizes through rift_srv_* (admission
    by HBM footprint): saturated, then Poisson arrivals at 0.8x and 1.2x the saturated
    rate.  Unless quick: every request one at a time at its served precision, and a fixed
    subset (every fp64_every-th request) served on its own and run one at a time through
    the plain FP64 GPU path (the same requests on both arms, no scaling), with each subset
    request's |d ln Z| against the FP64 path on the same sample stream (a solve's result is
    the same alone and in the mix, bitwise: tests/test_gpu_serve.py)."""
    reqs = serving_requests(G, n_requests, seed=17 + rank)
    budget, slots = 96 << 30, 16
    _serve(G, reqs[:64], None, budget, slots)   # warm-up: kernels, tuner classes, pool
    sat = _latency_stats(_serve(G, reqs, None, budget, slots))
    lam = sat["solves_per_s"]
    at08 = _latency_stats(_serve(G, reqs, 0.8 * lam, budget, slots))
    at12 = _latency_stats(_serve(G, reqs, 1.2 * lam, budget, slots))
    mix = {k: int(sum(r[0] == k for r in reqs)) for k in ("plain", "batched", "large", "high_snr")}
    out = {"requests": n_requests, "mix": mix, "hbm_budget_bytes": budget, "max_slots": slots,
           "saturated": sat, "poisson_0.8x": at08, "poisson_1.2x": at12}
    if quick:
        return out
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (k, p, it, n) in enumerate(reqs):
        with G.ILE(p, precision=_precision(G, k), max_samples=n, n_bins=64, seed=1 + i) as s:
            s.adapt(it, n)
    t_seq = time.perf_counter() - t0
    out["one_at_a_time_same_precision_solves_per_s"] = len(reqs) / t_seq
    out["speedup_vs_one_at_a_time_same_precision"] = sat["solves_per_s"] * t_seq / len(reqs)
    sub = list(range(0, len(reqs), fp64_every))
    subreqs = [reqs[i] for i in sub]
    got = _serve(G, subreqs, None, budget, slots)
    ssub = _latency_stats(got)
    byidx = {c["tag"]: c for c in got}
    dz = []
    for j, i in enumerate(sub):
        k, p, it, n = reqs[i]
        with G.ILE(p, precision=_precision(G, k), max_samples=n, n_bins=64, seed=1 + j) as s:
            r = s.adapt(it, n)
            assert r["lnZ"] == byidx[j]["lnZ"], (r["lnZ"], byidx[j]["lnZ"])   # alone == served
            dz.append(_lnz_last_vs_fp64(G, s, p, n, r["lnZ_iter"][-1]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j, i in enumerate(sub):
        k, p, it, n = reqs[i]
        with G.ILE(p, precision=G.RIFT_FP64, max_samples=n, n_bins=64, seed=1 + j) as s:
            s.adapt(it, n)
    t64 = time.perf_counter() - t0
    out["fp64_subset"] = {
        "requests": len(sub), "which": f"every {fp64_every}th request of the stream",
        "mix": {k: int(sum(reqs[i][0] == k for i in sub)) for k in ("plain", "batched", "large", "high_snr")},
        "served_solves_per_s": ssub["solves_per_s"], "fp64_one_at_a_time_solves_per_s": len(sub) / t64,
        "speedup_vs_fp64_one_at_a_time": ssub["solves_per_s"] * t64 / len(sub),
        "served_p50_ms": ssub["p50_ms"], "served_p99_ms": ssub["p99_ms"],
        "max_abs_dlnZ_vs_fp64": float(max(dz)), "abs_dlnZ_vs_fp64": [float(x) for x in dz],
        "dlnZ_basis": "each request's last iteration, its own samples re-evaluated by the FP64 GPU path"}
    return out


def run_serving(args, rank, world, local_rank):
    torch, G = _setup(local_rank)
    clk = _clock_monitor(torch, local_rank)
    clk.start()
    sv = measure_serving(torch, G, rank, args.requests, args.quick)
    clocks = clk.stop()
    sat = sv["saturated"]
    value = aggregate_over_ranks(args.requests, sat["span_s"], world)[0]
    out = {
        "metric": "ILE serving solves/s (p50/p99 latency)", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.requests, "warmup": 64, "ms_per_step": 1e3 * sat["span_s"] / args.requests,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"serving stream: {args.requests} requests (40% plain 2-det/2-mode 1e4 samples, 30% "
                               "batched-workload points with 3 iterations, 20% single large 1e6, 10% high-SNR "
                               "2 x 1e6); float32, RIFT_MIXED for the high-SNR points; admission by HBM footprint",
                   "problem_pool": "8 plain + 32 batched + 2 large + 2 high-SNR points, per-request seeds"},
        "serving": sv,
        "e2e": {"value": value, "unit": "solves/s", "note": "requests carry host Q/U/V; the serving loop uploads "
                "them and reads each result back (latency = submit to result)"},
        "gpu_launches": None, "clocks": clocks,
    }
    if rank == 0:
        emit(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--samples", type=int, default=N_SAMPLES, help="samples per step (profiling cases only)")
    ap.add_argument("--quick", action="store_true", help="skip the end-to-end and CPU-baseline legs (profiling)")
    ap.add_argument("--workload", default="single_large", choices=["single_large", "batched", "high_snr", "serving"])
    ap.add_argument("--points", type=int, default=512, help="points of the batched workload")
    ap.add_argument("--requests", type=int, default=2000, help="requests of the serving workload")
    ap.add_argument("--no-workloads", action="store_true",
                    help="single-large line only (no batched and serving blocks)")
    ap.add_argument("--snr", type=float, default=150.0, help="SNR of the high-SNR workload")
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
    run = {"single_large": run_ours, "batched": run_batched, "high_snr": run_high_snr,
           "serving": run_serving}[args.workload]
    try:
        run(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
