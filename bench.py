"""Throughput of the SAA hot path on GB300: scenario-decision evals/s.

One step = one saa_eval of the mean-variance SAA estimate (Eq. 4, Sec. 3.1 of
arXiv 2404.11631) over the whole workload: prologue (y_k = C'w_k), in-kernel
Philox scenario generation, the scenario x decision contraction, the fused
S1/S2 epilogue, the FP64 cross-block reduction and the finalize.  The line
also carries "eval_grad": saa_grad (value and gradient in w) on d = 1024,
N = 2^20 Gaussian scenarios, K = 64, timed the same way, and "fw":
Algorithm 1 (saa_solve) for 200 iterations on d = 1024, N = 2^22 Student-t
scenarios regenerated every iteration, "ragged": 4096 independent
instances in one graph-replayed persistent launch, and "newsvendor": the
Monte Carlo gradient of Sec. 3.2 for 10^6 products x 1000 demand samples,
"covariance_first": the value workload through saa_moments +
saa_eval_moments (value, and value with gradient), and "portfolio_large_d":
value and gradient, and Algorithm 1, for Sec. 4.1's 10^5 independent assets.

Workload (default): d = 128 assets, N = 2^20 scenarios (first half Gaussian,
second half standardised lognormal sigma = 1), K = 256 candidate decisions
x ~ U[0,1]^d, mu ~ U[-1,1]^d, Sigma = LL' + 0.1 I, Philox seed 0.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec P]   (P defaults to f16x3)
       python bench.py --impl reference ...   (the CPU oracle, bounded sample)
Under torchrun each rank evaluates its own independent instance (instance id
= rank): the work is partitioned with no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="batched_d128_N1M_K256_mix", d=128, N=1 << 20, K=256, law=3)
METRIC = "scenario-decision evals/s"


def _peaks():
    """Measured peaks (or the recipe's fallback), plus the SM count of the
    device the bench runs on (the ALU peak's unit count)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            peaks, src = json.load(fh), "measured"
    else:
        peaks, src = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                      "sm_max_mhz": 2070.0}, "fallback"
    import torch
    if torch.cuda.is_available():
        peaks["sm_count"] = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return peaks, src


def _alu_peak(peaks):
    """Lane-operations per second (in T/s): SMs x 128 FP32 lanes x the
    maximum SM clock, the SM count read from the device."""
    return int(peaks["sm_count"]) * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def _alu_peak_source(peaks):
    return f"derived: {int(peaks['sm_count'])} SMs (device) x 128 lanes x {float(peaks.get('sm_max_mhz', 2070.0))} MHz"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([c.strip() for c in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(d, K, law, n_target_s=12.0, N_full=1 << 20, rank=0):
    """Times the CPU oracle on a bounded sample of the workload (scenarios
    N' < N, all K decisions); returns (evals/s, sample description, cores)."""
    import oracle
    from paper_2404_11631_gb300 import inputs
    inst = inputs.instance(d, 0)
    X = inputs.decisions(K, d, 0)
    n = 1 << 12
    while True:
        prob = oracle.make_problem(d, n, inst.mu, inst.chol, law=law, seed=0, instance=rank)
        t0 = time.perf_counter()
        oracle.saa(prob, 32, X)
        dt = time.perf_counter() - t0
        if dt >= n_target_s / 4 or n * 2 > N_full:
            break
        n *= 2
    if dt < n_target_s and n * 2 <= N_full:
        scale = max(1, int(n_target_s / max(dt, 1e-3)))
        n2 = min(N_full, n * min(scale, 8))
        prob = oracle.make_problem(d, n2, inst.mu, inst.chol, law=law, seed=0, instance=rank)
        t0 = time.perf_counter()
        oracle.saa(prob, 32, X)
        dt = time.perf_counter() - t0
        n = n2
    return n * K / dt, dt, n, oracle.max_threads()


# Per-normal work of the scenario generator (the roofline's per-unit figure):
# thread-instructions per normal of the generator-only kernel
# (saa_generate_moments, FP32 mode, d = 128), counted by ncu
# (smsp__thread_inst_executed.sum / normals): 46.45 for a Gaussian normal and
# 61.70 for a standardised lognormal one, with the LOG quotient and the
# Box-Muller root formed by Markstein's corrections (57.15 and 72.65 with the
# IEEE divide and square-root sequences).  That kernel adds one add and one
# fma per normal to the draw.
GEN_INST_GAUSS = 46.45
GEN_INST_LOGN = 61.70 - 46.45
# The stricter count from the generator's specification, each IEEE
# add/sub/mul/fma/div/sqrt, integer op, fused 3-input xor or 32x32->64
# multiply being one operation: Philox4x32-10 10, uniforms 3, log 10.5,
# radius 1, sin/cos 12.5, products 1 -> 38 per Gaussian normal, +18 lognormal.
GEN_OPS_GAUSS = 38.0
GEN_OPS_LOGN = 18.0
# The method's own work per scenario-decision pair beyond the contraction:
# the S1 and S2 sums (Eq. 5 and the variance of Eq. 4).
PAIR_OPS = 2.0
# What the tensor-core kernels issue on top of the method's work (reported
# as issued_frac, not in frac): the hi/lo operand split and the m~ sum per
# normal, and per pair D1 + D2, square, reduce.
SPLIT_OPS = 4.0
EPI_OPS_TC = 3.0
EPI_OPS_SIMT = 2.0    # per pair: S1 and S2 updates (the contraction adds d FMAs)


def _gen_per_normal(law, measured=True):
    g, l = (GEN_INST_GAUSS, GEN_INST_LOGN) if measured else (GEN_OPS_GAUSS, GEN_OPS_LOGN)
    return g + (0.5 * l if law == 3 else l if law == 1 else 0.0)


def roofline(prec, d, N, K, law, kern_s, peaks, peak_src):
    """Roofline of the dominant (sample) kernel.  Every path here is bound by
    ALU issue (the in-kernel generator), except FP64 which is bound by the
    FP64 pipe; the tensor-core paths also report their tensor-pipe use.
    frac counts the method's work only: the generator-only kernel's measured
    instructions per normal, plus S1 and S2 per scenario-decision pair (the
    contraction itself runs on the tensor pipe; on CUDA cores its d FMAs per
    pair are counted too).  issued_frac adds what the tensor-core kernel
    issues on top (hi/lo split, m~ and the D1 + D2 epilogue);
    frac_spec_count uses the generator's specification count per normal."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = int(peaks["sm_count"])
    normals = float(N) * d
    gen = _gen_per_normal(law)
    gen_spec = _gen_per_normal(law, measured=False)
    if prec == "fp64":
        flops = 2.0 * N * d * K
        peak = sms * 2 * 2 * mhz * 1e6 / 1e12
        return {"bound": "alu", "achieved": flops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / kern_s / 1e12 / peak, "traffic": None, "kernel_ms": kern_s * 1e3,
                "peak_source": f"derived: {sms} SMs (device) x 2 FP64 FMA/clk x 2 x {mhz} MHz",
                "note": "FP64 contraction flops 2NdK; the FP64 generator work is extra"}
    tc = prec in ("bf16x3", "f16x3")

    def count(g):
        if tc:
            return normals * g + float(N) * K * PAIR_OPS
        return normals * g + float(N) * K * (d + PAIR_OPS)
    ops, ops_spec = count(gen), count(gen_spec)
    peak = _alu_peak(peaks)
    r = {"bound": "alu", "achieved": ops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
         "frac": ops / kern_s / 1e12 / peak, "traffic": None, "kernel_ms": kern_s * 1e3,
         "frac_spec_count": ops_spec / kern_s / 1e12 / peak,
         "peak_source": _alu_peak_source(peaks),
         "note": "lane-operations of the method: generator-only kernel's instructions per normal (ncu) + "
                 "S1, S2 per pair" + ("" if tc else " + the d FMAs of the CUDA-core contraction")}
    if tc:
        issued = normals * (gen + SPLIT_OPS) + float(N) * K * EPI_OPS_TC
        r["issued_frac"] = issued / kern_s / 1e12 / peak
        # ncu dram__bytes_read.sum + dram__bytes_write.sum of the tensor kernel
        # (F16, d = 128, K = 256, captured at N = 2^17): the per-launch operand
        # image and workspace reads, independent of N
        if prec == "f16x3" and d == 128 and K == 256:
            r["traffic"] = 194816
        tflops = 3 * 2.0 * N * d * K / kern_s / 1e12
        r["tensor"] = {"achieved": tflops, "peak": float(peaks["bf16_tflops"]), "unit": "TFLOP/s",
                       "frac": tflops / float(peaks["bf16_tflops"]), "peak_source": f"{peak_src} bf16 dense (burst)"}
    return r


GRAD_WORKLOAD = dict(name="grad_d1024_N1M_K64_gauss", d=1024, N=1 << 20, K=64, law=0)
EPI_OPS_TC_GRAD = 8.0   # per pair: chunk fold, D1 + D2, square + reduce, W hi/lo split
# DRAM bytes per launch of the value-and-gradient kernel, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on a small case, scaled to
# the launch's N where the traffic grows with the number of tiles; absent
# until taken on the current kernel.
GRAD_TRAFFIC = {("f16x3", 1024, 64): lambda n: 409600.0}   # N = 2^17 capture; image and partials, not N


def grad_roofline(prec, d, N, K, law, kern_s, peaks):
    """ALU roofline of the value-and-gradient kernel: the method draws each
    normal once and forms S1, S2 per pair (the forward and adjoint
    contractions run on the tensor pipe; on CUDA cores their 2d FMAs per pair
    are counted too)."""
    tc = prec in ("bf16x3", "f16x3")

    def count(g):
        if tc:
            return float(N) * d * g + float(N) * K * PAIR_OPS
        return float(N) * d * g + float(N) * K * (2 * d + PAIR_OPS)
    ops, ops_spec = count(_gen_per_normal(law)), count(_gen_per_normal(law, measured=False))
    peak = _alu_peak(peaks)
    r = {"bound": "alu", "achieved": ops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
         "frac": ops / kern_s / 1e12 / peak, "traffic": GRAD_TRAFFIC.get((prec, d, K), lambda n: None)(N),
         "kernel_ms": kern_s * 1e3, "frac_spec_count": ops_spec / kern_s / 1e12 / peak,
         "peak_source": _alu_peak_source(peaks),
         "note": "lane-operations of the method: one draw per normal + S1, S2 per pair"}
    if tc:
        issued = float(N) * d * (_gen_per_normal(law) + SPLIT_OPS) + float(N) * K * EPI_OPS_TC_GRAD
        r["issued_frac"] = issued / kern_s / 1e12 / peak
        tflops = 2 * 3 * 2.0 * N * d * K / kern_s / 1e12
        r["tensor"] = {"achieved": tflops, "peak": float(peaks["bf16_tflops"]), "unit": "TFLOP/s",
                       "frac": tflops / float(peaks["bf16_tflops"])}
    return r


def run_grad(args, dev, world, rank, flush, stream):
    """Value and gradient (saa_grad) on the adjoint workload: d = 1024,
    N = 2^20 Gaussian scenarios, K = 64 decisions; L2 flushed between steps."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    d, N, K, law = GRAD_WORKLOAD["d"], GRAD_WORKLOAD["N"], GRAD_WORKLOAD["K"], GRAD_WORKLOAD["law"]
    prec = args.prec
    inst = inputs.instance(d, 0)
    prob = saa.Problem(mu=torch.tensor(inst.mu, device=dev), chol=torch.tensor(inst.chol, device=dev), N=N,
                       law=law, seed=0, instance=rank)
    X = torch.tensor(inputs.decisions(K, d, 0), device=dev)
    ws = torch.empty(saa.workspace_size(prob, K, prec, 1), dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 20))
    for _ in range(3):
        saa.saa_grad(prob, X, prec, ws=ws)
    torch.cuda.synchronize(dev)
    saa.saa_profile_enable(True, dev.index)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        saa.saa_grad(prob, X, prec, ws=ws)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    main_ms, main_n, launched = saa.saa_profile_read(dev.index)
    saa.saa_profile_enable(False, dev.index)
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    peaks, _ = _peaks()
    kern_s = main_ms / 1e3 / max(1, main_n)
    # values only on the same workload (saa_eval: the cluster kernel without
    # its adjoint above d = 256 at the tensor precisions)
    vws = torch.empty(saa.workspace_size(prob, K, prec, 0), dtype=torch.uint8, device=dev)
    for _ in range(3):
        saa.saa_eval(prob, X, prec, ws=vws)
    torch.cuda.synchronize(dev)
    saa.saa_profile_enable(True, dev.index)
    vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        vev[i][0].record(stream)
        saa.saa_eval(prob, X, prec, ws=vws)
        vev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    vms, vn, _ = saa.saa_profile_read(dev.index)
    saa.saa_profile_enable(False, dev.index)
    vtotal = sum(a.elapsed_time(b) for a, b in vev) / 1e3
    vkern = vms / 1e3 / max(1, vn)
    vroof = {"bound": "alu", "frac": float(N) * d * _gen_per_normal(law) / vkern / 1e12 / _alu_peak(peaks),
             "kernel_ms": vkern * 1e3,
             "note": "one draw per normal (generator-only kernel's instructions per normal) over the ALU peak"}
    return {"metric": "scenario-decision evals/s with gradient", "value": world * N * K * steps / total_s,
            "unit": "evals/s", "ms_per_step": 1e3 * total_s / steps, "steps": steps,
            "config": {"workload": GRAD_WORKLOAD["name"], "d": d, "N": N, "K": K, "law": "Gaussian",
                       "prec": prec, "l2": "flushed between timed steps"},
            "gpu_launches": int(launched), "roofline": grad_roofline(prec, d, N, K, law, kern_s, peaks),
            "value_only": {"value": world * N * K * steps / vtotal, "unit": "evals/s",
                           "ms_per_step": 1e3 * vtotal / steps, "roofline": vroof}}


FW_WORKLOAD = dict(name="fw_d1024_N4M_t4_T200", d=1024, N=1 << 22, law=2, nu=4, T=200, M=1)


def run_fw(args, dev, world, rank):
    """Algorithm 1 (saa_solve): d = 1024, N = 2^22 Student-t (nu = 4)
    scenarios regenerated in-kernel every iteration (M = 1), T = 200
    iterations from w0 = (0.5/d) 1, each iteration one replay of a captured
    CUDA graph.  Reported per iteration."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    d, N, T = FW_WORKLOAD["d"], FW_WORKLOAD["N"], FW_WORKLOAD["T"]
    prec = "fp32"
    inst = inputs.instance(d, 0)
    prob = saa.Problem(mu=torch.tensor(inst.mu, device=dev), chol=torch.tensor(inst.chol, device=dev), N=N,
                       law=FW_WORKLOAD["law"], nu=FW_WORKLOAD["nu"], seed=0, instance=rank)
    w0 = torch.tensor(inputs.fw_start(d), device=dev)
    ws = torch.empty(saa.workspace_size(prob, 1, prec, 2), dtype=torch.uint8, device=dev)
    saa.saa_solve(prob, w0, T=2, M=FW_WORKLOAD["M"], prec=prec, ws=ws)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = saa.saa_solve(prob, w0, T=T, M=FW_WORKLOAD["M"], prec=prec, ws=ws)
    e1.record()
    torch.cuda.synchronize(dev)
    saa.saa_ctx_sync(dev.index)
    ms = e0.elapsed_time(e1) / T
    gap = out["gap_trace"].cpu().numpy()
    f = out["f_trace"].cpu().numpy()
    # the same run with the sample size growing per epoch (M = 1): N_k from
    # N / 64 doubling in seven equal stretches up to N; one graph per stretch
    sched = [max(2, N >> (6 - min(6, (7 * k) // T))) for k in range(T)]
    ws_a = torch.empty(max(ws.numel(), 1), dtype=torch.uint8, device=dev)
    saa.saa_solve_adaptive(prob, w0, sched[:2], M=FW_WORKLOAD["M"], prec=prec, ws=ws_a)
    torch.cuda.synchronize(dev)
    e0.record()
    ad = saa.saa_solve_adaptive(prob, w0, sched, M=FW_WORKLOAD["M"], prec=prec, ws=ws_a)
    e1.record()
    torch.cuda.synchronize(dev)
    saa.saa_ctx_sync(dev.index)
    ms_a = e0.elapsed_time(e1)
    normals_a = float(sum(sched)) * d
    adaptive = {"ms_total": ms_a, "normals_per_s": normals_a / (ms_a / 1e3), "iterations": T,
                "N_first_last": [sched[0], sched[-1]], "graphs": len(set(sched)),
                "note": "time includes capturing one graph per distinct N_k",
                "f_last": float(ad["f_trace"].cpu().numpy()[-1])}
    # ALU roofline per iteration: the generator-only kernel's count per
    # (Gaussian) normal, the t law's chi-square draws and one multiply-add
    # each for the forward dot product and the adjoint per normal
    peaks, _ = _peaks()
    peak = _alu_peak(peaks)
    ops = float(N) * d * (GEN_INST_GAUSS + 2.0)
    achieved = ops / (ms / 1e3) / 1e12
    return {"metric": "Frank-Wolfe iterations/s (Algorithm 1)", "value": world * 1e3 / ms, "unit": "iterations/s",
            "ms_per_iteration": ms, "normals_per_s": N * d / (ms / 1e3), "iterations": T,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "note": "lane-ops per iteration: generator per normal + 2 fma per normal; whole iteration"},
            "config": {"workload": FW_WORKLOAD["name"], "d": d, "N": N, "law": "Student-t nu=4", "M": 1,
                       "prec": prec, "graph": "one captured iteration replayed T times"},
            "f_first_last": [float(f[0]), float(f[-1])], "gap_last": float(gap[-1]), "adaptive_N": adaptive}


def run_ragged(args, dev, world, rank, flush, stream):
    """The ragged batch: 4096 independent Gaussian instances, d ~ U{8..512},
    N = floor(10^U[3,5]), K ~ U{1..16}, each with its own Sigma; FP32; one
    saa_batch (autotuned tile shape, the whole launch sequence captured in a
    CUDA graph) replayed per step.  evals = sum_b N_b K_b per replay."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    rb = inputs.ragged_batch(args.ragged_B, seed=rank)
    probs, Xs = [], []
    for b in range(len(rb.d)):
        inst = rb.instances[b]
        probs.append(saa.Problem(mu=torch.tensor(inst.mu, device=dev), chol=torch.tensor(inst.chol, device=dev),
                                 N=int(rb.N[b]), law=0, seed=int(rb.seeds[b]), instance=b))
        Xs.append(torch.tensor(rb.X[b], device=dev))
    batch = saa.Batch(probs, Xs, "fp32", want_pbar=False, want_var=False)
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize(dev)
    steps = max(3, min(args.steps, 10))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        batch.run()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    saa.saa_ctx_sync(dev.index)
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    evals = float(np.sum(rb.N.astype(np.float64) * rb.K))
    normals = float(np.sum(rb.N.astype(np.float64) * rb.d))
    batch.close()
    # ALU roofline: the generator-only kernel's count per (Gaussian) normal
    # plus the fused kernel's K_b multiply-adds per normal (dot products
    # formed while drawing), over the whole replay
    peaks, _ = _peaks()
    peak = _alu_peak(peaks)
    ops = normals * GEN_INST_GAUSS + float(np.sum(rb.N.astype(np.float64) * rb.d * rb.K))
    achieved = ops * steps / total_s / 1e12
    return {"metric": "scenario-decision evals/s (ragged batch)", "value": world * evals * steps / total_s,
            "unit": "evals/s", "ms_per_step": 1e3 * total_s / steps, "steps": steps,
            "normals_per_s": normals * steps / total_s,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "note": "lane-ops: generator per normal + K_b fma per normal; whole replay time"},
            "config": {"workload": f"ragged_{len(rb.d)}_gauss", "instances": len(rb.d), "d": "U{8..512}",
                       "N": "floor(10^U[3,5])", "K": "U{1..16}", "prec": "fp32", "sum_NK": evals, "sum_Nd": normals,
                       "graph": "autotuned tile shape, launch sequence captured once and replayed"}}


NV_WORKLOAD = dict(name="newsvendor_n1M_S1000_K1", n=1_000_000, S=1000, K=1)


LD_WORKLOAD = dict(name="portfolio_diag_d100000_N65536", d=100_000, N=1 << 16, M=50, T=20, d_small=5000, M_small=25,
                   T_small=1500)


def run_large_d(args, dev, world, rank, flush, stream):
    """Sec. 4.1's portfolio at its largest size: d = 10^5 independent assets
    (mu ~ U(-1,1), sigma ~ U(0, 0.025), Sigma = diag(sigma^2), no dense
    factor), N = 2^16 Gaussian samples, FP32.  One step is saa_grad at one
    decision (value and gradient); the unit is one (sample, asset) normal.
    Algorithm 1 is timed on the same problem (M = 50, as Sec. 4.1 uses at
    this size; T = 20 iterations, per-iteration time) and at d = 5000 for the
    paper's full 1500 iterations (M = 25)."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    d, N = LD_WORKLOAD["d"], LD_WORKLOAD["N"]

    def problem(dd):
        mu, sd = inputs.paper_assets(dd, 0)
        return saa.Problem(mu=torch.tensor(mu, device=dev), chol=None, sd=torch.tensor(sd, device=dev), N=N,
                           seed=0, instance=rank)
    prob = problem(d)
    X = torch.tensor(inputs.fw_start(d)[None], device=dev)
    ws = torch.empty(saa.workspace_size(prob, 1, "fp32", 1), dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 10))
    res_k = {}
    for name, fn in (("value", lambda: saa.saa_eval(prob, X, "fp32", ws=ws)),
                     ("grad", lambda: saa.saa_grad(prob, X, "fp32", ws=ws))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        saa.saa_profile_enable(True, dev.index)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        main_ms, main_n, launched = saa.saa_profile_read(dev.index)
        saa.saa_profile_enable(False, dev.index)
        saa.saa_ctx_sync(dev.index)
        res_k[name] = (sum(a.elapsed_time(b) for a, b in ev) / 1e3 / steps, main_ms / 1e3 / max(1, main_n),
                       launched / steps)
    # the same call drawing the samples twice (no sample store), for comparison
    saa.saa_ctx_set_sample_store(0, dev.index)
    ws_r = torch.empty(saa.workspace_size(prob, 1, "fp32", 1), dtype=torch.uint8, device=dev)
    saa.saa_grad(prob, X, "fp32", ws=ws_r)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        saa.saa_grad(prob, X, "fp32", ws=ws_r)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    saa.saa_ctx_set_sample_store(1 << 35, dev.index)
    redraw_ms = e0.elapsed_time(e1) / 3
    del ws_r
    step_s, kern_s, launches = res_k["grad"]
    fwd_s = res_k["value"][1]
    normals = float(N) * d
    peaks, _ = _peaks()
    peak = _alu_peak(peaks)
    # lane-ops: one draw per normal and a multiply-add in each pass (the
    # adjoint also its m~ sum); the adjoint reads the stored normals back
    ops_fwd = normals * (GEN_INST_GAUSS + 1.0)
    ops = normals * (GEN_INST_GAUSS + 3.0)
    store_bytes = float(N) * ((d + 3) // 4 * 4) * 4
    fw = {}
    for tag, dd, M, T in (("d100000", d, LD_WORKLOAD["M"], LD_WORKLOAD["T"]),
                          ("d5000", LD_WORKLOAD["d_small"], LD_WORKLOAD["M_small"], LD_WORKLOAD["T_small"])):
        pr = problem(dd)
        w0 = torch.tensor(inputs.fw_start(dd), device=dev)
        wsf = torch.empty(saa.workspace_size(pr, 1, "fp32", 2), dtype=torch.uint8, device=dev)
        saa.saa_solve(pr, w0, T=2, M=M, ws=wsf)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = saa.saa_solve(pr, w0, T=T, M=M, ws=wsf)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        saa.saa_ctx_sync(dev.index)
        ms = e0.elapsed_time(e1)
        fw[tag] = {"d": dd, "N": N, "M": M, "T": T, "ms_total": ms, "ms_per_iteration": ms / T,
                   "s_for_1500_iterations": 1.5 * ms / T, "f_first_last": [float(out["f_trace"][0]),
                                                                          float(out["f_trace"][-1])],
                   "gap_last": float(out["gap_trace"][-1])}
        try:   # Table 2's accuracy measure against the exact optimum (host arithmetic only)
            from paper_2404_11631_gb300.reporting import diag_optimum, rse
            mu_np, sd_np = inputs.paper_assets(dd, 0)
            _, f_star = diag_optimum(mu_np, sd_np)
            ft = out["f_trace"].cpu().numpy()
            w_fin = out["w"].cpu().numpy()
            fw[tag]["f_star"] = f_star
            fw[tag]["f_exact_last"] = float(0.5 * np.sum(sd_np ** 2 * w_fin ** 2) - mu_np @ w_fin)
            vals = {str(t): float(rse(ft[t - 1], f_star)) for t in (50, 100, 500, 1000) if t <= T}
            fw[tag]["rse_pct"] = {t: (v if np.isfinite(v) else None) for t, v in vals.items()}
        except Exception as exc:   # a reporting extra never stops the bench
            fw[tag]["rse_error"] = repr(exc)
    # Sec. 4.1's asset sizes: Algorithm 1 per iteration at each (T = 20 timed
    # iterations after 2; M = 25, 50 at 10^5 as the paper samples)
    sweep = {}
    if not args.ld_d:
        for dd in (500, 5000, 10_000, 50_000, 100_000):
            pr = problem(dd)
            w0 = torch.tensor(inputs.fw_start(dd), device=dev)
            M = 50 if dd == 100_000 else 25
            wsf = torch.empty(saa.workspace_size(pr, 1, "fp32", 2), dtype=torch.uint8, device=dev)
            saa.saa_solve(pr, w0, T=2, M=M, ws=wsf)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            saa.saa_solve(pr, w0, T=20, M=M, ws=wsf)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            saa.saa_ctx_sync(dev.index)
            sweep[str(dd)] = {"ms_per_iteration": e0.elapsed_time(e1) / 20,
                              "s_for_1500_iterations": 1.5 * e0.elapsed_time(e1) / 20, "M": M}
            del wsf
    res = {"metric": "normals/s (portfolio value and gradient, diagonal Sigma)", "value": world * normals / step_s,
           "unit": "normals/s", "ms_per_step": 1e3 * step_s, "steps": steps, "kernels_ms": 1e3 * kern_s,
           "forward_kernel_ms": 1e3 * fwd_s, "value_only_ms_per_step": 1e3 * res_k["value"][0],
           "adjoint_kernel_ms": 1e3 * (kern_s - fwd_s), "redraw_ms_per_step": redraw_ms,
           "gpu_launches_per_step": launches,
           "roofline": {"bound": "alu", "achieved": ops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": ops / kern_s / 1e12 / peak, "forward_frac": ops_fwd / fwd_s / 1e12 / peak,
                        "adjoint_hbm_frac": store_bytes / max(1e-9, kern_s - fwd_s) / 1e9 / peaks["hbm_gbs"],
                        "note": "lane-ops: one draw per normal + 3 per normal; forward + adjoint.  The forward "
                                "writes the FP32 normals, the adjoint reads them (adjoint_hbm_frac: that read "
                                "against the measured HBM copy bandwidth)"},
           "fw": fw, "fw_size_sweep_N65536": sweep,
           "config": {"workload": LD_WORKLOAD["name"], "d": d, "N": N, "K": 1, "law": "Gaussian",
                      "sigma": "diag, U(0, 0.025)", "prec": "fp32", "l2": "flushed between timed steps"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        mu, sd = inputs.paper_assets(d, 0)
        n = 16384
        op = oracle.make_problem(d, n, mu, None, seed=0, instance=rank, sd=sd)
        t0 = time.perf_counter()
        oracle.saa(op, 32, inputs.fw_start(d), grad=True)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": float(n) * d / dt, "unit": "normals/s", "cores": oracle.max_threads(),
                               "kind": "oracle", "sample": f"{n} of {N} samples x all {d} assets, value and gradient,"
                                                           f" {dt:.1f} s"}
    return res


LG_WORKLOAD = dict(name="logistic_n5000_N150000", n=5000, N=150_000, b=50, bH=600)


def run_logistic(args, dev, world, rank, flush, stream):
    """The binary-classification task (Sec. 3.3) at Sec. 4.1's largest size:
    n = 5000 binary features, N = 30 n = 150000 points (10 % label noise).
    One step is the full-data objective, gradient and Hessian product at one
    parameter vector; the unit is one (point, feature) pair.  The SQN-sized
    calls (gradient on b = 50 points, Hessian product on b_H = 600) are timed
    too: they are launch-bound."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    n, N = LG_WORKLOAD["n"], LG_WORKLOAD["N"]
    wstar = torch.tensor(inputs.logistic_weights(n, 0), device=dev)
    data = saa.saa_logistic_generate(n, N, wstar, seed=0, instance=rank)
    rng = np.random.default_rng(0)
    W = torch.tensor(0.02 * rng.normal(size=(1, n)), device=dev)
    V = torch.tensor(rng.normal(size=(1, n)), device=dev)
    out = saa.saa_logistic_eval(data["X"], data["z"], n, W, V)
    ws = out["ws"]
    for _ in range(3):
        saa.saa_logistic_eval(data["X"], data["z"], n, W, V, ws=ws)
    torch.cuda.synchronize(dev)
    saa.saa_profile_enable(True, dev.index)
    steps = max(3, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        saa.saa_logistic_eval(data["X"], data["z"], n, W, V, ws=ws)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    main_ms, main_n, launched = saa.saa_profile_read(dev.index)
    saa.saa_profile_enable(False, dev.index)
    saa.saa_ctx_sync(dev.index)
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    kern_s = main_ms / 1e3 / max(1, main_n)
    pairs = float(N) * n
    # masked adds per (point, feature): omega and v in the forward pass,
    # gradient and Hessian product in the adjoint
    ops = 4.0 * pairs
    peaks, _ = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = _alu_peak(peaks)
    # SQN-sized calls: mini-batch gradient (b = 50) and Hessian product (b_H = 600)
    mini = {}
    for name, b, want_v in (("grad_b50", LG_WORKLOAD["b"], False), ("hvp_b600", LG_WORKLOAD["bH"], True)):
        idx = torch.tensor(rng.integers(0, N, size=b), dtype=torch.int64, device=dev)
        for _ in range(3):
            saa.saa_logistic_eval(data["X"], data["z"], n, W, V if want_v else None, idx=idx)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            saa.saa_logistic_eval(data["X"], data["z"], n, W, V if want_v else None, idx=idx)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        mini[name] = {"us_per_call": 1e3 * e0.elapsed_time(e1) / 20}
    res = {"metric": "logistic point-feature pairs/s (F, gradient, Hessian product)",
           "value": world * pairs * steps / total_s, "unit": "pairs/s", "ms_per_step": 1e3 * total_s / steps,
           "kernels_ms": kern_s * 1e3, "gpu_launches_per_step": launched / steps,
           "roofline": {"bound": "alu", "achieved": ops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": ops / kern_s / 1e12 / peak,
                        "note": "lane-ops: 4 masked adds per (point, feature) pair; forward + adjoint kernels"},
           "mini_batch": mini,
           "config": {"workload": LG_WORKLOAD["name"], "n": n, "N": N, "K": 1, "features": "bits, Bernoulli(1/2)",
                      "labels": "integer linear rule, 10% flips", "data_bytes": int(data["X"].numel()) * 4}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        op = oracle.make_logistic(n, N, inputs.logistic_weights(n, 0), seed=0, instance=rank)
        t0 = time.perf_counter()
        oracle.logistic_eval(op, W.cpu().numpy(), V=V.cpu().numpy())
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": float(N) * n / dt, "unit": "pairs/s", "cores": oracle.max_threads(),
                               "kind": "oracle", "sample": f"all {N} points x {n} features, {dt:.1f} s"}
    return res


def run_newsvendor(args, dev, world, rank, flush, stream):
    """The newsvendor's Monte Carlo gradient (Sec. 3.2): n = 10^6 products
    (the largest inventory of Sec. 4.1), S = 1000 normal demand samples per
    product, mu ~ U(20, 50), sigma ~ U(10, 20), one decision vector.  The
    unit is one demand sample of one product (one normal + its compare)."""
    import torch
    from paper_2404_11631_gb300 import saa
    n, S, K = NV_WORKLOAD["n"], NV_WORKLOAD["S"], NV_WORKLOAD["K"]
    rng = np.random.default_rng([n, S, 11])
    arrs = dict(mu=rng.uniform(20.0, 50.0, n), sigma=rng.uniform(10.0, 20.0, n), k=rng.uniform(0.5, 2.0, n),
                h=rng.uniform(0.1, 1.0, n), v=rng.uniform(1.0, 4.0, n))
    prob = saa.Newsvendor(**{a: torch.tensor(x, device=dev) for a, x in arrs.items()}, S=S, seed=0, instance=rank)
    X = torch.tensor(arrs["mu"] + arrs["sigma"] * np.random.default_rng(1).uniform(-3.0, 3.0, (K, n)), device=dev)
    for _ in range(3):
        saa.saa_newsvendor_grad(prob, X)
    torch.cuda.synchronize(dev)
    steps = max(3, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        saa.saa_newsvendor_grad(prob, X)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    saa.saa_ctx_sync(dev.index)
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    samples = float(n) * S
    peaks, _ = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = _alu_peak(peaks)
    ops = samples * (GEN_INST_GAUSS + 2.0 * K)   # generator per normal + compare and count per decision
    # Sec. 4.1's inventory sizes, 10^2 .. 10^6 products (same S): one gradient each
    sweep = {}
    for nn in (100, 1000, 10_000, 100_000, 1_000_000):
        p2 = saa.Newsvendor(**{a: torch.tensor(x[:nn], device=dev) for a, x in arrs.items()}, S=S, seed=0,
                            instance=rank)
        X2 = X[:, :nn].contiguous()
        for _ in range(2):
            saa.saa_newsvendor_grad(p2, X2)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            saa.saa_newsvendor_grad(p2, X2)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sweep[str(nn)] = {"ms_per_gradient": e0.elapsed_time(e1) / 10}
    saa.saa_ctx_sync(dev.index)
    return {"metric": "demand samples/s (newsvendor MC gradient)", "value": world * samples * steps / total_s,
            "unit": "samples/s", "ms_per_step": 1e3 * total_s / steps, "steps": steps,
            "config": {"workload": NV_WORKLOAD["name"], "n": n, "S": S, "K": K, "prec": "fp32 normals, exact counts",
                       "l2": "flushed between timed steps"},
            "roofline": {"bound": "alu", "achieved": ops * steps / total_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": ops * steps / total_s / 1e12 / peak,
                         "note": "generator-only kernel's instructions per normal + 2 per sample and decision"},
            "size_sweep": sweep}


def run_covariance(args, dev, world, rank, flush, stream):
    """Covariance-first form on the value workload (d = 128, N = 2^20 half
    Gaussian / half lognormal, K = 256): one step is saa_moments (the sums
    M = sum_i a_i a_i', mt = sum_i a_i on the tensor cores) plus
    saa_eval_moments for all K decisions, value only and value + gradient."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    d, N, K, law = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["K"], WORKLOAD["law"]
    prec = args.prec if args.prec in ("f16x3", "bf16x3") else "f16x3"
    inst = inputs.instance(d, 0)
    prob = saa.Problem(mu=torch.tensor(inst.mu, device=dev), chol=torch.tensor(inst.chol, device=dev), N=N, law=law,
                       seed=0, instance=rank)
    X = torch.tensor(inputs.decisions(K, d, 0), device=dev)
    mws = torch.empty(1 << 26, dtype=torch.uint8, device=dev)
    ews = torch.empty(1 << 24, dtype=torch.uint8, device=dev)
    res = {}
    for mode, grad in (("value", False), ("value_and_gradient", True)):
        def step():
            mom = saa.saa_moments(prob, prec, ws=mws)
            return saa.saa_eval_moments(prob, X, mom, want_grad=grad, ws=ews)
        for _ in range(3):
            step()
        torch.cuda.synchronize(dev)
        saa.saa_profile_enable(True, dev.index)
        steps = max(3, min(args.steps, 50))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        main_ms, main_n, launched = saa.saa_profile_read(dev.index)
        saa.saa_profile_enable(False, dev.index)
        total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        kern_s = main_ms / 1e3 / max(1, main_n)
        peaks, _ = _peaks()
        mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = _alu_peak(peaks)
        ops = float(N) * d * _gen_per_normal(law)
        issued = float(N) * d * (_gen_per_normal(law) + SPLIT_OPS)
        res[mode] = {"value": world * N * K * steps / total_s, "unit": "evals/s", "ms_per_step": 1e3 * total_s / steps,
                     "gram_kernel_ms": kern_s * 1e3, "gpu_launches_per_step": launched / steps,
                     "roofline": {"bound": "alu", "achieved": ops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                                  "frac": ops / kern_s / 1e12 / peak, "issued_frac": issued / kern_s / 1e12 / peak,
                                  "note": "Gram kernel: generator-only kernel's instructions per normal "
                                          "(issued_frac adds the hi/lo split)"}}
    # blocked form at d = 1024 (M in 128 x 128 blocks, each block's CTAs
    # drawing its two dimension slices): value and gradient for K = 64
    db, Kb = 1024, 64
    instb = inputs.instance(db, 0)
    probb = saa.Problem(mu=torch.tensor(instb.mu, device=dev), chol=torch.tensor(instb.chol, device=dev), N=N,
                        law=law, seed=0, instance=rank)
    Xb = torch.tensor(inputs.decisions(Kb, db, 0), device=dev)
    ewsb = torch.empty(1 << 26, dtype=torch.uint8, device=dev)

    def stepb():
        mom = saa.saa_moments(probb, prec, ws=mws)
        return saa.saa_eval_moments(probb, Xb, mom, want_grad=True, ws=ewsb)
    stepb()
    torch.cuda.synchronize(dev)
    saa.saa_profile_enable(True, dev.index)
    nb_steps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nb_steps):
        stepb()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    main_ms, main_n, _ = saa.saa_profile_read(dev.index)
    saa.saa_profile_enable(False, dev.index)
    saa.saa_ctx_sync(dev.index)
    kern_s = main_ms / 1e3 / max(1, main_n)
    nslices = (db + 127) // 128
    ops = float(N) * db * _gen_per_normal(law)
    res["blocked_d1024_K64_value_and_gradient"] = {
        "ms_per_step": e0.elapsed_time(e1) / nb_steps, "gram_kernel_ms": kern_s * 1e3,
        "value": world * N * Kb / (e0.elapsed_time(e1) / nb_steps / 1e3), "unit": "evals/s",
        "roofline": {"bound": "alu", "frac": ops / kern_s / 1e12 / _alu_peak(_peaks()[0]),
                     "issued_frac": nslices * ops / kern_s / 1e12 / _alu_peak(_peaks()[0]),
                     "note": f"frac counts one draw per normal; every normal is drawn {nslices} times "
                             "(once per block that needs its slice)"}}
    return {"metric": "scenario-decision evals/s (covariance-first)", "config": {
        "workload": WORKLOAD["name"], "d": d, "N": N, "K": K, "prec": prec,
        "method": "M = sum a a' once on tcgen05, then S2 = y'My, G = My per decision in FP64"}, **res}


# DRAM bytes (read + write) per launch of the streamed kernel on the bench's
# workload (d = 128, N = 2^20, K = 256), from one ncu capture at full size
# (dram__bytes_read.sum + dram__bytes_write.sum): the algorithmic N d 4 =
# 536,870,912 B of samples plus the decision image and the partials.
STREAM_TRAFFIC = {("fp8x", 128, 1 << 20, 256): 537204480.0}


def run_streamed(args, dev, world, rank, flush, stream):
    """Streamed mode on the value workload's shape (d = 128, N = 2^20,
    K = 256): the N samples R_i are materialised once in HBM as FP32 rows
    (by saa_generate, outside the timed region) and every step reads them
    back through TMA into the tensor-core contraction (saa_eval_samples,
    center mu, sigma = sqrt(diag Sigma)).  The 512 MB sample matrix is
    larger than L2, so each step streams it from HBM.  Timed at the FP16
    hi/lo products (the line) and at SAA_FP8X (its "fp8x" entry: four E4M3
    products, counted against the FP8 tensor peak)."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    d, N, K, law = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["K"], WORKLOAD["law"]
    prec = args.prec if args.prec in ("f16x3", "bf16x3") else "f16x3"
    inst = inputs.instance(d, 0)
    prob = saa.Problem(mu=torch.tensor(inst.mu, device=dev), chol=torch.tensor(inst.chol, device=dev), N=N, law=law,
                       seed=0, instance=rank)
    R = saa.saa_generate(prob, 0, N, "fp32", want_xi=True)["xi"]
    X = torch.tensor(inputs.decisions(K, d, 0), device=dev)
    sd = torch.tensor(np.sqrt(np.diag(inst.sigma)), device=dev)
    peaks, src = _peaks()
    hbm_bytes = float(N) * d * 4                 # d FP32 values per scenario, one pass

    def timed(pr, products, tc_peak, tc_src):
        ws = saa.saa_eval_samples(R, X, prob.lam, pr, center=prob.mu, sigma=sd)["ws"]
        for _ in range(3):
            saa.saa_eval_samples(R, X, prob.lam, pr, center=prob.mu, sigma=sd, ws=ws)
        torch.cuda.synchronize(dev)
        saa.saa_profile_enable(True, dev.index)
        steps = max(3, min(args.steps, 50))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            ev[i][0].record(stream)
            out = saa.saa_eval_samples(R, X, prob.lam, pr, center=prob.mu, sigma=sd, ws=ws)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        main_ms, main_n, launched = saa.saa_profile_read(dev.index)
        saa.saa_profile_enable(False, dev.index)
        saa.saa_ctx_sync(dev.index)
        total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        kern_s = main_ms / 1e3 / max(1, main_n)
        tc_flops = products * 2.0 * N * d * K        # the split products, 2 N d K each
        t_hbm = hbm_bytes / (peaks["hbm_gbs"] * 1e9)
        t_tc = tc_flops / (tc_peak * 1e12)
        if t_tc >= t_hbm:
            roof = {"bound": "tensor", "achieved": tc_flops / kern_s / 1e12, "peak": tc_peak,
                    "unit": "TFLOP/s", "frac": tc_flops / kern_s / 1e12 / tc_peak}
        else:
            roof = {"bound": "hbm", "achieved": hbm_bytes / kern_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": hbm_bytes / kern_s / 1e9 / peaks["hbm_gbs"]}
        roof["peak_source"] = {"hbm": src, "tensor": tc_src}
        roof["traffic"] = STREAM_TRAFFIC.get((pr, d, N, K))
        roof["hbm"] = {"achieved_gbs": hbm_bytes / kern_s / 1e9, "frac": hbm_bytes / kern_s / 1e9 / peaks["hbm_gbs"]}
        roof["tensor"] = {"achieved_tflops": tc_flops / kern_s / 1e12, "frac": tc_flops / kern_s / 1e12 / tc_peak,
                          "products": products}
        return {"metric": "scenario-decision evals/s (streamed samples)", "value": world * N * K * steps / total_s,
                "unit": "evals/s", "ms_per_step": 1e3 * total_s / steps, "stream_kernel_ms": kern_s * 1e3,
                "gpu_launches_per_step": launched / steps, "roofline": roof,
                "config": {"workload": "streamed_" + WORKLOAD["name"], "d": d, "N": N, "K": K, "prec": pr,
                           "samples": "FP32 [N, d] in HBM (512 MB > L2), center mu, sigma sqrt(diag Sigma)"}}, out

    res, _ = timed(prec, 3.0, peaks["bf16_tflops"], src)
    # FP8 dense peak: the measured bf16 figure times the nominal FP8 / BF16
    # ratio (4.5 / 2.25 PFLOP/s)
    res["fp8x"], _ = timed("fp8x", 4.0, 2.0 * peaks["bf16_tflops"], src + " x 2 (nominal FP8 / BF16 ratio)")
    del R
    return res


def run_gen(args):
    """The bare generator (saa_generate_moments, FP32 mode) on the value
    workload's d and N, per law: normals/s.  This is the generator-only
    kernel whose ncu instruction count per normal is the roofline's
    per-unit figure."""
    import torch
    from paper_2404_11631_gb300 import inputs, saa
    dev = torch.device("cuda", 0)
    d, N = WORKLOAD["d"], WORKLOAD["N"]
    inst = inputs.instance(d, 0)
    out = {"metric": "generator normals/s", "unit": "normals/s", "config": {"d": d, "N": N, "prec": "fp32"}}
    for name, law in (("gauss", 0), ("lognormal", 1)):
        prob = saa.Problem(mu=torch.tensor(inst.mu, device=dev), chol=torch.tensor(inst.chol, device=dev), N=N,
                           law=law, seed=0)
        buf = saa.saa_generate_moments(prob, 0, N, "fp32")
        for _ in range(2):
            saa.saa_generate_moments(prob, 0, N, "fp32", out=buf)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(3, min(args.steps, 20))
        e0.record()
        for _ in range(steps):
            saa.saa_generate_moments(prob, 0, N, "fp32", out=buf)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"value": N * d / (ms / 1e3), "ms_per_call": ms}
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    d, N, K, law = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["K"], WORKLOAD["law"]
    import oracle
    from paper_2404_11631_gb300 import inputs
    inst = inputs.instance(d, 0)
    X = inputs.decisions(K, d, 0)
    # per-step sample sized so that warmup + steps stay within a few minutes
    n = 1 << 13
    prob = oracle.make_problem(d, n, inst.mu, inst.chol, law=law, seed=0)
    t0 = time.perf_counter()
    oracle.saa(prob, 32, X)
    one = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)
    while one * 2 < budget and n * 2 <= N:
        n *= 2
        one *= 2
    prob = oracle.make_problem(d, n, inst.mu, inst.chol, law=law, seed=0)
    for _ in range(args.warmup):
        oracle.saa(prob, 32, X)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.saa(prob, 32, X)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = n * K / (ms / 1e3)
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "d": d, "N": N, "K": K, "law": "half Gaussian / half lognormal",
                   "sample_N_per_step": n},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} of {N} scenarios x all {K} decisions per step (FP64 oracle, OpenMP)"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2404_11631_gb300 import inputs, saa

    world, rank, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    d, N, K, law = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["K"], WORKLOAD["law"]
    prec = args.prec
    inst = inputs.instance(d, 0)
    Xn = inputs.decisions(K, d, 0)
    mu = torch.tensor(inst.mu, device=dev)
    ch = torch.tensor(inst.chol, device=dev)
    X = torch.tensor(Xn, device=dev)
    prob = saa.Problem(mu=mu, chol=ch, N=N, law=law, seed=0, instance=rank)
    ws = torch.empty(saa.workspace_size(prob, K, prec, 0), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step():
        return saa.saa_eval(prob, X, prec, ws=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    saa.saa_profile_enable(True, dev.index)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else 0) as clk:
        for i in range(args.steps):
            flush.zero_()                       # L2 flushed between timed steps (outside the event pair)
            ev[i][0].record(stream)
            out = step()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    main_ms, main_n, launched = saa.saa_profile_read(dev.index)
    saa.saa_profile_enable(False, dev.index)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
        dist.barrier()
    ms_per_step = 1e3 * total_s / args.steps
    value = world * N * K * args.steps / total_s

    # e2e through the C ABI with host buffers: saa_eval_host takes mu, C and
    # X in pinned host memory, copies them in, evaluates (f, pbar and var, as
    # the timed leg does), copies the outputs back and waits for the stream;
    # each step is timed by the host wall clock around that one call.
    mu_h = torch.tensor(inst.mu).pin_memory()
    ch_h = torch.tensor(inst.chol).pin_memory()
    X_h = torch.tensor(Xn).pin_memory()
    out_h = {k: torch.empty(K, dtype=torch.float64).pin_memory() for k in ("f", "pbar", "var")}
    prob_h = saa.Problem(mu=mu_h, chol=ch_h, N=N, law=law, seed=0, instance=rank)
    ws_h = torch.empty(saa.saa_eval_host_workspace_size(prob_h, K, prec, dev.index), dtype=torch.uint8, device=dev)

    def e2e_step():
        saa.saa_eval_host(prob_h, X_h, prec, out=out_h, ws=ws_h, device=dev.index)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = 0.0
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_step()
        e2e_s += time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * N * K * args.steps / e2e_s
    h2d = (mu_h.numel() + ch_h.numel() + X_h.numel()) * 8
    d2h = 3 * K * 8
    e2e_f_match = bool(torch.equal(out_h["f"], out["f"].cpu()))

    peaks, peak_src = _peaks()
    kern_s = main_ms / 1e3 / max(1, main_n)
    roof = roofline(prec, d, N, K, law, kern_s, peaks, peak_src)

    # the plain FP64 GPU path on the same workload (the comparator of the metric)
    fp64 = None
    if prec != "fp64" and not args.no_fp64:
        ws64 = torch.empty(saa.workspace_size(prob, K, "fp64", 0), dtype=torch.uint8, device=dev)
        saa.saa_eval(prob, X, "fp64", ws=ws64)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            saa.saa_eval(prob, X, "fp64", ws=ws64)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1) / 3
        v64 = N * K / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": "evals/s", "ms_per_step": ms64, "speedup": value / world / v64}
        del ws64

    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "bf16x3", "f16x3": "f16x3"}[prec],
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "d": d, "N": N, "K": K,
                   "law": "half Gaussian / half standardised lognormal", "prec": prec,
                   "l2": "flushed (256 MB write) between timed steps", "instances": world},
        "gpu_launches": int(launched),
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "timing": "host wall clock around each saa_eval_host call (copies in, f/pbar/var, copies out, "
                          "stream wait); L2 flushed between calls", "f_equals_device_leg": e2e_f_match},
        "roofline": roof,
    }
    if fp64:
        line["fp64_gpu_path"] = fp64
    if not args.no_grad:
        line["eval_grad"] = run_grad(args, dev, world, rank, flush, stream)
    if not args.no_fw:
        line["fw"] = run_fw(args, dev, world, rank)
    if not args.no_ragged:
        line["ragged"] = run_ragged(args, dev, world, rank, flush, stream)
    if not args.no_newsvendor:
        line["newsvendor"] = run_newsvendor(args, dev, world, rank, flush, stream)
    if not args.no_cov:
        line["covariance_first"] = run_covariance(args, dev, world, rank, flush, stream)
    if not args.no_streamed:
        line["streamed"] = run_streamed(args, dev, world, rank, flush, stream)
    if not args.no_logistic:
        line["logistic"] = run_logistic(args, dev, world, rank, flush, stream)
    if not args.no_large_d:
        line["portfolio_large_d"] = run_large_d(args, dev, world, rank, flush, stream)
    if rank == 0:
        line["clocks"] = clk.summary()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, n, cores = oracle_sample(d, K, law)
        line["cpu_baseline"] = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n} of {N} scenarios x all {K} decisions, {dt:.1f} s (FP64 oracle)"}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=os.environ.get("SAA_BENCH_PREC", "f16x3"),
                    choices=["fp64", "fp32", "bf16x3", "f16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the FP64 GPU comparator")
    ap.add_argument("--no-grad", action="store_true", help="skip the value-and-gradient workload")
    ap.add_argument("--grad-N", type=int, default=None, help="override the gradient workload's scenario count")
    ap.add_argument("--grad-only", action="store_true", help="run only the value-and-gradient workload")
    ap.add_argument("--gen-only", action="store_true", help="time the bare generator (per-normal figure)")
    ap.add_argument("--no-fw", action="store_true", help="skip the Algorithm 1 (Frank-Wolfe) workload")
    ap.add_argument("--fw-only", action="store_true", help="run only the Algorithm 1 workload")
    ap.add_argument("--no-ragged", action="store_true", help="skip the 4096-instance ragged batch")
    ap.add_argument("--ragged-B", type=int, default=4096, help="instances of the ragged batch (profiling small cases)")
    ap.add_argument("--ragged-only", action="store_true", help="run only the ragged batch")
    ap.add_argument("--no-newsvendor", action="store_true", help="skip the newsvendor gradient workload")
    ap.add_argument("--no-cov", action="store_true", help="skip the covariance-first workload")
    ap.add_argument("--cov-only", action="store_true", help="run only the covariance-first workload")
    ap.add_argument("--nv-only", action="store_true", help="run only the newsvendor gradient workload")
    ap.add_argument("--no-streamed", action="store_true", help="skip the streamed-samples workload")
    ap.add_argument("--no-logistic", action="store_true", help="skip the binary-classification workload")
    ap.add_argument("--logistic-only", action="store_true", help="run only the binary-classification workload")
    ap.add_argument("--streamed-only", action="store_true", help="run only the streamed-samples workload")
    ap.add_argument("--no-large-d", action="store_true", help="skip the 10^5-asset diagonal portfolio workload")
    ap.add_argument("--large-d-only", action="store_true", help="run only the 10^5-asset diagonal portfolio workload")
    ap.add_argument("--ld-d", type=int, default=None, help="override the diagonal portfolio's dimension (profiling)")
    ap.add_argument("--ld-N", type=int, default=None, help="override the diagonal portfolio's sample count (profiling)")
    ap.add_argument("--nv-n", type=int, default=None, help="override the newsvendor product count")
    ap.add_argument("--fw-N", type=int, default=None, help="override the Algorithm 1 scenario count")
    ap.add_argument("--fw-T", type=int, default=None, help="override the Algorithm 1 iteration count")
    ap.add_argument("--N", type=int, default=None, help="override the scenario count (profiling small cases)")
    ap.add_argument("--K", type=int, default=None, help="override the decision count (profiling small cases)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.N:
        WORKLOAD["N"] = args.N
        WORKLOAD["name"] += f"_N{args.N}"
    if args.K:
        WORKLOAD["K"] = args.K
        WORKLOAD["name"] += f"_K{args.K}"
    if args.grad_N:
        GRAD_WORKLOAD["N"] = args.grad_N
        GRAD_WORKLOAD["name"] += f"_N{args.grad_N}"
    if args.impl == "reference":
        return run_reference(args)
    if args.fw_N:
        FW_WORKLOAD["N"] = args.fw_N
        FW_WORKLOAD["name"] += f"_N{args.fw_N}"
    if args.fw_T:
        FW_WORKLOAD["T"] = args.fw_T
        FW_WORKLOAD["name"] += f"_T{args.fw_T}"
    if args.gen_only:
        return run_gen(args)
    if args.ld_d or args.ld_N:
        LD_WORKLOAD["d"] = args.ld_d or LD_WORKLOAD["d"]
        LD_WORKLOAD["N"] = args.ld_N or LD_WORKLOAD["N"]
        LD_WORKLOAD["name"] = f"portfolio_diag_d{LD_WORKLOAD['d']}_N{LD_WORKLOAD['N']}"
    if args.nv_n:
        NV_WORKLOAD["n"] = args.nv_n
        NV_WORKLOAD["name"] = f"newsvendor_n{args.nv_n}_S{NV_WORKLOAD['S']}_K1"
    if args.grad_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps(run_grad(args, dev, 1, 0, flush, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.cov_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps(run_covariance(args, dev, 1, 0, flush, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.large_d_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps(run_large_d(args, dev, 1, 0, flush, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.logistic_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps(run_logistic(args, dev, 1, 0, flush, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.streamed_only:
        import torch
        dev = torch.device("cuda", 0)
        print(json.dumps(run_streamed(args, dev, 1, 0, None, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.nv_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps(run_newsvendor(args, dev, 1, 0, flush, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.ragged_only:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps(run_ragged(args, dev, 1, 0, flush, torch.cuda.current_stream(dev))), flush=True)
        return 0
    if args.fw_only:
        import torch
        print(json.dumps(run_fw(args, torch.device("cuda", 0), 1, 0)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
