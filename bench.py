#!/usr/bin/env python
"""Benchmark of the step-truncation RK4 TT solver (Burgers-Hopf, GB300).

One step = one full RK4 step of the hot path: 4 operator applies, 8 TT
roundings (right-to-left Householder orthogonalisation + left-to-right
truncated SVD) and 4 TT sums, on the d=32, n=128, rank<=64 workload, in the
"saturated" state (every interior rank at the cap 64: a seeded TT with random
orthonormal cores), complex values in FP64 storage.  ``value`` is the mixed-
precision solver (FP64 Householder scalars and SVD, double-float QR arithmetic); the FP64 solver
is timed on the same state under the ``fp64`` key, and the mixed-vs-FP64
error is measured on a physical state.  In the mixed solver the products of
the tall QR factorisations and Q applications run on the tensor cores
(tcgen05) as digit-split BF16 products with exact FP32 accumulation.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas (one per
GPU, launched by torchrun); value = steps of all ranks / max time over ranks.
``--impl reference`` times the CPU oracle on a bounded sample of the same
workload on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TT RK4 steps/s (d=32,n=128,r≤64) mixed vs FP64 @≤1e-6 err; roofline %"
FP64_PEAK_TFLOPS = 152 * 2070e6 * 4 / 1e12  # 152 SMs x 2 DFMA/clk x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 2070e6 * 256 / 1e12  # 152 SMs x 128 FFMA/clk x 2.07 GHz
# double-float complex multiply-add: 4 real multiply-adds of ~13 FP32
# operations each = 52 FP32 operations for 8 FP64-equivalent FLOPs
DF_OPS_PER_FLOP = 52.0 / 8.0


def workload():
    import synthetic
    w = synthetic.C3
    return w


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                smax.append(float(s[1]))
            except ValueError:
                continue
            for name, v in zip(names, s[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- oracle arm ----
def oracle_sample_seconds(d_sample: int = 4):
    """One full step-truncation RK4 step (four operator applies, eight
    roundings and the stage sums) by the CPU oracle on a d_sample-core slice
    of the saturated workload.  Returns (seconds, seconds per RK4 step at the
    workload's d extrapolated by the number of bonds, (d-1)/(d_sample-1)).
    The slice's two end cores are cheaper than interior ones, so the
    extrapolation overstates the oracle's rate."""
    from oracle import model, tt
    import synthetic
    w = workload()
    cores, _ = synthetic.saturated_tt_cores(d_sample, w.n, w.cap, seed=0)
    m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    W = model.mpo_blocks(d_sample, w.n, L, w.nu)
    bond = model.mpo_bond_dims(d_sample)
    t0 = time.perf_counter()
    tt.rk4_step(cores, w.dt, W, bond, w.tol, w.cap)
    sec = time.perf_counter() - t0
    return sec, sec * (w.d - 1) / (d_sample - 1)


def oracle_sample_text(sec):
    return (f"one full RK4 step (4 applies, 8 roundings, stage sums) on a 4-core slice (d=4, n=128, r=64) "
            f"of the saturated state, {sec:.1f} s measured; extrapolated to d=32 by bonds (x 31/3)")


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def max_over_ranks(x, world, device="cpu"):
    """Largest value of x over the ranks of the default process group
    (world 1: x itself): the slowest replica sets the job's time."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, slowest_seconds, world):
    """Whole-job throughput of `world` independent replicas that each
    processed `units_per_rank` units: all units over the slowest time."""
    return world * units_per_rank / slowest_seconds


def run_reference(args, rank):
    if rank != 0:
        return None
    w = workload()
    for _ in range(args.warmup):
        oracle_sample_seconds()
    per, secs = [], []
    for _ in range(args.steps):
        sec, full = oracle_sample_seconds()
        secs.append(sec)
        per.append(full)
    step_s = sum(per) / len(per)
    sample_s = sum(secs) / len(secs)
    value = 1.0 / step_s
    sample = oracle_sample_text(sample_s)
    # ms_per_step: the wall time of one bench step (the sample itself);
    # value: the extrapolated full-workload rate
    return {"metric": METRIC, "value": value, "unit": "steps/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sample_s * 1e3, "extrapolated_ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w),
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def config_dict(w):
    return {"workload": f"saturated TT, d={w.d}, n={w.n}, rank cap {w.cap} (all interior ranks at the cap), "
                        f"tol {w.tol:g}, dt {w.dt:g}, nu {w.nu}, FP64 complex",
            "d": w.d, "n": w.n, "rank_cap": w.cap, "tol": w.tol, "dt": w.dt,
            "precision": "mixed (value) and fp64 (fp64 key)",
            "state": "seeded random orthonormal cores (seed 0)",
            "l2": "working set (~20 GB) larger than L2; no flush needed",
            "parallelism": "replicas"}


# ---------------------------------------------------------------- our arm ----
def timed_steps(ctx, t, w, steps, warmup, stream, barrier):
    import torch
    for _ in range(warmup):
        ctx.hopf_step(t, w.dt, 1)
    ctx.hopf_profile_read(reset=True)
    ctx.hopf_profile_enable(True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.hopf_step(t, w.dt, 1)
    e1.record(stream)
    barrier()
    prof = ctx.hopf_profile_read(reset=True)
    ctx.hopf_profile_enable(False)
    return e0.elapsed_time(e1) / 1e3, prof


# Tensor-core products of the mixed path: every complex multiply-add (8
# FP64-equivalent FLOPs) costs 3 real products (3M) x 15 digit pairs (5
# digits per operand) of BF16 multiply-adds, i.e. 45 real multiply-adds
# where the FP64-equivalent count assigns 4.
TC_DIGIT_PAIRS = 15
TC_BF16_PER_FP64EQ = 3 * TC_DIGIT_PAIRS / 4.0


def tc_roofline(prof, peaks):
    """The tensor-core class (digit splitting included) against the measured
    sustained BF16 peak (the products run inside a seconds-long step),
    expressed in FP64-equivalent complex FLOP/s."""
    pd = prof.get("tc", {})
    if not pd or pd.get("ms", 0) <= 0 or pd.get("flops", 0) <= 0:
        return None
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    src = "of measured (bf16_tflops_sustained, MEASURED_PEAKS.json)"
    if not bf16:
        bf16, src = 1700.0, "of fallback (1.7 PFLOP/s sustained bf16)"
    achieved = pd["flops"] / (pd["ms"] / 1e3) / 1e12
    peak = bf16 / TC_BF16_PER_FP64EQ
    return {"bound": "tensor", "kernel": "tc (tc_zgemm_kernel + digit splitting)", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"{bf16:.1f} TFLOP/s bf16 {src} / {TC_BF16_PER_FP64EQ:.2f} bf16 multiply-adds "
                           "per FP64-equivalent one (3M x 15 digit pairs / 4)",
            "bf16_tflops_achieved": achieved * TC_BF16_PER_FP64EQ, "traffic": None}


# DRAM traffic of one 128-column mixed panel launch of geqrf_kernel, from the
# ncu capture summarised in profiles/geqrf_panel_16128x128_mixed.md:
# dram__bytes_read.sum + dram__bytes_write.sum = 35.4 MB for a 16128 x 128
# panel, i.e. bytes per panel element (the panel is read once; its write-back
# stays in L2).  Traffic grows with the panel's rows, so a launch of m rows
# moves about this many bytes per element of its m x 128 panel.
PANEL_COLS = 128
PANEL_DRAM_BYTES_PER_ELEM = (33.218304e6 + 2.177024e6) / (16128 * PANEL_COLS)


def panel_traffic(pd):
    """DRAM bytes per launch of the mixed tensor-core path's panel kernel,
    scaled from the capture by the mean panel rows m, recovered from the
    mean FLOPs per launch F = 8 m k^2 - 8 k^3 / 3 (k = 128)."""
    launches = max(pd.get("timed_launches", 0), 1)
    k = float(PANEL_COLS)
    m = (pd["flops"] / launches + 8.0 * k ** 3 / 3.0) / (8.0 * k * k)
    return PANEL_DRAM_BYTES_PER_ELEM * m * k


def roofline(prof, mixed, peaks, tensor_qr=False):
    """Dominant contraction kernel class (largest device time among classes
    with an algorithmic FLOP count) against the peak of its own arithmetic."""
    cls = [k for k in prof if isinstance(prof[k], dict) and prof[k].get("flops", 0) > 0 and prof[k]["ms"] > 0]
    dom = max(cls, key=lambda k: prof[k]["ms"])
    if dom == "tc":
        return tc_roofline(prof, peaks)
    pd = prof[dom]
    launch_s = pd["ms"] / 1e3 / max(pd["timed_launches"], 1)
    achieved = pd["flops"] / max(pd["timed_launches"], 1) / launch_s / 1e12
    if mixed:
        peak = FP32_PEAK_TFLOPS / DF_OPS_PER_FLOP
        src = ("double-float on the FP32 pipe: 152 SMs x 256 FLOP/clk x 2.07 GHz / 6.5 FP32 ops per "
               "FP64-equivalent FLOP (derived); Householder scalars in FP64 inside the same kernel")
    else:
        peak = FP64_PEAK_TFLOPS
        src = "FP64 FMA: 152 SMs x 4 FLOP/clk x 2.07 GHz (derived; DFMA microbenchmark measured 1.19)"
    out = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "peak_source": src, "traffic": None}
    if mixed and tensor_qr and dom == "qr":
        # only the tensor-core path's panel kernel has counters taken since
        # its last change; the whole-matrix variants' captures predate it
        out["traffic"] = panel_traffic(pd)
        out["traffic_source"] = ("ncu dram__bytes of one 16128 x 128 panel launch (35.4 MB), scaled to the mean "
                                 "launch's panel rows")
    return out


def natural_state_error(w, stream, nsteps=3, qr_method=1):
    """Mixed vs FP64 after nsteps from the physical C3 initial state: the
    Gaussian with the C3 mean and cell covariance (correlated), built by
    hopf_init_gaussian (TT-cross at this size; every interior rank at the
    cap), errors in Phi (TT difference norm), mean and covariance."""
    import numpy as np
    from paper_2403_04946_gb300 import binding as B
    c0 = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=1.0, stream=stream)
    m0, C0 = c0.hopf_cell_moments(w.alpha, w.beta, w.sigma, w.ell)
    c0.close()
    import torch
    out, rate = {}, {}
    for prec in (B.HOPF_FP64, B.HOPF_MIXED):
        ctx = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=0.0, stream=stream, precision=prec)
        ctx.hopf_set_qr_method(qr_method)
        t = ctx.hopf_init_gaussian(m0, C0)
        r0 = ctx.tt_get_ranks(t)
        ctx.hopf_step(t, w.dt, 1)  # first step: workspace set-up, untimed
        st = torch.cuda.ExternalStream(stream) if isinstance(stream, int) else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        ctx.hopf_step(t, w.dt, nsteps - 1)
        e1.record(st)
        torch.cuda.synchronize()
        rate[prec] = (nsteps - 1) / (e0.elapsed_time(e1) / 1e3)
        mean, cov, _ = ctx.hopf_eval_moments(t)
        out[prec] = (ctx.tt_to_host(t), mean, cov, ctx.tt_get_ranks(t), r0)
        ctx.close()
    (cf, mf, vf, rf, r0), (cm, mm, vm, rm, _) = out[B.HOPF_FP64], out[B.HOPF_MIXED]
    ctx = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=12.4, stream=stream)
    a = ctx.tt_from_host(cf, max_rank=max(rf))
    b = ctx.tt_from_host(cm, max_rank=max(rm))
    dif = ctx.tt_create(max(rf) + max(rm))
    ctx.tt_sum([a, b], [1.0, -1.0], dif)
    phi = ctx.tt_norm(dif) / ctx.tt_norm(a)
    ctx.close()
    return {"phi_rel_l2": phi, "mean_rel_max": float(np.abs(mm - mf).max() / np.abs(mf).max()),
            "cov_rel_max": float(np.abs(vm - vf).max() / np.abs(vf).max()), "steps": nsteps,
            "state": "C3 Gaussian initial state (correlated cell covariance), TT-cross construction rounded to "
                     "tol 1e-7 / cap 64",
            "initial_max_rank": int(max(r0)), "max_rank": int(max(rm)),
            "natural_steps_per_s": {"mixed": rate[B.HOPF_MIXED], "fp64": rate[B.HOPF_FP64],
                                    "note": "one RK4 step timed after one untimed step from the same state"}}


def paper_workload(stream_int, qr_method=1, d=20, n=64, r=128):
    """The paper's own experiment at its largest size (Sec. 5.1): the CDF
    equation with N = 20, n = 64 points per variable on [-1.3, 1.3]^20 and
    the explicit step-truncation midpoint scheme, on a saturated synthetic
    state with every interior rank at 128 (the paper reports ranks above
    100).  One untimed step (workspaces), one timed step."""
    import torch
    from paper_2403_04946_gb300 import binding as B
    import synthetic
    cores, _ = synthetic.saturated_tt_cores(d, n, r, seed=0)
    ctx = B.Context(d=d, n=n, nu=0.01, tol=1e-7, rank_cap=r, stream=stream_int, precision=B.HOPF_MIXED)
    ctx.hopf_set_qr_method(qr_method)
    ctx.hopf_set_equation(B.HOPF_EQ_CDF, 1.3)
    t = ctx.tt_from_host(cores, max_rank=r)
    ctx.hopf_step_scheme(t, B.HOPF_MIDPOINT, 1e-4, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.hopf_step_scheme(t, B.HOPF_MIDPOINT, 1e-4, 1)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ctx.tt_free(t)
    ctx.close()
    return {"equation": "CDF (Eq. cdf-burgers, alpha = 0), box [-1.3, 1.3]^20", "d": d, "n": n, "rank": r,
            "scheme": "explicit step-truncation midpoint (3 roundings per step)", "precision": "mixed",
            "seconds_per_step": sec,
            "paper_context": {"seconds_per_step": 45 * 60, "hardware": "Intel i9-7980XE workstation, CPU, FP64",
                              "ranks": "above 100", "note": "context only: other hardware and precision"}}


def ensemble_rate(stream_int, nsteps=1, qr_method=1):
    """An ensemble of uneven instances (saturated states, ranks at their
    caps), one RK4 step each: one instance at a time on the whole GPU versus
    all at once (hopf_step_ensemble, each context limited to its share of
    the SMs).  Steps per second of the whole ensemble, wall clock."""
    import torch
    from paper_2403_04946_gb300 import binding as B
    import synthetic
    specs = [(16, 64, 32), (12, 96, 32), (16, 64, 24), (8, 128, 32)]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    share = sms // len(specs)
    out = {}
    for mode in ("sequential", "concurrent"):
        members = []
        for i, (d, n, r) in enumerate(specs):
            cores, _ = synthetic.saturated_tt_cores(d, n, r, seed=40 + i)
            s = torch.cuda.Stream() if mode == "concurrent" else None
            ctx = B.Context(d=d, n=n, nu=0.02, tol=1e-7, rank_cap=r, L=12.4,
                            stream=s.cuda_stream if s is not None else stream_int, precision=B.HOPF_MIXED)
            ctx.hopf_set_qr_method(qr_method)
            if mode == "concurrent":
                ctx.hopf_set_max_ctas(share)
            members.append((ctx, ctx.tt_from_host(cores, max_rank=r), s))
        run = (lambda: B.hopf_step_ensemble([(c, t) for c, t, _ in members], 1.2e-5, nsteps)) \
            if mode == "concurrent" else \
            (lambda: [c.hopf_step(t, 1.2e-5, nsteps) for c, t, _ in members])
        run()  # warm-up: workspaces
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run()
        torch.cuda.synchronize()
        out[mode] = len(specs) * nsteps / (time.perf_counter() - t0)
        for c, t, _ in members:
            c.tt_free(t)
            c.close()
    return {"instances": [{"d": d, "n": n, "rank": r} for d, n, r in specs],
            "sms_per_instance_concurrent": share, "precision": "mixed",
            "steps_per_s_sequential": out["sequential"], "steps_per_s_concurrent": out["concurrent"],
            "speedup": out["concurrent"] / out["sequential"]}


def c4_sample(stream_int, count=4, nsteps=1, qr_method=1):
    """The first `count` draws of the C4 ensemble generator (seed 0..): d in
    8..48, n in {64, 96, 128}, nu, sigma, ell and four Fourier modes of the
    mean drawn per instance, cap 64, tol 1e-7, dt 1e-5, mixed precision; each
    from its own Gaussian initial state (hopf_cell_moments +
    hopf_init_gaussian).  After one untimed step (workspaces), one RK4 step
    of every instance one at a time on the whole GPU, then one all at once
    (hopf_step_ensemble, equal SM shares).  Ensemble steps per second, wall
    clock."""
    import torch
    from paper_2403_04946_gb300 import binding as B
    import synthetic
    draws = [synthetic.ensemble_member(s) for s in range(count)]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    share = max(1, sms // count)
    t0 = time.perf_counter()
    members = []
    for w in draws:
        s = torch.cuda.Stream()
        ctx = B.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=0.0, stream=s.cuda_stream,
                        precision=B.HOPF_MIXED)
        ctx.hopf_set_qr_method(qr_method)
        m0, C0 = ctx.hopf_cell_moments(w.alpha, w.beta, w.sigma, w.ell)
        t = ctx.hopf_init_gaussian(m0, C0)
        members.append((ctx, t, s, max(ctx.tt_get_ranks(t))))
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    for (c, t, _, _), w in zip(members, draws):
        c.hopf_step(t, w.dt, nsteps)  # workspaces
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (c, t, _, _), w in zip(members, draws):
        c.hopf_step(t, w.dt, nsteps)
    torch.cuda.synchronize()
    seq = len(draws) * nsteps / (time.perf_counter() - t0)
    for c, _, _, _ in members:
        c.hopf_set_max_ctas(share)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.hopf_step_ensemble([(c, t) for c, t, _, _ in members], draws[0].dt, nsteps)
    torch.cuda.synchronize()
    conc = len(draws) * nsteps / (time.perf_counter() - t0)
    ranks = [max(c.tt_get_ranks(t)) for c, t, _, _ in members]
    for c, t, _, _ in members:
        c.tt_free(t)
        c.close()
    return {"generator": "C4 (synthetic.ensemble_member), seeds 0..%d" % (count - 1),
            "instances": [{"d": w.d, "n": w.n, "initial_max_rank": m[3], "max_rank_after": r}
                          for w, m, r in zip(draws, members, ranks)],
            "initial_states_s": t_init, "sms_per_instance_concurrent": share, "precision": "mixed",
            "steps_per_s_sequential": seq, "steps_per_s_concurrent": conc, "speedup": conc / seq}


def surrogate_rate(ntrain=128, ncalib=16, nheld=24, iters=12000, batch=128):
    """The learned surrogate on the C4 parameter distribution at the C1 grid
    (d=4, n=24, dt=1e-2, T = 0.01..0.1): solver-made training data, GPU
    training of the 4-member ensemble, calibration of its bound on separate
    solves, then held-out queries answered with the solver as fallback
    (bound <= 1e-3), timed against the solver alone on the same queries."""
    import numpy as np
    from paper_2403_04946_gb300 import binding as B, surrogate as S
    import synthetic
    d, width, depth, members, tol = 4, 256, 4, 4, 1e-3
    snaps = list(range(1, 11))
    train = [synthetic.surrogate_member(s) for s in range(1, 1 + ntrain)]
    calib = [synthetic.surrogate_member(s) for s in range(10001, 10001 + ncalib)]
    held = [synthetic.surrogate_member(s) for s in range(20001, 20001 + nheld)]
    t0 = time.perf_counter()
    Xt, Rt, _, _, _ = S.dataset(train, snaps, concurrency=8)
    t_data = time.perf_counter() - t0
    Xc, _, Bc, YTc, Tc = S.dataset(calib, snaps, concurrency=8)
    dims = [S.n_in(d)] + [width] * depth + [S.n_out(d)]
    ctx = B.Context(d=4, n=8, nu=0.05, tol=1e-10, rank_cap=4, L=3.0)
    sur = S.Surrogate(ctx, d, synthetic.mlp_init(7, dims, members), width=width, depth=depth, members=members)
    lr = 1e-5 + 0.5 * (1e-3 - 1e-5) * (1 + np.cos(np.pi * np.arange(iters) / iters))
    t0 = time.perf_counter()
    loss = sur.fit(Xt, Rt, synthetic.batch_indices(8, iters, members, batch, len(Xt)), lr)
    t_train = time.perf_counter() - t0
    kappa, _, _ = sur.calibrate(Xc, Bc, Tc, YTc)
    steps = [snaps[i % len(snaps)] for i in range(nheld)]
    t0 = time.perf_counter()
    ref = np.concatenate([S.solve([held[i] for i in range(nheld) if steps[i] == s], [s], concurrency=8)[:, 0]
                          for s in sorted(set(steps))])
    t_solver = time.perf_counter() - t0
    order = np.concatenate([[i for i in range(nheld) if steps[i] == s] for s in sorted(set(steps))]).astype(int)
    y_ref = np.empty_like(ref)
    y_ref[order] = ref
    # the method without the network: the solver's first-order extrapolation
    # y(T) ~ y0 + T ydot0 (and, for reference, y(T) ~ y0)
    Y0h, Ydh = S.solve(held, [0], concurrency=8, rate0=True)
    y0_held = Y0h[:, 0]
    T_held = np.array([s * w.dt for w, s in zip(held, steps)])
    base_held = y0_held + T_held[:, None] * Ydh
    answers = {}
    for tq in (tol, 10 * tol):
        ans = sur.answer(held, steps, tq)
        t_answer = ans["t_y0"] + ans["t_net"] + ans["t_fallback"]
        answers[f"{tq:g}"] = {"accepted": float(ans["accepted"].mean()),
                              "max_err_served": float(S.rel_err(ans["y"], y_ref).max()),
                              "queries_per_s": nheld / t_answer, "gain_vs_solver": t_solver / t_answer,
                              "seconds_y0_net_fallback": [round(ans["t_y0"], 3), round(ans["t_net"], 4),
                                                          round(ans["t_fallback"], 3)]}
    err_net = S.rel_err(ans["y_net"], y_ref)
    # network throughput alone on a large query batch (inputs on the host)
    reps = -(-4096 // len(Xc))
    Xq, Y0q, Tq = (np.repeat(a, reps, axis=0)[:4096] for a in (Xc, Bc, Tc))
    sur.predict(Xq, Y0q, Tq)
    t0 = time.perf_counter()
    for _ in range(5):
        sur.predict(Xq, Y0q, Tq)
    t_q = (time.perf_counter() - t0) / 5
    sur.close()
    ctx.close()
    return {"config": "d=4, n=24, rank cap 16, tol 1e-10, dt 1e-2, T in 0.01..0.1; C4 parameter draws; "
                      f"MLP {dims[0]}->{width}x{depth}->{dims[-1]} GELU, {members} members, bf16 weights",
            "train_solves": ntrain, "train_pairs": int(len(Xt)), "data_s": round(t_data, 2),
            "train_steps": iters, "train_s": round(t_train, 2),
            "loss_first_last": [float(loss[:10].mean()), float(loss[-50:].mean())],
            "kappa": kappa, "held_out_queries": nheld,
            "median_err_network": float(np.median(err_net)),
            "median_err_without_network": float(np.median(S.rel_err(base_held, y_ref))),
            "without_network": "first-order extrapolation y0 + T ydot0 from the solver's initial state",
            "median_err_y0_only": float(np.median(S.rel_err(y0_held, y_ref))),
            "solver_queries_per_s": nheld / t_solver, "answers_at_bound": answers,
            "network_queries_per_s": 4096 / t_q}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2403_04946_gb300 import binding
    import synthetic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = workload()
    ctx0 = binding.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=1.0,
                           stream=stream.cuda_stream)
    m0, C0 = ctx0.hopf_cell_moments(w.alpha, w.beta, w.sigma, w.ell)
    ctx0.close()
    L = float(np.sqrt(36.8 / np.min(np.diag(C0))))
    cores, ranks = synthetic.saturated_tt_cores(w.d, w.n, w.cap, seed=0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def maxover(x):
        return max_over_ranks(x, world, dev)

    gpu_id = "0"
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass

    # primary arm: mixed precision (FP64 Householder scalars and SVD, double-float QR arithmetic)
    qr_method = binding.HOPF_QR_TENSOR if args.qr_method == "tensor" else binding.HOPF_QR_DOUBLEFLOAT
    ctx = binding.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L,
                          stream=stream.cuda_stream, precision=binding.HOPF_MIXED)
    ctx.hopf_set_qr_method(qr_method)
    if not args.no_autotune:
        ctx.hopf_set_autotune(True)  # shapes are tuned during the warm-up steps
    t = ctx.tt_from_host(cores, max_rank=w.cap)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    elapsed, prof = timed_steps(ctx, t, w, args.steps, args.warmup, stream, barrier)
    clocks.stop()
    elapsed = maxover(elapsed)

    # end to end through the C ABI: pinned host state in, step, state out
    ranks_np = np.asarray(ranks, dtype=np.int32)
    _, flat = binding.cores_to_flat(cores)
    host_in = torch.from_numpy(flat.copy()).pin_memory()
    nd = flat.size
    host_out = torch.empty(nd, dtype=torch.float64).pin_memory()
    import ctypes
    pin_in = ctypes.cast(host_in.data_ptr(), ctypes.POINTER(ctypes.c_double))
    pin_out = ctypes.cast(host_out.data_ptr(), ctypes.POINTER(ctypes.c_double))
    k_e2e = max(1, args.steps)
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        ctx.tt_set_from_host(t, ranks=ranks_np, flat=pin_in)
        ctx.hopf_step(t, w.dt, 1)
        ctx.tt_to_host_into(t, pin_out, ctx.tt_size(t))
    barrier()
    e2e_s = maxover(time.perf_counter() - t0)
    out_bytes = ctx.tt_size(t) * 8
    tune_table = ctx.hopf_get_autotune()
    ctx.tt_free(t)
    ctx.close()

    # FP64 arm on the same state (the comparison the metric names)
    ctx = binding.Context(d=w.d, n=w.n, nu=w.nu, tol=w.tol, rank_cap=w.cap, L=L,
                          stream=stream.cuda_stream, precision=binding.HOPF_FP64)
    t = ctx.tt_from_host(cores, max_rank=w.cap)
    el64, prof64 = timed_steps(ctx, t, w, args.steps, 1, stream, barrier)
    el64 = maxover(el64)
    ctx.tt_free(t)
    ctx.close()

    err = natural_state_error(w, stream.cuda_stream, qr_method=qr_method) if not args.no_error_check else None
    ens = ensemble_rate(stream.cuda_stream, qr_method=qr_method) if not args.no_error_check else None
    c4 = c4_sample(stream.cuda_stream, count=args.c4_count, qr_method=qr_method) \
        if (not args.no_error_check and args.c4_count > 0) else None
    sur = surrogate_rate() if (world == 1 and not args.no_surrogate) else None
    paper = paper_workload(stream.cuda_stream, qr_method=qr_method) if not args.no_error_check else None

    result = None
    if rank == 0:
        peaks = read_peaks()
        value = replica_rate(args.steps, elapsed, world)
        total_ms = sum(v["ms"] for v in prof.values() if isinstance(v, dict))
        shares = {k: round(v["ms"] / total_ms, 4) for k, v in prof.items() if isinstance(v, dict) and v["ms"] > 0}
        total64 = sum(v["ms"] for v in prof64.values() if isinstance(v, dict))
        shares64 = {k: round(v["ms"] / total64, 4) for k, v in prof64.items() if isinstance(v, dict) and v["ms"] > 0}
        apply_gbs = (prof["apply"]["bytes"] / (prof["apply"]["ms"] / 1e3) / 1e9) if prof["apply"]["ms"] > 0 else None
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            sec, per_step = oracle_sample_seconds()
            cpu = {"value": 1.0 / per_step, "unit": "steps/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": oracle_sample_text(sec)}
        cfg = config_dict(w)
        cfg["qr_method"] = args.qr_method
        cfg["autotune"] = not args.no_autotune
        result = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f64 storage; QR trailing products and Q applications of tall factors on tensor cores "
                      "(bf16 digit products, 5 digits, exact f32 accumulation, 3M complex); QR panels and merges "
                      "in double-float (2 x f32); f64 Householder scalars and SVD"),
            "data": "synthetic", "config": cfg,
            "roofline": roofline(prof, True, peaks, tensor_qr=(qr_method == binding.HOPF_QR_TENSOR)),
            "tensor_core_roofline": tc_roofline(prof, peaks),
            "kernel_shares": shares,
            "autotune": tune_table,
            "fp64": {"value": replica_rate(args.steps, el64, world), "unit": "steps/s", "ms_per_step": el64 / args.steps * 1e3,
                     "roofline": roofline(prof64, False, peaks), "kernel_shares": shares64},
            "mixed_vs_fp64_error": err,
            "ensemble": ens,
            "c4_sample": c4,
            "surrogate": sur,
            "paper_workload": paper,
            "apply_gbs": apply_gbs,
            "jacobi_sweeps_per_svd": prof["svd"].get("sweeps", 0) / max(1, prof["svd"].get("count", 0)),
            "cpu_baseline": cpu,
            "e2e": {"value": replica_rate(k_e2e, e2e_s, world), "unit": "steps/s",
                    "h2d_bytes_per_step": int(nd * 8), "d2h_bytes_per_step": int(out_bytes)},
            "gpu_launches": int(sum(v["launches"] for v in prof.values() if isinstance(v, dict))),
            "clocks": clocks.summary(),
        }
    return result


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error-check", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--c4-count", type=int, default=4,
                    help="instances of the C4 ensemble generator stepped alone and together (0: skip)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --qr-method for every shape instead of the per-shape autotuned configuration")
    ap.add_argument("--qr-method", choices=["tensor", "doublefloat"], default="tensor",
                    help="how the mixed arm factors its tall flattenings (hopf_set_qr_method)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
