#!/usr/bin/env python
"""Throughput of the Monte Carlo four-component MP2 step on one GB300 per rank.

Workload (medium system): 6 centres (four Z=50, two Z=17), n_L = 300 Cartesian
Gaussians (600 kinetically balanced small components), 80 occupied / 400
virtual Kramers-paired spinors, m = 1024 electron-pair walkers, 4 imaginary
times per step; synthetic seeded inputs.  One step = Metropolis move, basis
values, spinors, times, propagator blocks and traced products over all
mC2 = 523,776 pairs of walker pairs for each time, and the blocking update.

metric: pair-pair samples per second (C(m,2) x n_tau per step), whole job
over all ranks; ranks are independent replicas with their own seeds (the
method's own parallel scheme: no communication in the step).

``--impl reference`` times the oracle (plain FP64 CPU restatement) on this
host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

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

METRIC = "pair-pair samples/s and time to 0.1% rel. error: mixed-prec vs FP64 on 1 GB300"
UNIT = "pair-pair samples/s"
M, N_TAU = 1024, 4
WORKLOAD = ("medium: 6 centres (4 x Z=50, 2 x Z=17), n_L=300 (+600 small), 80 occ / 400 vir spinors, "
            "m=1024 walker pairs, 4 tau per step")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_NOMINAL_TFLOPS = 1.25  # GB300 CUDA-core FP64 (no FP64 tensor path on this part)
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate
# DRAM bytes (read + write) of one contraction launch at m = 1024, 4 tau, keyed
# by (form, spinor components), from the ncu captures summarised in
# profiles/pairs_mixed_{bf16x3,tf32,bf16x3_2c}_medium_m1024.md (the kernels as
# they stand; None where no capture of the current kernel exists).
PAIRS_TRAFFIC_BYTES = {("mixed", 4): 299.6e6, ("tf32", 4): 297.2e6, ("mixed", 2): 137.5e6}


def flops_per_sample(n_occ, n_vir, n_comp=4):
    """Algorithmic flops of one pair-of-pairs sample: the six n_comp x n_comp complex
    propagator blocks the trace form needs (two G- over n_occ, four G+ over n_vir),
    8 flops per complex multiply-add."""
    nn = n_comp * n_comp
    return 8 * (2 * nn * n_occ + 4 * nn * n_vir)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.rows = []
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_oracle_rate(system, m_sample, n_tau, seed=1, steps=1, n_threads=None, interaction=0):
    """Pair-pair samples/s of the oracle on this host's cores (bounded sample)."""
    import oracle
    import synthetic
    orc = oracle.Oracle(system, n_threads=n_threads, interaction=interaction)
    r = synthetic.walker_positions(system.centres, steps, m_sample, seed=seed)
    tau = synthetic.imaginary_times(orc.lam(), steps, n_tau, seed=seed + 1)
    t0 = time.perf_counter()
    orc.eval_steps(r, tau)
    dt = time.perf_counter() - t0
    samples = steps * m_sample * (m_sample - 1) // 2 * n_tau
    return samples / dt, dt, samples, orc.n_threads


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import synthetic
    system = synthetic.make_system("medium")
    rate0, _, _, cores = cpu_oracle_rate(system, 32, N_TAU)
    budget = 100.0  # seconds for warm-up plus timed steps
    per_step_samples = rate0 * budget / max(1, args.steps + args.warmup)
    m_s = int(max(8, min(M, (1 + math.sqrt(1 + 8 * per_step_samples / N_TAU)) / 2)))
    for w in range(args.warmup):
        cpu_oracle_rate(system, m_s, N_TAU, seed=100 + w)
    total_t, total_n = 0.0, 0
    for k in range(args.steps):
        _, dt, n, cores = cpu_oracle_rate(system, m_s, N_TAU, seed=200 + k)
        total_t += dt
        total_n += n
    value = total_n / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": f"one step of m={m_s} walker pairs x {N_TAU} tau"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of m={m_s} walker pairs x {N_TAU} tau of the medium system"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_steps(ctx, torch, steps, seed, flush):
    """Device time of `steps` steps (CUDA events on the context's stream), L2 flushed between steps."""
    st = ctx.stream
    total = 0.0
    for _ in range(steps):
        with torch.cuda.stream(st):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_steps_async(1, seed)
        e1.record(st)
        st.synchronize()
        total += e0.elapsed_time(e1)
    return total


def issued_per_algorithmic(n_occ, n_vir, products, n_comp=4):
    """Tensor flops the contraction issues per algorithmic flop: every 128 x 128
    tile computes all four electron blocks of G- (the trace form needs two) and
    G+ (it needs all four), `products` split products per real product."""
    issued = products * 8 * (2 * n_comp) ** 2 * (n_occ + n_vir)
    return issued / flops_per_sample(n_occ, n_vir, n_comp)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "tf32", "fp64"], default="mixed")
    ap.add_argument("--interaction", choices=["coulomb", "gaunt", "breit"], default="coulomb",
                    help="two-electron operator of Sec. II (Gaunt / Breit terms: four-component spinors)")
    ap.add_argument("--components", type=int, choices=[4, 2], default=4,
                    help="spinor components: 4, or 2 for the two-component variant")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 form beside the mixed run")
    ap.add_argument("--tf32-steps", type=int, default=200, help="timed steps of the TF32 form beside the mixed run")
    ap.add_argument("--breit-steps", type=int, default=100,
                    help="timed steps of the same form with the full Breit interaction beside the Coulomb run")
    ap.add_argument("--stat-steps", type=int, default=10000, help="steps of the run that estimates sigma for time-to-0.1%%")
    ap.add_argument("--cpu-sample-m", type=int, default=1024)
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--m", type=int, default=M, help="walker pairs (the workload is m=1024; smaller m only "
                                                     "for sized profiler captures)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    two_c = args.components == 2
    system = synthetic.make_system("medium", two_component=two_c)
    peaks, peak_kind = load_peaks()
    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[args.precision]
    inter = {"coulomb": pkg.MCMP2_COULOMB, "gaunt": pkg.MCMP2_GAUNT, "breit": pkg.MCMP2_BREIT}[args.interaction]
    if inter != pkg.MCMP2_COULOMB and two_c:
        ap.error("the Gaunt / Breit terms need the small components (four-component spinors)")
    seed = 5632 + rank
    m_run = args.m
    samples_per_step = m_run * (m_run - 1) // 2 * N_TAU
    flop_unit = flops_per_sample(system.n_occ, system.n_vir, args.components)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def make_ctx(p):
        ctx = pkg.Context(system, m_run, N_TAU, p, device=local)
        if inter != pkg.MCMP2_COULOMB:
            ctx.set_interaction(inter)
        r0 = synthetic.walker_positions(system.centres, 1, m_run, seed=seed)[0]
        ctx.set_walkers(r0, seed, 200)
        return ctx

    ctx = make_ctx(prec)
    ctx.run_steps(args.warmup, seed)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile(1)
    dev_ms = time_steps(ctx, torch, args.steps, seed, flush)
    prof = ctx.profile(0)
    ctx.profile(2)  # timing off again
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    t_max = dev_ms
    if dist:
        t = torch.tensor([dev_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = world * args.steps * samples_per_step / (t_max / 1e3)
    ms_per_step = t_max / args.steps
    pair_ms = prof["pair_ms"] / max(1, prof["pair_launches"])
    achieved = flop_unit * samples_per_step / max(1, prof["pair_launches"] // args.steps) / (pair_ms / 1e3) / 1e12

    # End to end through the public replay call: host positions and times from
    # pinned memory copied in, the step estimate copied out, every step.
    e2e_steps = max(3, min(args.steps, 50))
    r_host = torch.from_numpy(synthetic.walker_positions(system.centres, e2e_steps, m_run, seed=seed + 7)).pin_memory()
    lam = 2.0 * (system.eps[system.n_occ:].min() - system.eps[:system.n_occ].max())
    t_host = torch.from_numpy(synthetic.imaginary_times(lam, e2e_steps, N_TAU, seed=seed + 8)).pin_memory()
    o_host = torch.zeros(e2e_steps, dtype=torch.float64).pin_memory()
    ctx.eval_fixed_ptr(1, r_host.data_ptr(), t_host.data_ptr(), o_host.data_ptr())  # warm
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx.eval_fixed_ptr(1, r_host[k].data_ptr(), t_host[k].data_ptr(), o_host[k].data_ptr())
    e2e_s = time.perf_counter() - t0
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * e2e_steps * samples_per_step / float(e2e_t.item())

    # Statistics for the time to 0.1 % relative error (sigma from blocking).
    stat = None
    if args.stat_steps > 0 and rank == 0:
        sctx = make_ctx(prec)
        res = sctx.run_steps(args.stat_steps, seed + 1000)
        if res["n_blocks"] >= 2 and res["energy"] != 0.0:
            n_req = res["steps"] * (res["error"] / (1e-3 * abs(res["energy"]))) ** 2
            stat = {"steps": res["steps"], "blocks": res["n_blocks"], "energy": res["energy"],
                    "sigma_bar": res["error"], "steps_to_0.1pct": n_req,
                    "time_to_0.1pct_s": n_req * ms_per_step / 1e3, "kind": "extrapolated from the run's sigma"}
        sctx.close()

    # The soft medium system (the workload's sizes with exponents and energies inside
    # the weight function's reach) has a finite variance: its time to 0.1 % at the
    # workload's m and n_tau, extrapolated from a run of the same length.
    stat_soft_medium = None
    if args.stat_steps > 0 and rank == 0:
        softm = synthetic.make_system("medium", soft=True, two_component=two_c)
        mctx = pkg.Context(softm, m_run, N_TAU, prec, device=local)
        if inter != pkg.MCMP2_COULOMB:
            mctx.set_interaction(inter)
        mctx.set_walkers(None, seed + 3000, 1000)
        res = mctx.run_steps(args.stat_steps, seed + 3000)
        if res["n_blocks"] >= 2 and res["energy"] != 0.0:
            n_req = res["steps"] * (res["error"] / (1e-3 * abs(res["energy"]))) ** 2
            stat_soft_medium = {"system": "soft medium (the medium sizes, even-tempered ratio 1.4, soft energies)",
                                "m": m_run, "n_tau": N_TAU, "steps": res["steps"], "blocks": res["n_blocks"],
                                "energy": res["energy"], "sigma_bar": res["error"], "steps_to_0.1pct": n_req,
                                "time_to_0.1pct_s": n_req * ms_per_step / 1e3,
                                "kind": "extrapolated from the run's sigma"}
        mctx.close()

    # The medium synthetic system's estimator is heavy-tailed (its sigma-bar is not
    # stable between runs); the soft tiny system has a finite variance, and m = 512
    # minimises sigma_step^2 t_step there (mscan), so its time to 0.1 % is reported
    # beside, extrapolated from a 20,000-step run (200 blocks).
    stat_soft = None
    if args.stat_steps > 0 and rank == 0:
        soft = synthetic.make_system("tiny", soft=True)
        qctx = pkg.Context(soft, 512, 2, prec, device=local)
        if inter != pkg.MCMP2_COULOMB:
            qctx.set_interaction(inter)
        qctx.set_walkers(None, seed + 2000, 500)
        qctx.run_steps(3, seed + 2000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(qctx.stream)
        qctx.run_steps_async(50, seed + 2000)
        e1.record(qctx.stream)
        qctx.stream.synchronize()
        t_soft = e0.elapsed_time(e1) / 50 / 1e3
        res = qctx.run_steps(20000, seed + 2000)
        if res["n_blocks"] >= 2 and res["energy"] != 0.0:
            n_req = res["steps"] * (res["error"] / (1e-3 * abs(res["energy"]))) ** 2
            stat_soft = {"system": "soft tiny (Zn + H, n_L = 20, 4 occ / 16 vir)", "m": 512, "n_tau": 2,
                         "steps": res["steps"], "blocks": res["n_blocks"], "energy": res["energy"],
                         "sigma_bar": res["error"], "ms_per_step": t_soft * 1e3, "steps_to_0.1pct": n_req,
                         "time_to_0.1pct_s": n_req * t_soft, "kind": "extrapolated from the run's sigma"}
        qctx.close()

    fp64 = None
    if prec != pkg.MCMP2_FP64 and args.fp64_steps > 0:
        fctx = make_ctx(pkg.MCMP2_FP64)
        fctx.run_steps(1, seed)
        fctx.profile(1)
        f_ms = time_steps(fctx, torch, args.fp64_steps, seed, flush)
        fp = fctx.profile(0)
        fctx.profile(2)
        f_pair = fp["pair_ms"] / max(1, fp["pair_launches"])
        fp64 = {"value": args.fp64_steps * samples_per_step / (f_ms / 1e3), "ms_per_step": f_ms / args.fp64_steps,
                "pair_kernel_ms": f_pair,
                "achieved_tflops": flop_unit * samples_per_step / (f_pair / 1e3) / 1e12}
        fctx.close()

    tf32 = None
    if prec == pkg.MCMP2_MIXED and args.tf32_steps > 0:
        tctx = make_ctx(pkg.MCMP2_TF32)
        tctx.run_steps(3, seed)
        tctx.profile(1)
        t_ms = time_steps(tctx, torch, args.tf32_steps, seed, flush)
        tp = tctx.profile(0)
        tctx.profile(2)
        t_pair = tp["pair_ms"] / max(1, tp["pair_launches"])
        t_ach = flop_unit * samples_per_step / (t_pair / 1e3) / 1e12
        t_peak = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]) * TF32_OVER_BF16
        tf32 = {"value": args.tf32_steps * samples_per_step / (t_ms / 1e3), "ms_per_step": t_ms / args.tf32_steps,
                "pair_kernel_ms": t_pair, "achieved_tflops": t_ach,
                "roofline_frac": t_ach / t_peak, "peak_tflops": t_peak,
                "issued_frac": t_ach * issued_per_algorithmic(system.n_occ, system.n_vir, 1, args.components) / t_peak,
                "peak_kind": f"{peak_kind} bf16 sustained x nominal tf32/bf16 ratio (1.1/2.25)"}
        tctx.close()

    if prec == pkg.MCMP2_MIXED:
        peak = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
        issued = achieved * issued_per_algorithmic(system.n_occ, system.n_vir, 3, args.components)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": PAIRS_TRAFFIC_BYTES.get(("mixed", args.components)) if m_run == M and inter == 0 else None,
                "peak_kind": f"{peak_kind} bf16 sustained",
                "issued": {"tflops": issued, "frac": issued / peak,
                           "note": "BF16 tensor work actually issued: 3 split products, full 128 x 128 tiles"}}
    elif prec == pkg.MCMP2_TF32:
        peak = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]) * TF32_OVER_BF16
        issued = achieved * issued_per_algorithmic(system.n_occ, system.n_vir, 1, args.components)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": PAIRS_TRAFFIC_BYTES.get(("tf32", args.components)) if m_run == M and inter == 0 else None,
                "peak_kind": f"{peak_kind} bf16 sustained x nominal tf32/bf16 ratio (1.1/2.25)",
                "issued": {"tflops": issued, "frac": issued / peak,
                           "note": "TF32 tensor work actually issued: full 128 x 128 tiles"}}
    else:
        peak = FP64_NOMINAL_TFLOPS
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": "nominal FP64 CUDA-core rate"}

    # The same form with the Breit terms of Sec. II in the trace epilogue (four-component
    # spinors): the contraction's extra cost over the Coulomb operator.
    breit = None
    if prec != pkg.MCMP2_FP64 and inter == pkg.MCMP2_COULOMB and not two_c and args.breit_steps > 0:
        bctx = pkg.Context(system, m_run, N_TAU, prec, device=local)
        bctx.set_interaction(pkg.MCMP2_BREIT)
        bctx.set_walkers(synthetic.walker_positions(system.centres, 1, m_run, seed=seed)[0], seed, 200)
        bctx.run_steps(3, seed)
        bctx.profile(1)
        b_ms = time_steps(bctx, torch, args.breit_steps, seed, flush)
        bp_ = bctx.profile(0)
        bctx.profile(2)
        breit = {"interaction": "breit (Coulomb + Gaunt + gauge)", "value": args.breit_steps * samples_per_step / (b_ms / 1e3),
                 "ms_per_step": b_ms / args.breit_steps,
                 "pair_kernel_ms": bp_["pair_ms"] / max(1, bp_["pair_launches"])}
        bctx.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, dt, n, cores = cpu_oracle_rate(system, args.cpu_sample_m, N_TAU, steps=args.cpu_sample_steps,
                                             interaction=inter)
        rate1, dt1, n1, _ = cpu_oracle_rate(system, 128 if inter == 0 else 32, N_TAU, seed=3, n_threads=1,
                                            interaction=inter)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample_steps} step(s) of m={args.cpu_sample_m} walker pairs x {N_TAU} tau of the "
                         f"medium system ({n} pair-pair samples, {dt:.1f} s)",
               "one_core": {"value": rate1, "unit": UNIT, "cores": 1,
                            "sample": f"one step of m={128 if inter == 0 else 32} x {N_TAU} tau ({n1} samples, {dt1:.1f} s)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {pkg.MCMP2_MIXED: "bf16x3", pkg.MCMP2_TF32: "tf32"}.get(prec, "f64"),
            "data": "synthetic",
            "config": {"workload": (WORKLOAD if m_run == M else WORKLOAD.replace("m=1024", f"m={m_run}"))
                       + (", two-component spinors (large basis only)" if two_c else ""),
                       "precision": args.precision, "interaction": args.interaction,
                       "l2": "flushed between timed steps",
                       "parallelism": f"{world} independent replicas"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": m_run * 6 * 8 + N_TAU * 8,
                    "d2h_bytes_per_step": 8, "call": "mcmp2_eval_fixed, pinned host buffers"},
            "gpu_launches": prof["launches"],
            "roofline": roof,
            "time_to_0.1pct": stat,
            "time_to_0.1pct_soft_medium": stat_soft_medium,
            "time_to_0.1pct_soft_tiny": stat_soft,
            "fp64_form": fp64,
            "tf32_form": tf32,
            "breit_form": breit,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
