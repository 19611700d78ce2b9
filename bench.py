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
PAIRS_TRAFFIC_BYTES = {("mixed", 4): 216.7e6, ("tf32", 4): 215.8e6, ("mixed", 2): 107.9e6}


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
    """nvidia-smi clocks and throttle reasons sampled every 20 ms during the timed region
    (start() returns once the first sample has arrived, so sampling covers the region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.rows = []
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.rows and self.proc.poll() is None and time.time() - t0 < 5.0:
            time.sleep(0.01)

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


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1,
                    help="ranks (one per GPU); without a launcher's environment, N > 1 starts N local ranks")
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
    ap.add_argument("--stat-steps", type=int, default=40000,
                    help="steps of each rank's walk that estimates sigma-bar for the time to 0.1%% (its replica result)")
    ap.add_argument("--adjoint-steps", type=int, default=4, help="replay steps of the adjoint timing")
    ap.add_argument("--sustained-steps", type=int, default=2000,
                    help="back-to-back steps (no flush, rank 0) that give the long-run rate under the power limit")
    ap.add_argument("--peak-seconds", type=float, default=2.0,
                    help="sustained part of the live TF32 / FP64 peak measurement (0: skip it)")
    ap.add_argument("--cpu-sample-m", type=int, default=1024)
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--m", type=int, default=M, help="walker pairs (the workload is m=1024; smaller m only "
                                                     "for sized profiler captures)")
    return ap.parse_args(argv)


def main(argv=None):
    args = parse_args(argv)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # Not started by a launcher: start the ranks here, one process per GPU.
        from paper_2203_05632_gb300 import replicas
        cmd = [sys.executable, os.path.abspath(__file__)] + list(sys.argv[1:] if argv is None else argv)
        codes = replicas.spawn_local(args.gpus, cmd)
        return 0 if all(c == 0 for c in codes) else 1
    if world != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but the launcher started {world} ranks", file=sys.stderr)
        return 2
    return run_ours(args, rank, world, local)


def run_ours(args, rank, world, local, work=None, backend="nccl"):
    """One rank: its replica's measurement (`work`, default measure_rank), then the
    max over ranks of the timed region, the combination of the replicas' results
    (inverse-variance weighted, Sec. III), and rank 0's JSON line."""
    import torch

    from paper_2203_05632_gb300 import replicas
    dist = None
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)

    def barrier():
        if dist:
            dist.barrier()

    res = (work or measure_rank)(args, rank, world, local, barrier)
    t_max, e2e_max = res["dev_ms"], res["e2e_s"]
    if dist:
        dev = torch.device("cuda", local) if backend == "nccl" else torch.device("cpu")
        t = torch.tensor([res["dev_ms"], res["e2e_s"]], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max, e2e_max = float(t[0]), float(t[1])
        combined, gathered = replicas.gather_and_combine(res["replica"])
    else:
        combined, gathered = replicas.combine([res["replica"]]), [res["replica"]]
    if rank == 0:
        print(json.dumps(assemble_line(args, world, res, t_max, e2e_max, combined, gathered)), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def assemble_line(args, world, res, t_max, e2e_max, combined, gathered):
    """Rank 0's JSON line: whole-job throughput over all ranks (each rank's fixed work,
    max-over-ranks time), end to end likewise, and the combined replica result."""
    spp = res["samples_per_step"]
    value = world * args.steps * spp / (t_max / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": res["dtype"], "data": "synthetic", "config": res["config"],
        "clocks": res["clocks"],
        "e2e": {"value": world * res["e2e_steps"] * spp / e2e_max, "unit": UNIT,
                "h2d_bytes_per_step": res["h2d_bytes_per_step"], "d2h_bytes_per_step": res["d2h_bytes_per_step"],
                "call": "mcmp2_eval_fixed, pinned host buffers"},
        "gpu_launches": res["gpu_launches"],
        "replicas": {"n": world, "combined": combined, "per_rank": gathered,
                     "note": "each rank's own walk (seed 5632 + rank), combined by inverse variance (Sec. III)"},
    }
    line.update(res.get("extras", {}))
    return line


def walk_stat(ctx, steps, seed, burn_in=1000, segments=4):
    """A walk of `steps` production steps in equal segments: I_N, sigma-bar_N and
    sigma-bar_N sqrt(N) after each (constant for a finite-variance estimator)."""
    ctx.set_walkers(None, seed, burn_in)
    seg = max(1, steps // segments)
    rows, res = [], None
    for _ in range(segments):
        res = ctx.run_steps(seg, seed)
        n = res["steps"]
        rows.append({"steps": n, "energy": res["energy"], "sigma_bar": res["error"],
                     "sigma_bar_sqrtN": res["error"] * math.sqrt(n)})
    return res, rows


def time_to_target(res, ms_per_step):
    """Steps and seconds to a relative sigma-bar of 0.1 % (Eq. uncertainty: sigma-bar ~ 1/sqrt(N))."""
    if not res or res["n_blocks"] < 2 or res["energy"] == 0.0:
        return None, None
    n_req = res["steps"] * (res["error"] / (1e-3 * abs(res["energy"]))) ** 2
    return n_req, n_req * ms_per_step / 1e3


def measure_rank(args, rank, world, local, barrier):
    """This rank's replica on its GPU: the timed steps, the end-to-end replay, the walk
    that gives the replica result, and (rank 0) the forms, scans and baselines beside."""
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    two_c = args.components == 2
    system = synthetic.make_system("medium", two_component=two_c)
    peaks, peak_kind = load_peaks()
    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[args.precision]
    inter = {"coulomb": pkg.MCMP2_COULOMB, "gaunt": pkg.MCMP2_GAUNT, "breit": pkg.MCMP2_BREIT}[args.interaction]
    if inter != pkg.MCMP2_COULOMB and two_c:
        raise SystemExit("the Gaunt / Breit terms need the small components (four-component spinors)")
    seed = 5632 + rank
    m_run = args.m
    samples_per_step = m_run * (m_run - 1) // 2 * N_TAU
    flop_unit = flops_per_sample(system.n_occ, system.n_vir, args.components)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def make_ctx(p, sysobj=system, m=m_run, n_tau=N_TAU):
        ctx = pkg.Context(sysobj, m, n_tau, p, device=local)
        if inter != pkg.MCMP2_COULOMB:
            ctx.set_interaction(inter)
        return ctx

    ctx = make_ctx(prec)
    ctx.set_walkers(synthetic.walker_positions(system.centres, 1, m_run, seed=seed)[0], seed, 200)
    ctx.run_steps(args.warmup, seed)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    # The timed steps replay the step graph exactly as run_steps does; a second pass
    # of the same length, whose graph holds events around the contraction, gives
    # the kernel's own time.
    dev_ms = time_steps(ctx, torch, args.steps, seed, flush)
    ctx.profile(1)
    time_steps(ctx, torch, args.steps, seed, flush)
    prof = ctx.profile(0)
    ctx.profile(2)  # timing off again
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_per_step = dev_ms / args.steps
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

    # The long-run rate: back-to-back replays of the step graph, no L2 flush and no
    # host gaps, as a production walk runs them; the board's power limit sets the clock.
    sustained = None
    if rank == 0 and args.sustained_steps > 0:
        sclk = ClockSampler(uuid)
        sclk.start()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        ctx.run_steps_async(args.sustained_steps, seed)
        e1.record(ctx.stream)
        ctx.stream.synchronize()
        s_ms = e0.elapsed_time(e1) / args.sustained_steps
        sustained = {"steps": args.sustained_steps, "ms_per_step": s_ms,
                     "value": samples_per_step / (s_ms / 1e3), "unit": UNIT, "clocks": sclk.stop(),
                     "note": "back-to-back steps, no L2 flush: the long-run rate under the power limit"}
    ctx.close()

    # This replica's result: a walk of the workload with its own seed (Eq. uncertainty).
    replica, stat = None, None
    if args.stat_steps > 0:
        sctx = make_ctx(prec)
        res, rows = walk_stat(sctx, args.stat_steps, seed + 1000)
        sctx.close()
        replica = {"energy": res["energy"], "error": res["error"], "steps": res["steps"], "rank": rank}
        n_req, t_req = time_to_target(res, ms_per_step)
        stat = {"system": "medium (the workload)", "m": m_run, "n_tau": N_TAU, "steps": res["steps"],
                "blocks": res["n_blocks"], "energy": res["energy"], "sigma_bar": res["error"],
                "segments": rows, "steps_to_0.1pct": n_req, "time_to_0.1pct_s": t_req,
                "kind": "extrapolated from the run's sigma-bar (sigma-bar sqrt(N) per segment beside it)"}

    extras = {}
    if rank == 0:
        # The soft tiny system (finite variance at a size the walk finishes outright; m = 512
        # minimises sigma_step^2 t_step there): its time to 0.1 %, extrapolated.
        stat_soft = None
        if args.stat_steps > 0:
            soft = synthetic.make_system("tiny", soft=True)
            qctx = make_ctx(prec, soft, 512, 2)
            qctx.set_walkers(None, seed + 2000, 500)
            qctx.run_steps(3, seed + 2000)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(qctx.stream)
            qctx.run_steps_async(50, seed + 2000)
            e1.record(qctx.stream)
            qctx.stream.synchronize()
            t_soft = e0.elapsed_time(e1) / 50
            res = qctx.run_steps(20000, seed + 2000)
            n_req, t_req = time_to_target(res, t_soft)
            stat_soft = {"system": "soft tiny (Zn + H, n_L = 20, 4 occ / 16 vir)", "m": 512, "n_tau": 2,
                         "steps": res["steps"], "blocks": res["n_blocks"], "energy": res["energy"],
                         "sigma_bar": res["error"], "ms_per_step": t_soft, "steps_to_0.1pct": n_req,
                         "time_to_0.1pct_s": t_req, "kind": "extrapolated from the run's sigma-bar"}
            qctx.close()

        def timed_form(p, steps, interaction=None):
            fctx = pkg.Context(system, m_run, N_TAU, p, device=local)
            fctx.set_interaction(inter if interaction is None else interaction)
            fctx.set_walkers(synthetic.walker_positions(system.centres, 1, m_run, seed=seed)[0], seed, 200)
            fctx.run_steps(3 if p != pkg.MCMP2_FP64 else 1, seed)
            f_ms = time_steps(fctx, torch, steps, seed, flush)
            fctx.profile(1)
            time_steps(fctx, torch, steps, seed, flush)
            fp = fctx.profile(0)
            fctx.close()
            f_pair = fp["pair_ms"] / max(1, fp["pair_launches"])
            return {"value": steps * samples_per_step / (f_ms / 1e3), "ms_per_step": f_ms / steps,
                    "pair_kernel_ms": f_pair, "achieved_tflops": flop_unit * samples_per_step / (f_pair / 1e3) / 1e12}

        fp64 = timed_form(pkg.MCMP2_FP64, args.fp64_steps) if prec != pkg.MCMP2_FP64 and args.fp64_steps > 0 else None
        tf32 = timed_form(pkg.MCMP2_TF32, args.tf32_steps) if prec == pkg.MCMP2_MIXED and args.tf32_steps > 0 else None
        breit = None
        if prec != pkg.MCMP2_FP64 and inter == pkg.MCMP2_COULOMB and not two_c and args.breit_steps > 0:
            breit = timed_form(prec, args.breit_steps, pkg.MCMP2_BREIT)
            breit["interaction"] = "breit (Coulomb + Gaunt + gauge)"
        if stat and fp64:
            # Both forms estimate the same walk's integrand (their per-step difference is far
            # below sigma), so the FP64 form needs the same number of steps.
            fp64["time_to_0.1pct_s"] = stat["steps_to_0.1pct"] * fp64["ms_per_step"] / 1e3 \
                if stat["steps_to_0.1pct"] else None
            fp64["time_kind"] = "steps to 0.1 % of the workload's walk x this form's step time"

        # Adjoint (dE/d eps, dE/dC under common random numbers) on its workload: 3 centres,
        # n_L = 120, 24 / 120 spinors, m = 512, 1 time per step, FP64.
        adjoint = None
        if args.adjoint_steps > 0 and not two_c:
            adj = synthetic.make_system("adjoint")
            actx = pkg.Context(adj, 512, 1, pkg.MCMP2_FP64, device=local)
            lam_a = 2.0 * (adj.eps[adj.n_occ:].min() - adj.eps[:adj.n_occ].max())
            ra = synthetic.walker_positions(adj.centres, args.adjoint_steps, 512, seed=seed + 11)
            ta = synthetic.imaginary_times(lam_a, args.adjoint_steps, 1, seed=seed + 12)
            actx.eval_fixed(ra[:1], ta[:1])
            actx.backward(ra[:1], ta[:1])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            actx.eval_fixed(ra, ta)
            t1 = time.perf_counter()
            actx.backward(ra, ta)
            t2 = time.perf_counter()
            actx.close()
            adjoint = {"workload": "adjoint: Z=50 + 2 x Z=17, n_L=120, 24 occ / 120 vir, m=512, 1 tau",
                       "forward_ms_per_step": 1e3 * (t1 - t0) / args.adjoint_steps,
                       "backward_ms_per_step": 1e3 * (t2 - t1) / args.adjoint_steps,
                       "ratio": (t2 - t1) / (t1 - t0), "steps": args.adjoint_steps,
                       "timing": "host clock around the replay calls (mcmp2_eval_fixed / mcmp2_backward)"}

        # Peaks the TF32 and FP64 rooflines divide by, measured on this GPU now.
        live = None
        if args.peak_seconds > 0:
            from paper_2203_05632_gb300 import peaks as peak_probe
            live = peak_probe.measure(args.peak_seconds, local)
        bf16_sust = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
        if live:
            tf32_peak, tf32_kind = live["tf32_tflops_sustained"], "measured live: cuBLAS TF32 matmul, sustained"
            fp64_peak, fp64_kind = live["fp64_fma_tflops"], "measured live: DFMA probe (probes/dfma.cu)"
        else:
            tf32_peak = bf16_sust * TF32_OVER_BF16
            tf32_kind = f"{peak_kind} bf16 sustained x nominal tf32/bf16 ratio (1.1/2.25)"
            fp64_peak, fp64_kind = FP64_NOMINAL_TFLOPS, "nominal FP64 CUDA-core rate"
        if tf32:
            tf32.update({"roofline_frac": tf32["achieved_tflops"] / tf32_peak, "peak_tflops": tf32_peak,
                         "issued_frac": tf32["achieved_tflops"] * issued_per_algorithmic(
                             system.n_occ, system.n_vir, 1, args.components) / tf32_peak, "peak_kind": tf32_kind})
        if fp64:
            fp64.update({"roofline_frac": fp64["achieved_tflops"] / fp64_peak, "peak_tflops": fp64_peak,
                         "peak_kind": fp64_kind})
        traffic = PAIRS_TRAFFIC_BYTES.get((args.precision, args.components)) if m_run == M and inter == 0 else None
        if prec == pkg.MCMP2_FP64:
            roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": None, "peak_kind": fp64_kind}
        else:
            products = 3 if prec == pkg.MCMP2_MIXED else 1
            peak = bf16_sust if prec == pkg.MCMP2_MIXED else tf32_peak
            kind = f"{peak_kind} bf16 sustained" if prec == pkg.MCMP2_MIXED else tf32_kind
            issued = achieved * issued_per_algorithmic(system.n_occ, system.n_vir, products, args.components)
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic, "peak_kind": kind,
                    "issued": {"tflops": issued, "frac": issued / peak,
                               "note": f"tensor work actually issued: {products} product(s) per real product, "
                                       "full 128 x 128 tiles"}}

        cpu = None
        if not args.no_cpu_baseline:
            rate, dt, n, cores = cpu_oracle_rate(system, args.cpu_sample_m, N_TAU, steps=args.cpu_sample_steps,
                                                 interaction=inter)
            m1 = 128 if inter == 0 else 32
            rate1, dt1, n1, _ = cpu_oracle_rate(system, m1, N_TAU, seed=3, n_threads=1, interaction=inter)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{args.cpu_sample_steps} step(s) of m={args.cpu_sample_m} walker pairs x {N_TAU} tau "
                             f"of the medium system ({n} pair-pair samples, {dt:.1f} s)",
                   "one_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                "sample": f"one step of m={m1} x {N_TAU} tau ({n1} samples, {dt1:.1f} s)"}}
        extras = {"roofline": roof, "time_to_0.1pct": stat, "time_to_0.1pct_soft_tiny": stat_soft,
                  "fp64_form": fp64, "tf32_form": tf32, "breit_form": breit, "adjoint": adjoint,
                  "peaks_live": live, "cpu_baseline": cpu, "sustained": sustained}

    workload = WORKLOAD if m_run == M else WORKLOAD.replace("m=1024", f"m={m_run}")
    return {
        "dev_ms": dev_ms, "e2e_s": e2e_s, "e2e_steps": e2e_steps, "samples_per_step": samples_per_step,
        "dtype": {pkg.MCMP2_MIXED: "bf16x3", pkg.MCMP2_TF32: "tf32"}.get(prec, "f64"),
        "config": {"workload": workload + (", two-component spinors (large basis only)" if two_c else ""),
                   "precision": args.precision, "interaction": args.interaction,
                   "l2": "flushed between timed steps", "parallelism": f"{world} independent replicas"},
        "clocks": clk, "gpu_launches": prof["launches"],
        "h2d_bytes_per_step": m_run * 6 * 8 + N_TAU * 8, "d2h_bytes_per_step": 8,
        "replica": replica, "extras": extras,
    }


if __name__ == "__main__":
    sys.exit(main())
