"""Run a Monte Carlo walk until a target relative statistical error is reached.

Sec. IV reports the wall time needed to reach a given relative statistical
uncertainty sigma-bar_N / |I_N| (Figs. 3-4).  This driver measures it outright
rather than extrapolating: it runs the walk in chunks of production steps,
reads the blocked statistics (N_b = 100, Eq. uncertainty) after each chunk,
and stops once sigma-bar / |I_N| <= target (after at least `min_blocks`
blocks), reporting the device time of the production steps (CUDA events on
the context's stream) and the wall time of the whole loop.

Usage (one GPU):
    python -m paper_2203_05632_gb300.run_to_target --system tiny --soft --m 512 --n-tau 2
"""
from __future__ import annotations

import argparse
import json
import time


def run(system_name="tiny", soft=True, m=512, n_tau=2, precision="mixed", target=1e-3, chunk=50000,
        max_steps=20_000_000, burn=500, seed=5632, min_blocks=100):
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic

    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[precision]
    system = synthetic.make_system(system_name, soft=soft)
    ctx = pkg.Context(system, m, n_tau, prec)
    ctx.set_walkers(None, seed, burn)
    st = ctx.stream
    device_ms = 0.0
    trace = []
    t0 = time.perf_counter()
    res = None
    while True:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_steps_async(chunk, seed)
        e1.record(st)
        st.synchronize()
        device_ms += e0.elapsed_time(e1)
        res = ctx.run_steps(0, seed)  # statistics only
        rel = res["error"] / abs(res["energy"]) if res["energy"] else float("inf")
        trace.append({"steps": res["steps"], "energy": res["energy"], "sigma_bar": res["error"], "relative": rel})
        if (res["n_blocks"] >= min_blocks and rel <= target) or res["steps"] >= max_steps:
            break
    wall = time.perf_counter() - t0
    ctx.close()
    return {"system": system_name + (" (soft)" if soft else ""), "m": m, "n_tau": n_tau, "precision": precision,
            "target": target, "reached": trace[-1]["relative"] <= target, "steps": res["steps"],
            "energy": res["energy"], "sigma_bar": res["error"], "relative_error": trace[-1]["relative"],
            "device_s": device_ms / 1e3, "wall_s": wall, "trace": trace}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--system", default="tiny")
    ap.add_argument("--soft", action="store_true")
    ap.add_argument("--m", type=int, default=512)
    ap.add_argument("--n-tau", type=int, default=2)
    ap.add_argument("--precision", choices=["mixed", "tf32", "fp64"], default="mixed")
    ap.add_argument("--target", type=float, default=1e-3)
    ap.add_argument("--chunk", type=int, default=50000)
    ap.add_argument("--max-steps", type=int, default=20_000_000)
    args = ap.parse_args()
    out = run(args.system, args.soft, args.m, args.n_tau, args.precision, args.target, args.chunk, args.max_steps)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
