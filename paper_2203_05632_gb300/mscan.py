"""Redundant-walker scan: statistical efficiency and cost of the step vs m.

Sec. III's redundant-walker scheme evaluates all mC2 pairs of the m walker
pairs each step, so the variance of a step estimate would fall as 1/mC2 if
the pairs of pairs were independent; they share walkers, so the gain over
one pair of pairs saturates (the paper observes an (m - 1)-fold speed-up that
levels off).  For each m this driver measures, on the device, the time per
step and the per-step standard deviation sigma_step = sigma-bar * sqrt(N)
from a blocked run, and reports
  * cost = sigma_step^2 * t_step, proportional to the time to any fixed
    relative error (smaller is better), and
  * the pair efficiency sigma_step^2(m) * mC2 / (sigma_step^2(m0) * m0C2),
    1 while the pairs of pairs act independently and growing once they do not.

Usage (one GPU):  python -m paper_2203_05632_gb300.mscan --m 64 128 256 512 1024 2048
"""
from __future__ import annotations

import argparse
import json
import math


def run(ms, system_name="medium", n_tau=4, precision="mixed", burn=300, steps=5000, budget_s=20.0, seed=2203,
        soft=False):
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic

    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[precision]
    system = synthetic.make_system(system_name, soft=soft)
    rows = []
    for m in ms:
        ctx = pkg.Context(system, m, n_tau, prec)
        ctx.set_walkers(None, seed + m, burn)
        ctx.run_steps(3, seed + m)
        st = ctx.stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_steps_async(20, seed + m)
        e1.record(st)
        st.synchronize()
        t_step = e0.elapsed_time(e1) / 20 / 1e3
        n = int(min(steps, max(1000, budget_s / t_step)))
        n -= n % 100
        res = ctx.run_steps(n, seed + m)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
        sigma_step = res["error"] * math.sqrt(res["n_blocks"] * 100)
        pairs = m * (m - 1) // 2 * n_tau
        rows.append({"m": m, "steps": res["n_blocks"] * 100, "blocks": res["n_blocks"], "t_step_s": t_step,
                     "samples_per_s": pairs / t_step, "energy": res["energy"], "sigma_bar": res["error"],
                     "sigma_step": sigma_step, "cost": sigma_step ** 2 * t_step,
                     "accept_rate": res["accept_rate"]})
    base = rows[0]
    b_pairs = base["m"] * (base["m"] - 1) // 2
    for r in rows:
        pairs = r["m"] * (r["m"] - 1) // 2
        r["pair_efficiency"] = r["sigma_step"] ** 2 * pairs / (base["sigma_step"] ** 2 * b_pairs)
        r["cost_relative"] = r["cost"] / base["cost"]
    best = min(rows, key=lambda r: r["cost"])
    return {"system": system_name + (" (soft)" if soft else ""), "n_tau": n_tau, "precision": precision,
            "rows": rows, "best_m": best["m"]}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--m", type=int, nargs="+", default=[64, 128, 256, 512, 1024, 2048])
    ap.add_argument("--system", default="medium")
    ap.add_argument("--soft", action="store_true")
    ap.add_argument("--n-tau", type=int, default=4)
    ap.add_argument("--precision", choices=["mixed", "tf32", "fp64"], default="mixed")
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--budget", type=float, default=20.0, help="seconds of walk per m (at least 1000 steps)")
    args = ap.parse_args()
    out = run(args.m, args.system, args.n_tau, args.precision, steps=args.steps, budget_s=args.budget,
              soft=args.soft)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
