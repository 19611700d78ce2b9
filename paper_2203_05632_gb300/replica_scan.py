"""Independent replicas sharing one GPU: aggregate throughput and the combined result.

The paper's parallel scheme (Sec. III, end) runs independent Monte Carlo
integrations with distinct seeds and combines them by a weighted average;
its Fig. 5 shows the resulting strong scaling over processors.  On one GB300
the same scheme applies to R contexts, each on its own CUDA stream: a small-m
replica cannot fill 152 SMs, and R of them side by side can.  For each (m, R)
this driver runs R replicas for `steps` steps each (steps issued round-robin
so the streams overlap), and reports the aggregate pair-pair samples/s, the
speed-up over one replica, and the inverse-variance combination of the R
results (replicas.combine), whose sigma-bar falls as 1/sqrt(R) for
independent replicas.

Usage (one GPU):  python -m paper_2203_05632_gb300.replica_scan --m 128 512 --replicas 1 2 4 8
"""
from __future__ import annotations

import argparse
import json
import time


def run(ms, rs, system_name="medium", n_tau=4, precision="mixed", steps=300, burn=100, seed=5632):
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic
    from paper_2203_05632_gb300 import replicas

    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[precision]
    system = synthetic.make_system(system_name)
    rows = []
    for m in ms:
        base_rate = None
        for R in rs:
            ctxs = []
            for k in range(R):
                st = torch.cuda.Stream()
                ctx = pkg.Context(system, m, n_tau, prec, stream=st)
                ctx.set_walkers(None, seed + 7919 * k, burn)
                ctx.run_steps(2, seed + 7919 * k)
                ctxs.append(ctx)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                for k, ctx in enumerate(ctxs):
                    ctx.run_steps_async(1, seed + 7919 * k)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            results = [ctx.run_steps(0, seed + 7919 * k) for k, ctx in enumerate(ctxs)]
            for ctx in ctxs:
                ctx.close()
            del ctxs
            torch.cuda.empty_cache()
            comb = replicas.combine([{"energy": r["energy"], "error": r["error"]} if r["n_blocks"] >= 2 else None
                                     for r in results])
            rate = R * steps * m * (m - 1) // 2 * n_tau / wall
            base_rate = base_rate or rate
            rows.append({"m": m, "replicas": R, "steps_each": steps, "wall_s": wall, "samples_per_s": rate,
                         "speedup": rate / base_rate, "combined": comb})
    return {"system": system_name, "n_tau": n_tau, "precision": precision, "rows": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--m", type=int, nargs="+", default=[128, 512])
    ap.add_argument("--replicas", type=int, nargs="+", default=[1, 2, 4, 8])
    ap.add_argument("--precision", choices=["mixed", "tf32", "fp64"], default="mixed")
    ap.add_argument("--steps", type=int, default=300)
    args = ap.parse_args()
    print(json.dumps(run(args.m, args.replicas, precision=args.precision, steps=args.steps)))


if __name__ == "__main__":
    main()
