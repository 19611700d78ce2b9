"""Weight-function scan: stability of sigma-bar sqrt(N) for candidate g parameters.

The weight function g of Eq. basisSet has two s Gaussians per centre whose
parameters (c1, zeta1, c2, zeta2) Table 1 gives for H, O, Cu, Ag and Au only.
For other nuclear charges they are a choice, and it decides whether the
estimator of Eq. redundant has a finite variance in practice: where the
occupied density is much more compact than g, rare walkers in the cores carry
huge quotients and sigma-bar_N (Eq. uncertainty) does not settle as 1/sqrt(N).

For each candidate this runs independent walks of the workload's launch (m
walker pairs, n_tau times, split BF16 x3 by default) and prints, after every
segment, N, I_N, sigma-bar_N and sigma-bar_N sqrt(N) (constant for a
finite-variance estimator), plus the Metropolis acceptance.

  python -m paper_2203_05632_gb300.wscan --system medium \\
      --candidate '{"50": [0.1, 0.1, 0.8, 0.6], "17": [0.8, 0.2, 1.0, 0.4]}' ...
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--system", default="medium")
    ap.add_argument("--candidate", action="append", default=[],
                    help='JSON {"Z": [c1, zeta1, c2, zeta2], ...}; repeat for several')
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n-tau", type=int, default=4)
    ap.add_argument("--segments", type=int, default=4)
    ap.add_argument("--segment-steps", type=int, default=10000)
    ap.add_argument("--burn-in", type=int, default=2000)
    ap.add_argument("--seeds", type=int, nargs="+", default=[7001, 7002])
    ap.add_argument("--precision", choices=["mixed", "tf32", "fp64"], default="mixed")
    args = ap.parse_args()

    import paper_2203_05632_gb300 as pkg
    import synthetic

    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[args.precision]
    cands = args.candidate or ["{}"]
    for cand in cands:
        w = {int(k): tuple(float(x) for x in v) for k, v in json.loads(cand).items()}
        system = synthetic.make_system(args.system, weights=w or None)
        for seed in args.seeds:
            ctx = pkg.Context(system, args.m, args.n_tau, prec)
            t0 = time.perf_counter()
            ctx.set_walkers(None, seed, args.burn_in)
            rows = []
            for k in range(args.segments):
                res = ctx.run_steps(args.segment_steps, seed)
                n = res["steps"]
                rows.append({"steps": n, "energy": res["energy"], "sigma_bar": res["error"],
                             "sigma_bar_sqrtN": res["error"] * n ** 0.5, "accept": res["accept_rate"]})
            _, delta = ctx.get_walkers()
            ctx.close()
            print(json.dumps({"weights": {str(k): v for k, v in w.items()}, "seed": seed, "m": args.m,
                              "n_tau": args.n_tau, "delta": delta, "seconds": time.perf_counter() - t0,
                              "segments": rows}), flush=True)


if __name__ == "__main__":
    main()
