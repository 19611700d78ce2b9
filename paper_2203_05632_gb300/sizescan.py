"""Size-scaling series: cost of the Monte Carlo step and of a target accuracy vs system size.

The paper observes (Sec. IV) that the cost per MC step is quadratic in the
number of electrons or basis functions at its walker count, and that the
wall time to a fixed relative statistical error grows roughly quadratically
(at most cubically) for compact heavy-element clusters.  This driver runs the
analogous series on synthetic clusters of n units (one Z=80 centre plus two
Z=17 centres; 110 Cartesian Gaussians, 40 occupied and 180 virtual spinors
per unit) and reports, per n, the device time per step, the pair-pair sample
rate, the blocked statistics of a fixed-length walk, the extrapolated time to
a relative error (sigma-bar / |I_N|), and log-log fits of both against the
electron count (one electron per occupied spinor) and the basis size.

Usage (one GPU):  python -m paper_2203_05632_gb300.sizescan --units 1 2 4 8
"""
from __future__ import annotations

import argparse
import json
import math
import time


def run(units, m=4096, n_tau=8, burn=200, steps=400, timed=20, precision="mixed", seed=2203, target=1e-3,
        soft=False):
    import numpy as np
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic

    prec = pkg.MCMP2_MIXED if precision == "mixed" else pkg.MCMP2_FP64
    rows = []
    for n in units:
        system = synthetic.make_system("size", seed=seed, n_units=n, soft=soft)
        ctx = pkg.Context(system, m, n_tau, prec)
        ctx.set_walkers(None, seed + n, burn)
        ctx.run_steps(3, seed + n)
        st = ctx.stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.run_steps_async(timed, seed + n)
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / timed
        t0 = time.perf_counter()
        res = ctx.run_steps(steps, seed + n)
        wall = time.perf_counter() - t0
        samples = m * (m - 1) // 2 * n_tau
        row = {
            "units": n, "n_electrons": system.n_occ, "n_basis": system.n_l, "n_spinors": system.n_orb,
            "ms_per_step": ms, "pair_pair_samples_per_s": samples / (ms / 1e3),
            "steps": res["steps"], "blocks": res["n_blocks"], "energy": res["energy"], "sigma_bar": res["error"],
            "walk_wall_s": wall,
        }
        if res["n_blocks"] >= 2 and res["energy"] != 0.0:
            rel = res["error"] / abs(res["energy"])
            n_req = res["steps"] * (rel / target) ** 2
            row.update(relative_error=rel, steps_to_target=n_req, time_to_target_s=n_req * ms / 1e3)
        rows.append(row)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()

    def fit(key, xkey):
        pts = [(math.log(r[xkey]), math.log(r[key])) for r in rows if r.get(key, 0) > 0]
        if len(pts) < 2:
            return None
        x = np.array([p[0] for p in pts])
        y = np.array([p[1] for p in pts])
        slope, _ = np.polyfit(x, y, 1)
        return float(slope)

    fits = {
        "step_cost_vs_electrons": fit("ms_per_step", "n_electrons"),
        "step_cost_vs_basis": fit("ms_per_step", "n_basis"),
        "time_to_target_vs_electrons": fit("time_to_target_s", "n_electrons"),
        "time_to_target_vs_basis": fit("time_to_target_s", "n_basis"),
    }
    return {"m": m, "n_tau": n_tau, "precision": precision, "soft": soft, "target_relative_error": target,
            "rows": rows, "exponents": fits}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--units", type=int, nargs="+", default=[1, 2, 4, 8])
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--n-tau", type=int, default=8)
    ap.add_argument("--burn", type=int, default=200)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--soft", action="store_true",
                    help="soft units (exponents and energies inside the weight function's reach): finite variance")
    args = ap.parse_args()
    out = run(args.units, m=args.m, n_tau=args.n_tau, burn=args.burn, steps=args.steps, precision=args.precision,
              soft=args.soft)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
