"""Forward and backward replay time of the FP64 adjoint on the adjoint workload.

The adjoint system (Z = 50 + 2 x Z = 17, n_L = 120, 24 occupied / 120 virtual
spinors) with m walker pairs and one imaginary time per step: `steps` seeded
replay steps through `mcmp2_eval_fixed` (forward) and `mcmp2_backward`
(energy, dE/d eps and dE/dC under the same samples), after one warm-up call,
timed on the host around the calls.  Also the command a profiler wraps to
capture the adjoint kernels on a small case.

Usage (one GPU):  python -m paper_2203_05632_gb300.adjoint_time --m 256 --steps 1
"""
from __future__ import annotations

import argparse
import json
import time


def run(m=512, steps=4, seed=11):
    import paper_2203_05632_gb300 as pkg
    import synthetic

    adj = synthetic.make_system("adjoint")
    lam = 2.0 * (adj.eps[adj.n_occ:].min() - adj.eps[:adj.n_occ].max())
    ctx = pkg.Context(adj, m, 1, pkg.MCMP2_FP64)
    r = synthetic.walker_positions(adj.centres, steps, m, seed=seed)
    tau = synthetic.imaginary_times(lam, steps, 1, seed=seed + 1)
    ctx.eval_fixed(r, tau)  # warm-up
    t0 = time.perf_counter()
    ctx.eval_fixed(r, tau)
    t1 = time.perf_counter()
    energy, _, _ = ctx.backward(r, tau)
    t2 = time.perf_counter()
    ctx.close()
    return {"m": m, "steps": steps, "forward_ms_per_step": 1e3 * (t1 - t0) / steps,
            "backward_ms_per_step": 1e3 * (t2 - t1) / steps, "energy": energy}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--m", type=int, default=512)
    ap.add_argument("--steps", type=int, default=4)
    args = ap.parse_args(argv)
    print(json.dumps(run(args.m, args.steps)))


if __name__ == "__main__":
    main()
