"""Run a Monte Carlo walk until a target relative statistical error is reached.

Sec. IV reports the wall time needed to reach a given relative statistical
uncertainty sigma-bar_N / |I_N| (Figs. 3-4).  This driver measures it outright
rather than extrapolating: it runs the walk in chunks of production steps,
reads the blocked statistics (N_b = 100, Eq. uncertainty) after each chunk,
and stops once sigma-bar / |I_N| <= target (after at least `min_blocks`
blocks), reporting the device time of the production steps (CUDA events on
the context's stream) and the wall time of the whole loop.

As the paper's runs do (Sec. III: each processor periodically records N, I_N
and sigma-bar_N, and a run can be restarted indefinitely), the driver can
append one JSON line per chunk to a log (--log: N, I_N, sigma-bar_N, the
acceptance rate and the chunk's pair-pair samples per second) and keep a
checkpoint of the walk after every chunk (--checkpoint; written to a
temporary file and renamed, so a killed run leaves the previous one intact).
With --resume and an existing checkpoint the walk continues from it, and the
continued run's statistics equal those of an uninterrupted one bit for bit
(the checkpoint holds the walkers, the step counter that keys the random
streams, the step size and the blocking accumulators).

Usage (one GPU):
    python -m paper_2203_05632_gb300.run_to_target --system tiny --soft --m 512 --n-tau 2 \
        --log walk.jsonl --checkpoint walk.ckpt --resume
"""
from __future__ import annotations

import argparse
import json
import os
import time


def _write_atomic(path, blob):
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(blob)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def run(system_name="tiny", soft=True, m=512, n_tau=2, precision="mixed", target=1e-3, chunk=50000,
        max_steps=20_000_000, burn=500, seed=5632, min_blocks=100, log=None, checkpoint=None, resume=False):
    import torch

    import paper_2203_05632_gb300 as pkg
    import synthetic

    prec = {"mixed": pkg.MCMP2_MIXED, "tf32": pkg.MCMP2_TF32, "fp64": pkg.MCMP2_FP64}[precision]
    system = synthetic.make_system(system_name, soft=soft)
    ctx = pkg.Context(system, m, n_tau, prec)
    resumed = bool(resume and checkpoint and os.path.exists(checkpoint))
    if resumed:
        with open(checkpoint, "rb") as f:
            ctx.restore(f.read())
    else:
        ctx.set_walkers(None, seed, burn)
    st = ctx.stream
    samples_per_step = m * (m - 1) // 2 * n_tau
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
        chunk_ms = e0.elapsed_time(e1)
        device_ms += chunk_ms
        res = ctx.run_steps(0, seed)  # statistics only
        rel = res["error"] / abs(res["energy"]) if res["energy"] else float("inf")
        trace.append({"steps": res["steps"], "energy": res["energy"], "sigma_bar": res["error"], "relative": rel})
        if checkpoint:
            _write_atomic(checkpoint, ctx.checkpoint())
        if log:
            with open(log, "a") as f:
                f.write(json.dumps({"N": res["steps"], "blocks": res["n_blocks"], "I_N": res["energy"],
                                    "sigma_bar_N": res["error"], "relative": rel,
                                    "accept_rate": res["accept_rate"],
                                    "samples_per_s": chunk * samples_per_step / (chunk_ms / 1e3),
                                    "time": time.time()}) + "\n")
        if (res["n_blocks"] >= min_blocks and rel <= target) or res["steps"] >= max_steps:
            break
    wall = time.perf_counter() - t0
    ctx.close()
    return {"system": system_name + (" (soft)" if soft else ""), "m": m, "n_tau": n_tau, "precision": precision,
            "target": target, "reached": trace[-1]["relative"] <= target, "resumed": resumed, "steps": res["steps"],
            "energy": res["energy"], "sigma_bar": res["error"], "relative_error": trace[-1]["relative"],
            "device_s": device_ms / 1e3, "wall_s": wall, "trace": trace}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--system", default="tiny")
    ap.add_argument("--soft", action="store_true")
    ap.add_argument("--m", type=int, default=512)
    ap.add_argument("--n-tau", type=int, default=2)
    ap.add_argument("--precision", choices=["mixed", "tf32", "fp64"], default="mixed")
    ap.add_argument("--target", type=float, default=1e-3)
    ap.add_argument("--chunk", type=int, default=50000)
    ap.add_argument("--max-steps", type=int, default=20_000_000)
    ap.add_argument("--log", help="append one JSON line per chunk (N, I_N, sigma-bar_N, acceptance, samples/s)")
    ap.add_argument("--checkpoint", help="checkpoint file written after every chunk")
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint if it exists")
    args = ap.parse_args(argv)
    out = run(args.system, args.soft, args.m, args.n_tau, args.precision, args.target, args.chunk, args.max_steps,
              log=args.log, checkpoint=args.checkpoint, resume=args.resume)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
