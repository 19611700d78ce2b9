"""One rank of bench.py's multi-replica orchestration with a stand-in for its GPU work.

A test helper (not collected by pytest): tests/test_bench_host.py starts two of
these through paper_2203_05632_gb300.replicas.spawn_local, so the launch
environment, the gloo process group, the max-over-ranks timing and the
combination of the replicas' results run exactly as in bench.py; only
measure_rank, which needs a GB300, is replaced by fixed numbers.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def stand_in_work(args, rank, world, local, barrier):
    barrier()
    return {"dev_ms": 10.0 * (1 + rank), "e2e_s": 0.5 + rank, "e2e_steps": 3, "samples_per_step": 1000,
            "dtype": "bf16x3", "config": {"workload": "stand-in"}, "clocks": {}, "gpu_launches": 0,
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8,
            "replica": {"energy": -1.0 - 0.1 * rank, "error": 0.05 * (1 + rank), "steps": 100, "rank": rank},
            "extras": {}}


if __name__ == "__main__":
    a = bench.parse_args(sys.argv[1:])
    sys.exit(bench.run_ours(a, int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"]),
                            int(os.environ["LOCAL_RANK"]), work=stand_in_work, backend="gloo"))
