"""Host-side arithmetic of bench.py (CPU only): the algorithmic work per pair-of-pairs
sample and the issued-work ratio its roofline reports, against the counts of the trace
form, and the DRAM traffic figures against the ncu summaries they come from."""
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def test_flops_per_sample_counts_the_six_blocks():
    # Trace form: G-(1p,1q), G-(2p,2q) over the occupied and the four G+ blocks over the
    # virtual spinors, each n_comp x n_comp complex entries of k-term sums, 8 flop per
    # complex multiply-add.
    assert bench.flops_per_sample(80, 400, 4) == 225_280
    assert bench.flops_per_sample(80, 400, 2) == 56_320
    for n_occ, n_vir, nc in [(4, 16, 4), (3, 11, 2), (40, 180, 4)]:
        cmacs = sum(blocks * nc * nc * k for blocks, k in ((2, n_occ), (4, n_vir)))
        assert bench.flops_per_sample(n_occ, n_vir, nc) == 8 * cmacs


def test_issued_ratio_counts_the_unused_g_minus_blocks():
    # The contraction's tiles compute all four electron blocks of G- and G+; the trace form
    # uses two of G- and four of G+; split BF16 issues three real products per product.
    assert bench.issued_per_algorithmic(80, 400, 3, 4) == pytest.approx(3 * (4 * 480) / (2 * 80 + 4 * 400))
    assert bench.issued_per_algorithmic(80, 400, 1, 4) == pytest.approx(1920 / 1760)
    assert bench.issued_per_algorithmic(80, 400, 3, 2) == pytest.approx(3 * 1920 / 1760)


@pytest.mark.parametrize("key,profile", [(("mixed", 4), "pairs_mixed_bf16x3_medium_m1024.md"),
                                         (("tf32", 4), "pairs_mixed_tf32_medium_m1024.md"),
                                         (("mixed", 2), "pairs_mixed_bf16x3_2c_medium_m1024.md")])
def test_traffic_figures_come_from_the_committed_summaries(key, profile):
    text = open(os.path.join(ROOT, "profiles", profile)).read()
    mb = bench.PAIRS_TRAFFIC_BYTES[key] / 1e6
    assert re.search(r"traffic %.1f MB" % mb, text), (key, mb, profile)


def test_traffic_table_has_only_captured_instances():
    assert set(bench.PAIRS_TRAFFIC_BYTES) == {("mixed", 4), ("tf32", 4), ("mixed", 2)}


def test_two_local_ranks_print_one_line_with_the_combined_replicas(capfd):
    """bench.py's multi-replica path on CPU: two ranks started by replicas.spawn_local (the
    path `bench.py --gpus 2` takes without a launcher), a gloo process group, the max over
    ranks of the timed region and the inverse-variance combination of the replicas'
    results (Sec. III); the GPU work is a stand-in (tests/bench_rank_stand_in.py)."""
    import json
    import math
    import sys

    from paper_2203_05632_gb300 import replicas
    helper = os.path.join(ROOT, "tests", "bench_rank_stand_in.py")
    codes = replicas.spawn_local(2, [sys.executable, helper, "--gpus", "2", "--steps", "5", "--warmup", "3"],
                                 timeout=300)
    assert codes == [0, 0]
    lines = [l for l in capfd.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["steps"] == 5
    assert line["ms_per_step"] == pytest.approx(20.0 / 5)  # the slower rank's 20 ms
    assert line["value"] == pytest.approx(2 * 5 * 1000 / 0.020)  # whole job: both ranks' samples
    assert line["e2e"]["value"] == pytest.approx(2 * 3 * 1000 / 1.5)
    comb = line["replicas"]["combined"]
    w0, w1 = 1 / 0.05 ** 2, 1 / 0.10 ** 2
    assert comb["n_replicas"] == 2
    assert comb["energy"] == pytest.approx((w0 * -1.0 + w1 * -1.1) / (w0 + w1))
    assert comb["error"] == pytest.approx(1 / math.sqrt(w0 + w1))
    assert [r["rank"] for r in line["replicas"]["per_rank"]] == [0, 1]


def test_gpus_flag_starts_local_ranks_or_must_match_the_launcher(monkeypatch):
    from paper_2203_05632_gb300 import replicas
    calls = []
    monkeypatch.setattr(replicas, "spawn_local", lambda n, cmd, timeout=None: calls.append((n, cmd)) or [0] * n)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.main(["--gpus", "3", "--steps", "7"]) == 0
    n, cmd = calls[0]
    assert n == 3 and cmd[1].endswith("bench.py") and cmd[2:] == ["--gpus", "3", "--steps", "7"]
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--gpus", "3"]) == 2  # a launcher's world size that disagrees with --gpus
