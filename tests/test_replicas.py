"""Replica bookkeeping on the host (no GPU): weighted combination, concatenation,
and the end-of-run gather over a gloo process group of two ranks, including a
rank that failed."""
import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2203_05632_gb300 import replicas


def test_combine_is_inverse_variance_weighted():
    res = replicas.combine([{"energy": 1.0, "error": 0.1}, {"energy": 2.0, "error": 0.2}, None,
                            {"energy": 5.0, "error": float("nan")}])
    w1, w2 = 100.0, 25.0
    assert res["n_replicas"] == 2
    assert res["energy"] == pytest.approx((w1 * 1.0 + w2 * 2.0) / (w1 + w2))
    assert res["error"] == pytest.approx(1.0 / math.sqrt(w1 + w2))
    assert replicas.combine([None])["n_replicas"] == 0


def test_concatenation_equals_blocking_of_the_joined_run():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(2300) + 0.3
    a = x[:1200]
    b = x[1200:2300]
    ia, sa, ea, na = oracle.blocking(a)
    ib, sb, eb, nb = oracle.blocking(b)
    joined = replicas.concatenate({"energy": ia, "variance": sa, "n_blocks": na},
                                  {"energy": ib, "variance": sb, "n_blocks": nb})
    i, s, e, n = oracle.blocking(np.concatenate([a, b]))
    assert joined["n_blocks"] == n == 23
    assert joined["energy"] == pytest.approx(i, rel=1e-12)
    assert joined["variance"] == pytest.approx(s, rel=1e-10)
    assert joined["error"] == pytest.approx(e, rel=1e-10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        combined, gathered = replicas.gather_and_combine(results[rank])
        out_q.put((rank, combined, gathered))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("failed_rank", [None, 1])
def test_gather_over_gloo_two_ranks(failed_rank):
    import torch.multiprocessing as mp
    results = [{"energy": -1.0, "error": 0.05}, {"energy": -1.2, "error": 0.1}]
    if failed_rank is not None:
        results[failed_rank] = None
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = replicas.combine(results)
    for rank, combined, gathered in outs:
        assert gathered == results
        assert combined["n_replicas"] == (2 if failed_rank is None else 1)
        assert combined["energy"] == pytest.approx(want["energy"])


def _replica_process(directory, replica, energy, error, crash):
    from paper_2203_05632_gb300 import replicas as R
    if crash:
        raise SystemExit(3)  # dies before writing anything
    R.write_result(directory, replica, {"energy": energy, "error": error, "steps": 1000})


def test_surviving_replicas_are_combined_after_a_crash(tmp_path):
    """A replica that dies leaves no result; the others are combined (the paper's
    weighted average over surviving processors)."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    specs = [(0, -1.00, 0.05, False), (1, -1.10, 0.10, True), (2, -0.95, 0.05, False)]
    procs = [ctx.Process(target=_replica_process, args=(str(tmp_path), *s)) for s in specs]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert [p.exitcode for p in procs] == [0, 3, 0]
    (tmp_path / "replica-9.json").write_text("{truncated")  # a torn file is ignored
    out = replicas.combine_directory(str(tmp_path))
    assert out["n_replicas"] == 2
    assert out["energy"] == pytest.approx(-0.975)
    assert out["error"] == pytest.approx(0.05 / math.sqrt(2))
