"""The run-to-target driver's log and checkpoint/resume (Sec. III: runs record N, I_N and
sigma-bar_N periodically and can be restarted indefinitely).

A walk cut after its first chunk and resumed from the checkpoint in a fresh context ends
with the same statistics, bit for bit, as the same walk run without the cut; the log
holds one line per chunk with the blocked statistics."""
import json

import pytest

from paper_2203_05632_gb300 import run_to_target

pytestmark = pytest.mark.gpu

KW = dict(system_name="tiny", soft=True, m=64, n_tau=2, precision="mixed", target=1e-9, chunk=300, burn=200,
          seed=77, min_blocks=1)


def test_resumed_walk_equals_the_uninterrupted_one(tmp_path):
    whole = run_to_target.run(max_steps=600, log=str(tmp_path / "whole.jsonl"), **KW)
    ck = str(tmp_path / "walk.ckpt")
    first = run_to_target.run(max_steps=300, checkpoint=ck, log=str(tmp_path / "cut.jsonl"), **KW)
    second = run_to_target.run(max_steps=600, checkpoint=ck, resume=True, log=str(tmp_path / "cut.jsonl"), **KW)
    assert not first["resumed"] and second["resumed"]
    assert whole["steps"] == second["steps"] == 600
    assert whole["energy"] == second["energy"]
    assert whole["sigma_bar"] == second["sigma_bar"]
    lines = [json.loads(x) for x in open(tmp_path / "whole.jsonl")]
    assert [x["N"] for x in lines] == [300, 600]
    assert lines[-1]["I_N"] == whole["energy"] and lines[-1]["sigma_bar_N"] == whole["sigma_bar"]
    assert all(x["blocks"] == x["N"] // 100 and x["samples_per_s"] > 0 and 0 < x["accept_rate"] < 1 for x in lines)
    cut = [json.loads(x) for x in open(tmp_path / "cut.jsonl")]
    assert [x["N"] for x in cut] == [300, 600] and cut[-1]["I_N"] == whole["energy"]


def test_resume_without_a_checkpoint_starts_a_new_walk(tmp_path):
    out = run_to_target.run(max_steps=300, checkpoint=str(tmp_path / "none.ckpt"), resume=True, **KW)
    assert not out["resumed"] and out["steps"] == 300
