"""Independent replicas and their combination (the paper's parallel scheme).

Sec. III: each processor runs its own Monte Carlo integration with a distinct
seed and no communication; only at the end are the results of the surviving
processors combined by a weighted average.  Runs are restartable and
concatenable.  Here a replica is one library context (one GPU); this module
holds the host-side bookkeeping:

* ``combine`` — inverse-variance weighted mean of replica results
  (weights 1/sigma-bar^2), with its standard error;
* ``concatenate`` — merge the blocking statistics of two runs of one replica
  chain (block counts add; means and squared deviations combine exactly);
* ``gather_and_combine`` — collect every rank's result over a
  ``torch.distributed`` process group at the end of a run and combine them.
  Ranks that failed pass ``None`` and are left out.
* ``spawn_local`` — start N local ranks (one process per GPU) of a command
  with the torch.distributed environment set, for a run that was not started
  by a launcher;
* ``write_result`` / ``combine_directory`` — the fault-tolerant path: each
  replica writes its result file atomically when it finishes (or at each
  checkpoint); the combination reads whatever the surviving replicas wrote,
  so a replica that died leaves nothing behind and is simply absent.
"""
from __future__ import annotations

import json
import math
import os
import socket
import subprocess


def combine(results):
    """Inverse-variance weighted average of replica results.

    results: iterable of dicts with keys 'energy' and 'error' (sigma-bar);
    entries that are None, or have a non-positive or non-finite error, are
    skipped.  Returns dict(energy, error, n_replicas)."""
    num = 0.0
    den = 0.0
    n = 0
    for r in results:
        if r is None:
            continue
        e, s = r.get("energy"), r.get("error")
        if e is None or s is None or not math.isfinite(e) or not math.isfinite(s) or s <= 0.0:
            continue
        w = 1.0 / (s * s)
        num += w * e
        den += w
        n += 1
    if n == 0:
        return {"energy": float("nan"), "error": float("nan"), "n_replicas": 0}
    return {"energy": num / den, "error": math.sqrt(1.0 / den), "n_replicas": n}


def concatenate(a, b, block_size=100):
    """Blocking statistics of the concatenation of two runs of complete blocks.

    a, b: dicts with 'energy' (I_N), 'variance' (sigma_N^2) and 'n_blocks'.
    Means and sums of squared deviations of block means combine exactly
    (parallel form of Welford's update)."""
    na, nb = int(a["n_blocks"]), int(b["n_blocks"])
    if na == 0:
        return dict(b)
    if nb == 0:
        return dict(a)
    n = na + nb
    d = b["energy"] - a["energy"]
    mean = a["energy"] + d * nb / n
    m2 = a["variance"] * na + b["variance"] * nb + d * d * na * nb / n
    var = m2 / n
    return {"energy": mean, "variance": var, "error": math.sqrt(var) / math.sqrt(n), "n_blocks": n,
            "steps": n * block_size}


def gather_and_combine(result, group=None):
    """All-gather each rank's result (a dict or None) and combine them on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gathered = [None] * world
    dist.all_gather_object(gathered, result, group=group)
    return combine(gathered), gathered


def write_result(directory, replica, result):
    """Atomically write one replica's result (a dict) as <directory>/replica-<id>.json."""
    os.makedirs(directory, exist_ok=True)
    final = os.path.join(directory, f"replica-{int(replica)}.json")
    tmp = final + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(result, f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, final)
    return final


def combine_directory(directory):
    """Combine the results of the replicas that wrote one; unreadable files are skipped."""
    results = {}
    if os.path.isdir(directory):
        for name in sorted(os.listdir(directory)):
            if not (name.startswith("replica-") and name.endswith(".json")):
                continue
            try:
                with open(os.path.join(directory, name)) as f:
                    results[name] = json.load(f)
            except (OSError, ValueError):
                continue
    out = combine(results.values())
    out["replicas"] = sorted(results)
    return out


def free_port() -> int:
    """A free TCP port on 127.0.0.1 for the rendezvous of local ranks."""
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def spawn_local(n_ranks: int, cmd, timeout=None):
    """Run `cmd` (an argv list) as n_ranks local processes, rank r with RANK = LOCAL_RANK = r,
    WORLD_SIZE = n_ranks and a rendezvous on 127.0.0.1 (one process per GPU, the replicas
    of the paper's parallel scheme).  Standard output and error are inherited.  Returns
    the exit codes in rank order; a rank still running after `timeout` seconds is killed
    (its exit code is then negative)."""
    port = free_port()
    procs = []
    for r in range(n_ranks):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n_ranks),
                   LOCAL_WORLD_SIZE=str(n_ranks), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen(list(cmd), env=env))
    codes = []
    for p in procs:
        try:
            codes.append(p.wait(timeout=timeout))
        except subprocess.TimeoutExpired:
            p.kill()
            codes.append(p.wait())
    return codes
