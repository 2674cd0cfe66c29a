"""The exchange step of the sharded power iteration on CPU: two gloo ranks
reduce their [k, tally] sums and gather their ordered banks (64-byte site
records) into the global bank in rank order -- bytes only; the resampling and
statistics run in the library and are checked on the GPU."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch
import torch.distributed as dist
from paper_2501_05440_gb300 import SITE_DTYPE
from paper_2501_05440_gb300.sharded import exchange, shard_range
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
N = 1003
j0, j1 = shard_range(N, rank, world)
rng = np.random.default_rng(rank + 5)
# a rank's ordered bank: parents in its own range, children 0..k-1 per parent
# (rank 1 banks nothing when EMPTY1 is set)
m = 0 if (rank == 1 and os.environ.get("EMPTY1")) else 700 + 37 * rank
par = np.sort(rng.integers(j0, j1, size=m))
bank = np.zeros(len(par), dtype=SITE_DTYPE)
bank["parent"] = par
bank["child"] = np.concatenate([np.arange(c) for c in np.bincount(par - j0)]) if len(par) else []
bank["x"] = rng.random(len(par))
raw = torch.from_numpy(np.frombuffer(bank.tobytes(), dtype=np.uint8).reshape(-1, 64).copy())
sums = torch.tensor([1.0 + rank, 2.0, 0.5, rank * 1.0], dtype=torch.float64)
gs, gb = exchange(dist, sums, raw)
np.savez(os.environ["OUT"] + f".{rank}.npz", sums=gs.numpy(), glob=gb.numpy().reshape(-1),
         own=np.frombuffer(bank.tobytes(), dtype=np.uint8))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_partition():
    from paper_2501_05440_gb300.sharded import shard_range
    for N in (1, 7, 1000, 1003):
        for w in (1, 2, 3, 8):
            r = [shard_range(N, k, w) for k in range(w)]
            assert r[0][0] == 0 and r[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))


@pytest.mark.parametrize("empty1", [False, True])
def test_two_rank_exchange_equals_one_bank(tmp_path, empty1):
    from paper_2501_05440_gb300 import SITE_DTYPE
    script = tmp_path / "rank.py"
    script.write_text(RANK)
    port = _free_port()
    out = str(tmp_path / "res")
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OUT=out, CUDA_VISIBLE_DEVICES="")
        if empty1:
            env["EMPTY1"] = "1"
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for p in procs:
        _, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
    res = [np.load(f"{out}.{r}.npz") for r in range(2)]
    own = [np.frombuffer(r["own"].tobytes(), dtype=SITE_DTYPE) for r in res]
    whole = np.concatenate(own)
    for r in res:
        glob = np.frombuffer(r["glob"].tobytes(), dtype=SITE_DTYPE)
        assert glob.tobytes() == whole.tobytes()                 # rank order = global order
        assert np.array_equal(r["sums"], [3.0, 4.0, 1.0, 1.0])
    # global (parent, child) order holds across the rank boundary
    key = whole["parent"] * 1000 + whole["child"]
    assert np.all(np.diff(key) > 0)
