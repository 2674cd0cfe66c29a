"""The exchange steps of the domain-decomposed power iteration on CPU: two gloo
ranks gather their outboxes of 128-byte flight records (sizes differ by rank,
one may be empty) in rank order, and sum their cycle-end arrays -- bytes only;
transport, statistics and the bank order run in the library and are checked
on the GPU."""
import math
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
from paper_2501_05440_gb300.domain import FLIGHT_BYTES, gather_rows, sum_over
dist.init_process_group("gloo")
rank = dist.get_rank()
sizes = [int(x) for x in os.environ["SIZES"].split(",")]
rng = np.random.default_rng(rank + 11)
rows = torch.from_numpy(rng.integers(0, 256, size=(sizes[rank], FLIGHT_BYTES), dtype=np.uint8))
got = gather_rows(dist, rows)
nfis = torch.from_numpy(rng.integers(0, 4, size=257).astype(np.int32))
sums = torch.from_numpy(rng.random(9))
np.savez(os.environ["OUT"] + f".{rank}.npz", rows=rows.numpy(), got=got.numpy(),
         nfis=nfis.numpy(), nfis_sum=sum_over(dist, nfis).numpy(),
         sums=sums.numpy(), sums_sum=sum_over(dist, sums).numpy())
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("sizes", ["5,3", "0,7", "4,0", "0,0"])
def test_two_rank_gather_and_sums(tmp_path, sizes):
    script = tmp_path / "rank.py"
    script.write_text(RANK)
    port = _free_port()
    out = str(tmp_path / "res")
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OUT=out, SIZES=sizes, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for p in procs:
        _, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
    res = [np.load(f"{out}.{r}.npz") for r in range(2)]
    whole = np.concatenate([r["rows"] for r in res])
    for r in res:
        assert r["got"].shape == whole.shape
        assert np.array_equal(r["got"], whole)
        assert np.array_equal(r["nfis_sum"], res[0]["nfis"] + res[1]["nfis"])
        assert r["nfis_sum"].dtype == np.int32
        assert np.array_equal(r["sums_sum"], res[0]["sums"] + res[1]["sums"])


def test_one_rank_without_group_is_identity():
    import torch
    from paper_2501_05440_gb300.domain import gather_rows, sum_over
    t = torch.arange(12, dtype=torch.uint8).reshape(3, 4)
    assert gather_rows(None, t) is t
    assert sum_over(None, t) is t


def test_slab_count_must_match_ranks():
    from paper_2501_05440_gb300.domain import run_domain_eigen, run_domains_one_process

    class Ctx:
        class opts:
            device = 0
    with pytest.raises(ValueError):
        run_domain_eigen(Ctx(), 10, 1, 1, 1, [-math.inf, 0.0, math.inf], group=None)
    with pytest.raises(ValueError):
        run_domains_one_process([Ctx()], 10, 1, 1, 1, [-math.inf, 0.0, math.inf])
