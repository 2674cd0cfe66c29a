"""Sharded power iteration through the C ABI: one rank equals the single-device
run; two ranks (two processes on this device, gloo exchange) give the same
per-cycle bank sizes and the same final bank, site by site."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _problem():
    return W.c5g7_like_lattice(n=6000, inactive=2, active=3)


def _single(m, pb):
    c = m.load_problem(m.Context(mode=1, record_histories=True), pb)
    c.run()
    return c


@pytest.mark.parametrize("mode", [1, 0])
def test_one_rank_equals_single_run(mcgb, mode):
    from paper_2501_05440_gb300.sharded import run_sharded_eigen
    pb = _problem()
    r = pb["run"]
    ncyc = r["inactive"] + r["active"]
    ref = _single(mcgb, pb)
    c = mcgb.load_problem(mcgb.Context(mode=mode), pb)
    res = run_sharded_eigen(c, r["n"], r["inactive"], r["active"], r["seed"])
    k_tl, k_c, m = ref.get_cycle_k(ncyc)
    s_tl, s_c, s_m = c.get_cycle_k(ncyc)
    assert s_m.tolist() == m.tolist()
    assert np.allclose(s_tl, k_tl, rtol=1e-12) and np.allclose(s_c, k_c, rtol=1e-12)
    b = ref.get_bank()
    g = res["bank"]
    assert np.array_equal(g["parent"], b["parent"]) and np.array_equal(g["child"], b["child"])
    xyz = np.stack([g["x"], g["y"], g["z"]], axis=1).ravel()
    assert np.array_equal(xyz, np.asarray(b["xyz"]).ravel())
    for t in range(len(pb["tallies"])):
        mean, sd = ref.get_tally(t)
        smean, ssd = c.get_tally(t)
        assert np.allclose(smean, mean, rtol=1e-9, atol=1e-300)
        assert np.allclose(ssd, sd, rtol=1e-6, atol=1e-14)
    for key in ("k", "k_col", "k_analog"):
        assert abs(c.get_k()[key] - ref.get_k()[key]) <= 1e-12 * abs(ref.get_k()[key])


def test_shard_calls_out_of_order(mcgb):
    pb = _problem()
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    with pytest.raises(mcgb.McgbError) as e:
        c.shard_cycle(0)
    assert e.value.code == -2                      # no shard begun
    c.shard_begin(6000, 0, 6000, 1, 1, 3)
    with pytest.raises(mcgb.McgbError) as e:
        c.shard_cycle(1)
    assert e.value.code == -2                      # cycles in order
    with pytest.raises(mcgb.McgbError) as e:
        c.shard_finish()
    assert e.value.code == -2                      # cycles remain


RANK = r"""
import os, sys
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch.distributed as dist
import paper_2501_05440_gb300 as m
import workloads as W
from paper_2501_05440_gb300.sharded import run_sharded_eigen
dist.init_process_group("gloo")
pb = W.c5g7_like_lattice(n=6000, inactive=2, active=3)
r = pb["run"]
c = m.load_problem(m.Context(mode=1), pb)
res = run_sharded_eigen(c, r["n"], r["inactive"], r["active"], r["seed"], group=dist)
mean, sd = c.get_tally(0)
np.savez(os.environ["OUT"] + f".{dist.get_rank()}.npz", bank_m=c.get_cycle_k(5)[2],
         k_tl=c.get_cycle_k(5)[0], bank=np.frombuffer(res["bank"].tobytes(), dtype=np.uint8),
         tally=mean.ravel(), k=c.get_k()["k"])
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_equal_single_run(mcgb, tmp_path):
    """two processes on this device (their kernels never wait on each other),
    exchanging over gloo"""
    from paper_2501_05440_gb300 import SITE_DTYPE
    pb = _problem()
    r = pb["run"]
    ref = _single(mcgb, pb)
    script = tmp_path / "rank.py"
    script.write_text(RANK)
    out = str(tmp_path / "res")
    port = _free_port()
    procs = []
    for k in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(k), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OUT=out)
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for p in procs:
        _, err = p.communicate(timeout=600)
        assert p.returncode == 0, err[-3000:]
    _, _, m = ref.get_cycle_k(r["inactive"] + r["active"])
    b = ref.get_bank()
    mean, _ = ref.get_tally(0)
    for k in range(2):   # every rank holds the whole run's results
        res = np.load(f"{out}.{k}.npz")
        assert res["bank_m"].tolist() == m.tolist()
        g = np.frombuffer(res["bank"].tobytes(), dtype=SITE_DTYPE)
        assert np.array_equal(g["parent"], b["parent"]) and np.array_equal(g["child"], b["child"])
        xyz = np.stack([g["x"], g["y"], g["z"]], axis=1).ravel()
        assert np.array_equal(xyz, np.asarray(b["xyz"]).ravel())
        assert np.allclose(res["tally"], mean.ravel(), rtol=1e-9, atol=1e-300)
        assert abs(float(res["k"]) - ref.get_k()["k"]) <= 1e-12 * abs(ref.get_k()["k"])
