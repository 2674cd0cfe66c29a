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
    ref = _single(mcgb, pb)
    c = mcgb.load_problem(mcgb.Context(mode=mode), pb)
    res = run_sharded_eigen(c, r["n"], r["inactive"], r["active"], r["seed"])
    k_tl, k_c, m = ref.get_cycle_k(r["inactive"] + r["active"])
    assert res["bank_m"].tolist() == m.tolist()
    assert np.allclose(res["k_tl"], k_tl, rtol=1e-12) and np.allclose(res["k_col"], k_c, rtol=1e-12)
    b = ref.get_bank()
    g = res["bank"]
    assert np.array_equal(g["parent"], b["parent"]) and np.array_equal(g["child"], b["child"])
    xyz = np.stack([g["x"], g["y"], g["z"]], axis=1).ravel()
    assert np.array_equal(xyz, np.asarray(b["xyz"]).ravel())
    mean, _ = ref.get_tally(0)
    assert np.allclose(res["tally_mean"], mean.ravel(), rtol=1e-9, atol=1e-300)
    assert abs(res["k"] - ref.get_k()["k"]) <= 1e-12 * abs(ref.get_k()["k"])


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
if dist.get_rank() == 0:
    np.savez(os.environ["OUT"], bank_m=res["bank_m"], k_tl=res["k_tl"], bank=res["bank"].tobytes(),
             tally=res["tally_mean"])
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_equal_single_run(mcgb, tmp_path):
    from paper_2501_05440_gb300 import SITE_DTYPE
    pb = _problem()
    r = pb["run"]
    ref = _single(mcgb, pb)
    script = tmp_path / "rank.py"
    script.write_text(RANK)
    out = str(tmp_path / "res.npz")
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
    res = np.load(out)
    _, _, m = ref.get_cycle_k(r["inactive"] + r["active"])
    assert res["bank_m"].tolist() == m.tolist()
    g = np.frombuffer(res["bank"].tobytes(), dtype=SITE_DTYPE)
    b = ref.get_bank()
    assert np.array_equal(g["parent"], b["parent"]) and np.array_equal(g["child"], b["child"])
    xyz = np.stack([g["x"], g["y"], g["z"]], axis=1).ravel()
    assert np.array_equal(xyz, np.asarray(b["xyz"]).ravel())
    mean, _ = ref.get_tally(0)
    assert np.allclose(res["tally"], mean.ravel(), rtol=1e-9, atol=1e-300)
