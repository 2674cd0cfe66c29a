"""Multi-rank bench path on CPU: two gloo ranks run the same aggregation the
GPU ranks run under torchrun (barrier, slowest-rank time, summed units), and
replicas share the problem but not the random streams."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import bench
import workloads as W

class A: pass
rank, world, local, pg = bench.dist_setup(A())
assert pg is not None and pg.get_backend() == "gloo"
bench.barrier(pg)
ms = [12.5, 20.0][rank]
units = [1000, 3000][rank]
ms_max, total, value = bench.aggregate(pg, ms, units)
pb = bench.replica_problem(W, 100, rank)
print(json.dumps({"rank": rank, "world": world, "ms_max": ms_max, "total": total,
                  "value": value, "seed": pb["run"]["seed"],
                  "sigt0": float(pb["materials"][0]["sigma_t"][0])}), flush=True)
pg.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_aggregate_like_torchrun(tmp_path):
    pytest.importorskip("torch.distributed")
    script = tmp_path / "rank.py"
    script.write_text(RANK_SCRIPT)
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(__import__("json").loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2
        assert o["ms_max"] == 20.0                        # slowest rank
        assert o["total"] == 4000.0                       # units of both ranks
        assert o["value"] == pytest.approx(4000.0 / 0.020)
    # same problem tables on both replicas, distinct master seeds
    assert outs[0]["sigt0"] == outs[1]["sigt0"]
    assert outs[0]["seed"] != outs[1]["seed"]


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_cpu():
    """`bench.py --impl reference` (the oracle on this host's cores) prints one
    JSON line with the contract's keys, its cpu_baseline and e2e describing the
    same run."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = __import__("json").loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "histories/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_gpus_flag_starts_ranks_or_refuses():
    """--gpus N is honoured: outside torchrun bench.py starts N ranks itself,
    and refuses (exit 2) when it cannot, instead of running one."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    env.pop("WORLD_SIZE", None)
    # the CUDA arm with no GPU visible: refused, nothing run
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 2 and "refusing" in r.stderr
    # a rank count that contradicts the launcher's
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"],
                       env=dict(env, WORLD_SIZE="1", RANK="0"), capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 2 and "refusing" in r.stderr
    # the reference arm (CPU oracle) under two ranks started by bench.py itself:
    # rank 0 prints the one JSON line, rank 1 exits without work
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    import json
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2


def test_workload_option_selects_the_headline_problem():
    """--workload picks the problem of the headline leg: the lattice by
    default, the continuous-energy pin cell for profiling; replicas keep the
    problem and take their own master seed."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    lat = bench.replica_problem(W, 1000, 0)
    ce = bench.replica_problem(W, 1000, 1, "ce-pin")
    assert lat["name"] == bench.WORKLOADS["lattice"] and lat["lattices"]
    assert ce["name"] == bench.WORKLOADS["ce-pin"] and not ce["lattices"]
    assert ce["run"]["seed"] == bench.replica_problem(W, 1000, 0, "ce-pin")["run"]["seed"] + 1000003
    assert set(bench.WORKLOADS) == {"lattice", "ce-pin"}
