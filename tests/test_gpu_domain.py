"""Spatial domain decomposition through the C ABI.

One slab (-inf, inf) must reproduce the single-device run exactly.  With
several slabs a flight that crosses a cut is stopped on it and continued by
the neighbouring slab with the rest of its sampled collision distance (no new
draw), so histories are the single-device ones up to the rounding of those
split flights: compared at the method's tolerances (>= 99.9% of histories
with equal collision counts, tallies |z| < 4, k within 3 sd), with the
per-cycle bank sizes reported.  The slabs run as several contexts of one
process on this device, and as two processes over gloo.
"""
import math
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INF = math.inf


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _single(m, pb):
    c = m.load_problem(m.Context(mode=1, record_histories=True), pb)
    c.run()
    return c


def _records(ctxs, N):
    """per-history records of the last cycle, summed over the slabs' contexts"""
    import torch
    tot = None
    for c in ctxs:
        a = [torch.zeros(N, dtype=torch.int32, device="cuda") for _ in range(5)]
        rng = torch.zeros(N, dtype=torch.int64, device="cuda")
        c.domain_records(*[t.data_ptr() for t in a], rng.data_ptr())
        vals = [t.cpu().numpy().astype(np.int64) for t in a] + [rng.cpu().numpy().view(np.uint64)]
        tot = vals if tot is None else [x + y for x, y in zip(tot, vals)]
    keys = ["n_coll", "n_cross", "n_fis", "fate", "g_end", "rng_end"]
    return dict(zip(keys, tot))


def _domains(mcgb, pb, cuts, axis=0):
    from paper_2501_05440_gb300.domain import run_domains_one_process
    r = pb["run"]
    ctxs = [mcgb.load_problem(mcgb.Context(mode=1), pb) for _ in range(len(cuts) - 1)]
    sweeps = run_domains_one_process(ctxs, r["n"], r["inactive"], r["active"], r["seed"], cuts, axis)
    return ctxs, sweeps


def test_one_slab_equals_single_device(mcgb):
    pb = W.c5g7_like_lattice(n=6000, inactive=2, active=3)
    ncyc = 5
    ref = _single(mcgb, pb)
    (c,), sweeps = _domains(mcgb, pb, [-INF, INF])
    assert sweeps == [1] * ncyc                      # nothing ever leaves the only slab
    assert c.get_cycle_k(ncyc)[2].tolist() == ref.get_cycle_k(ncyc)[2].tolist()
    for a, b in zip(c.get_cycle_k(ncyc)[:2], ref.get_cycle_k(ncyc)[:2]):
        assert np.allclose(a, b, rtol=1e-12, atol=0)
    h, hr = _records([c], 6000), ref.get_histories()
    for k in ["n_coll", "n_cross", "n_fis", "fate", "g_end"]:
        assert np.array_equal(h[k], np.asarray(hr[k]).astype(np.int64)), k
    assert np.array_equal(h["rng_end"], np.asarray(hr["rng_end"]).astype(np.uint64))
    for t in range(len(pb["tallies"])):
        gm, gs = c.get_tally(t)
        rm, rs = ref.get_tally(t)
        assert np.allclose(gm, rm, rtol=1e-9, atol=1e-300)
    for key in ("k", "k_col", "k_analog"):
        assert abs(c.get_k()[key] - ref.get_k()[key]) <= 1e-12 * abs(ref.get_k()[key])


def _compare(ref, ctxs, pb, label):
    ncyc = pb["run"]["inactive"] + pb["run"]["active"]
    N = pb["run"]["n"]
    mg, mr = ctxs[0].get_cycle_k(ncyc)[2], ref.get_cycle_k(ncyc)[2]
    diff = np.nonzero(mg != mr)[0]
    print(f"\n{label}: bank sizes differ in {len(diff)} of {ncyc} cycles")
    if len(diff) == 0:
        h, hr = _records(ctxs, N), ref.get_histories()
        same = np.mean(h["n_coll"] == np.asarray(hr["n_coll"]))
        print(f"  last cycle: {same:.6f} of histories with equal collision counts")
        assert same >= 0.999
    gk, rk = ctxs[0].get_k(), ref.get_k()
    for key, sd in [("k", "k_sd"), ("k_col", "k_col_sd"), ("k_analog", "k_analog_sd")]:
        assert abs(gk[key] - rk[key]) <= 3 * math.hypot(gk[sd], rk[sd]) + 1e-12, key
    for t in range(len(pb["tallies"])):
        gm, gs = ctxs[0].get_tally(t)
        rm, rs = ref.get_tally(t)
        s = np.sqrt(np.asarray(gs) ** 2 + np.asarray(rs) ** 2)
        pos = s > 0
        assert np.all(np.abs(np.asarray(gm)[pos] - np.asarray(rm)[pos]) / s[pos] < 4.0)
    # every slab's context ends with the same (whole-run) results
    for c in ctxs[1:]:
        assert c.get_cycle_k(ncyc)[2].tolist() == mg.tolist()
        assert c.get_k()["k"] == gk["k"]


@pytest.mark.parametrize("cuts,axis", [([-INF, 32.13, INF], 0),
                                       ([-INF, 10.0, 21.4, 45.0, INF], 1)])
def test_lattice_slabs_match_single_device(mcgb, cuts, axis):
    pb = W.c5g7_like_lattice(n=6000, inactive=2, active=3)
    ref = _single(mcgb, pb)
    ctxs, sweeps = _domains(mcgb, pb, cuts, axis)
    assert max(sweeps) > 1                        # particles did cross the cuts
    _compare(ref, ctxs, pb, f"lattice, {len(cuts) - 1} slabs along axis {axis}")


def test_ce_pin_slabs_match_single_device(mcgb):
    pb = W.ce_pin_cell(n=3000, inactive=1, active=3, npts=5000, nres=40)
    ref = _single(mcgb, pb)
    ctxs, sweeps = _domains(mcgb, pb, [-INF, 0.0, INF], 0)
    assert max(sweeps) > 1
    _compare(ref, ctxs, pb, "CE pin, 2 slabs")


def test_domain_calls_out_of_order(mcgb):
    pb = W.pin_cell_mg(n=1000, inactive=1, active=1)
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    with pytest.raises(mcgb.McgbError) as e:
        c.domain_sweep()
    assert e.value.code == -2
    with pytest.raises(mcgb.McgbError) as e:
        c.domain_begin(1000, 1, 1, 1, 0, [0.0, INF], 0)     # the outer cuts must be infinite
    assert e.value.code == -1
    with pytest.raises(mcgb.McgbError) as e:
        c.domain_begin(1000, 1, 1, 1, 0, [-INF, 1.0, 0.5, INF], 0)   # not increasing
    assert e.value.code == -1
    c.domain_begin(1000, 1, 1, 1, 0, [-INF, INF], 0)
    with pytest.raises(mcgb.McgbError) as e:
        c.domain_sweep()                                  # sources first
    assert e.value.code == -2
    c.domain_sources(0)
    with pytest.raises(mcgb.McgbError) as e:
        c.domain_import(0, 0, 0, 0, 1)                    # export first
    assert e.value.code == -2


RANK = r"""
import math, os, sys
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch.distributed as dist
import paper_2501_05440_gb300 as m
import workloads as W
from paper_2501_05440_gb300.domain import run_domain_eigen
dist.init_process_group("gloo")
pb = W.c5g7_like_lattice(n=4000, inactive=1, active=2)
r = pb["run"]
c = m.load_problem(m.Context(mode=1), pb)
sweeps = run_domain_eigen(c, r["n"], r["inactive"], r["active"], r["seed"],
                          [-math.inf, 32.13, math.inf], 0, group=dist)
mean, sd = c.get_tally(0)
np.savez(os.environ["OUT"] + f".{dist.get_rank()}.npz", bank_m=c.get_cycle_k(3)[2],
         k=c.get_k()["k"], tally=mean.ravel(), sweeps=np.array(sweeps))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_processes_over_gloo_equal_one_process(mcgb, tmp_path):
    """two ranks on this device (their kernels never wait on each other),
    exchanging over gloo, give the one-process two-slab run's results"""
    pb = W.c5g7_like_lattice(n=4000, inactive=1, active=2)
    ctxs, _ = _domains(mcgb, pb, [-INF, 32.13, INF], 0)
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
    mean, _ = ctxs[0].get_tally(0)
    for k in range(2):
        res = np.load(f"{out}.{k}.npz")
        assert res["bank_m"].tolist() == ctxs[0].get_cycle_k(3)[2].tolist()
        assert abs(float(res["k"]) - ctxs[0].get_k()["k"]) <= 1e-12 * abs(ctxs[0].get_k()["k"])
        assert np.allclose(res["tally"], mean.ravel(), rtol=1e-9, atol=1e-300)
