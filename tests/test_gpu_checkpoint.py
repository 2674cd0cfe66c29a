"""Checkpoint and restart of a power iteration through the C ABI: a run
restored from a checkpoint -- on a fresh context, in another execution mode
-- finishes with the uninterrupted run's bank sizes, last-cycle histories and
bank bit for bit, and its k and tallies (sums over slots, taken in the same
order up to the atomics of the reductions) to a relative 1e-12 (standard
deviations, which cancel, 1e-9); taking the checkpoint leaves the run
unchanged; bad records are refused."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
INACTIVE, ACTIVE = 2, 4
NCYC = INACTIVE + ACTIVE


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _ctx(m, pb, mode):
    return m.load_problem(m.Context(mode=mode, record_histories=True), pb)


def _results(c, pb):
    out = {"cycle": c.get_cycle_k(NCYC), "k": c.get_k(), "hist": c.get_histories(), "bank": c.get_bank(),
           "tally": [c.get_tally(t) for t in range(len(pb["tallies"]))]}
    return out


def _same(a, b):
    assert a["cycle"][2].tolist() == b["cycle"][2].tolist()          # bank sizes
    for x, y in zip(a["cycle"][:2], b["cycle"][:2]):
        assert np.allclose(x, y, rtol=1e-12, atol=0)
    for key in a["hist"]:
        assert np.array_equal(a["hist"][key], b["hist"][key]), key
    for x, y in zip(a["bank"], b["bank"]):
        assert np.array_equal(x, y)
    for (ma, sa), (mb, sb) in zip(a["tally"], b["tally"]):
        assert np.allclose(ma, mb, rtol=1e-12, atol=1e-300)
        assert np.allclose(sa, sb, rtol=1e-9, atol=1e-300)
    for key in a["k"]:   # an sd cancels: sum of squares less the squared sum
        tol = 1e-9 if key.endswith("_sd") else 1e-12
        assert abs(a["k"][key] - b["k"][key]) <= tol * max(abs(b["k"][key]), 1e-300), key


@pytest.mark.parametrize("at", [1, 2, NCYC - 1])
def test_restored_run_equals_uninterrupted(mcgb, at):
    pb = W.c5g7_like_lattice(n=4000, inactive=INACTIVE, active=ACTIVE)
    r = pb["run"]
    ref = _ctx(mcgb, pb, mcgb.MODE_PERSISTENT)
    ref.eigen_begin(r["n"], INACTIVE, ACTIVE, r["seed"])
    ref.eigen_cycles(NCYC)
    ref.eigen_finish()
    want = _results(ref, pb)

    a = _ctx(mcgb, pb, mcgb.MODE_PERSISTENT)
    a.eigen_begin(r["n"], INACTIVE, ACTIVE, r["seed"])
    a.eigen_cycles(at)
    blob = a.eigen_checkpoint()
    a.eigen_cycles(NCYC - at)          # the checkpoint leaves the run as it was
    a.eigen_finish()
    _same(_results(a, pb), want)

    for mode in (mcgb.MODE_EVENT, mcgb.MODE_PERSISTENT):
        b = _ctx(mcgb, pb, mode)
        b.eigen_restore(blob)
        b.eigen_cycles(NCYC - at)
        b.eigen_finish()
        _same(_results(b, pb), want)


def test_ce_pin_restored(mcgb):
    pb = W.ce_pin_cell(n=2000, inactive=1, active=3, npts=5000, nres=40)
    r = pb["run"]
    ref = mcgb.load_problem(mcgb.Context(mode=mcgb.MODE_PERSISTENT), pb)
    ref.eigen_begin(r["n"], 1, 3, r["seed"])
    ref.eigen_cycles(2)
    blob = ref.eigen_checkpoint()
    ref.eigen_cycles(2)
    ref.eigen_finish()
    b = mcgb.load_problem(mcgb.Context(mode=mcgb.MODE_SEGMENT), pb)
    b.eigen_restore(blob)
    b.eigen_cycles(2)
    b.eigen_finish()
    assert b.get_cycle_k(4)[2].tolist() == ref.get_cycle_k(4)[2].tolist()
    assert abs(b.get_k()["k"] - ref.get_k()["k"]) <= 1e-12 * ref.get_k()["k"]


def test_checkpoint_refusals(mcgb):
    pb = W.pin_cell_mg(n=1000, inactive=1, active=2)
    r = pb["run"]
    c = mcgb.load_problem(mcgb.Context(mode=mcgb.MODE_PERSISTENT), pb)
    with pytest.raises(mcgb.McgbError) as e:
        c.eigen_checkpoint()                    # no run
    assert e.value.code == -2
    c.eigen_begin(r["n"], 1, 2, r["seed"])
    with pytest.raises(mcgb.McgbError) as e:
        c.eigen_checkpoint()                    # no cycle run yet
    assert e.value.code == -2
    c.eigen_cycles(1)
    blob = c.eigen_checkpoint()
    c.eigen_cycles(2)
    with pytest.raises(mcgb.McgbError) as e:
        c.eigen_checkpoint()                    # no cycle left
    assert e.value.code == -2

    fresh = mcgb.load_problem(mcgb.Context(mode=mcgb.MODE_PERSISTENT), pb)
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x40                  # one flipped bit in the sources
    for rec in (bytes(bad), blob[:-9], blob[:40], b"\0" * len(blob)):
        with pytest.raises(mcgb.McgbError) as e:
            fresh.eigen_restore(rec)
        assert e.value.code == -1
    other = mcgb.load_problem(mcgb.Context(mode=mcgb.MODE_PERSISTENT),
                              W.pin_cell_mg(seed=2, n=1000, inactive=1, active=2))
    with pytest.raises(mcgb.McgbError) as e:
        other.eigen_restore(blob)               # another problem's checkpoint
    assert e.value.code == -1
    fresh.eigen_restore(blob)                   # the good record still restores
    fresh.eigen_cycles(2)
    fresh.eigen_finish()
    c.eigen_finish()
    assert fresh.get_cycle_k(3)[2].tolist() == c.get_cycle_k(3)[2].tolist()
