"""Argument and state checks of the time, free-gas and shard calls: bad
arguments fail with MCGB_E_INVALID_ARG (-1) or MCGB_E_STATE (-2), nothing runs.
Iteration limits fail with MCGB_E_TIMEOUT (-7)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import assert_same_histories

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _code(fn, *a):
    import paper_2501_05440_gb300 as m
    with pytest.raises(m.McgbError) as e:
        fn(*a)
    return e.value.code


def test_time_and_free_gas_arguments(mcgb):
    c = mcgb.load_problem(mcgb.Context(), W.pin_cell_mg(n=100, inactive=1, active=1))
    assert _code(c.set_time, 1e-5, 1e-6) == -1          # t_cut <= t0
    assert _code(c.set_time, -1.0, 1e-6) == -1          # t0 < 0
    assert _code(c.set_time, 0.0, float("inf")) == -1
    assert _code(c.set_inverse_speeds, [1e-6, 1e-6]) == -1   # wrong group count
    assert _code(c.set_inverse_speeds, [0.0] * 7) == -1
    assert _code(c.set_tally_time_bins, 0, [0.0]) == -1      # one edge
    assert _code(c.set_tally_time_bins, 0, [0.0, 1e-6, 1e-6]) == -1
    assert _code(c.set_tally_time_bins, 0, [-1e-6, 1e-6]) == -1
    assert _code(c.set_tally_time_bins, 5, [0.0, 1e-6]) == -1     # no such tally
    assert _code(c.set_free_gas, 0.0) == -1
    assert _code(c.set_free_gas, 0.0253, -1.0) == -1


def test_time_without_speeds_fails_at_run(mcgb):
    pb = W.diff_slab(n=500, batches=2)
    c = mcgb.load_problem(mcgb.Context(), pb)
    c.set_time(0.0, 1e-5)                                # multigroup, no 1/v given
    assert _code(c.run) in (-1, -2)


def test_shard_states_and_arguments(mcgb):
    import torch

    from paper_2501_05440_gb300 import SITE_DTYPE
    pb = W.pin_cell_mg(n=1000, inactive=1, active=1)
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    assert _code(c.shard_cycle, 0) == -2                       # no shard begun
    assert _code(c.shard_begin, 1000, 900, 200, 1, 1, 1) == -1  # slice past N
    assert _code(c.shard_begin, 0, 0, 1, 1, 1, 1) == -1
    assert _code(c.shard_begin, 1000, 0, 500, 1, 0, 1) == -1    # no active cycle
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    c.shard_begin(1000, 0, 500, 1, 1, 1)
    ns = c.shard_sums_size()
    sums = torch.empty(ns, dtype=torch.float64, device="cuda")
    assert _code(c.shard_import, 0, sums.data_ptr(), 0, 0) == -2   # export first
    m = c.shard_cycle(0)
    assert m > 0
    bank = torch.empty((m, 64), dtype=torch.uint8, device="cuda")
    assert _code(c.shard_export, bank.data_ptr(), m - 1, sums.data_ptr(), ns) == -1  # too small
    c.shard_export(bank.data_ptr(), m, sums.data_ptr(), ns)
    b = np.frombuffer(bank.cpu().numpy().tobytes(), dtype=SITE_DTYPE)
    assert np.all(b["parent"] < 500)
    assert np.all(np.diff(b["parent"] * 64 + b["child"]) > 0)   # (parent, child) order
    s = sums.cpu().numpy()
    assert s[0] > 0 and s[1] > 0
    assert _code(c.shard_import, 0, sums.data_ptr(), bank.data_ptr(), 0) == -2   # empty bank
    t = W.time_pulse_mg(W.mg_material(np.random.default_rng(1), 2, fissile=False), [1.0, 0.0],
                        [1e-6, 1e-5], t_cut=1e-5, t_edges=[0.0, 1e-5], n=100)
    ct = mcgb.load_problem(mcgb.Context(mode=1), t)
    assert _code(ct.shard_begin, 100, 0, 100, 1, 1, 1) == -1   # time-dependent: fixed source only


# Iteration limits: reaching one is an error status the host reads (no trap, no
# hang); the unfinished histories are abandoned and the device stays usable.
@pytest.mark.parametrize("mode", [0, 2])
def test_event_iteration_limit_times_out(mcgb, mode):
    pb = W.pin_cell_mg(n=2000, inactive=0, active=1)
    c = mcgb.load_problem(mcgb.Context(mode=mode, max_iterations=1), pb)
    with pytest.raises(mcgb.McgbError) as e:
        c.run()
    assert e.value.code == -7
    ok = mcgb.load_problem(mcgb.Context(mode=mode), pb)
    ok.run()
    assert ok.get_k()["k"] > 0


@pytest.mark.parametrize("pool", [0, 512, 64, -1])
@pytest.mark.parametrize("fixed", [False, True])
def test_persistent_pass_limit_times_out(mcgb, pool, fixed):
    pb = W.diff_slab(n=3000, batches=5) if fixed else W.pin_cell_mg(n=3000, inactive=1, active=1)
    c = mcgb.load_problem(mcgb.Context(mode=1, pool=pool, max_iterations=2), pb)
    with pytest.raises(mcgb.McgbError) as e:
        c.run()
    assert e.value.code == -7
    # a limit the run never reaches changes nothing
    a = mcgb.load_problem(mcgb.Context(mode=1, pool=pool, record_histories=True,
                                       max_iterations=1_000_000), pb)
    a.run()
    b = mcgb.load_problem(mcgb.Context(mode=1, pool=pool, record_histories=True), pb)
    b.run()
    assert_same_histories(a.get_histories(), b.get_histories())
