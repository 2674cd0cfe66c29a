"""GPU vs oracle parity of time-dependent fixed-source runs.

The particle clock, the cutoff and the fission-site times are IEEE double
expressions evaluated alike on both sides, so generation-0 histories (counts,
end states, fates including the time cutoff) and banks are bit-identical; the
time-binned population tallies are sums in different orders (relative 1e-9).
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import assert_same_histories, gpu_run, oracle_run, rel_close

pytestmark = pytest.mark.gpu
SUM_RTOL = 1e-9
# (mode, pool, graphs): one kernel per event, monolithic segment, persistent
# with the default pool, a warp pool and the register variant
MODES = [(0, 0, 0), (2, 0, 0), (1, 0, 0), (1, 64, 0), (1, -1, 0)]


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _mat(sigma_t, sigma_s, nu_sigma_f, chi):
    return {"sigma_t": np.asarray(sigma_t, float), "sigma_s": np.asarray(sigma_s, float),
            "nu_sigma_f": np.asarray(nu_sigma_f, float), "chi": np.asarray(chi, float)}


def _parity(pb, mode, pool=0, graphs=0):
    c = gpu_run(pb, mode=mode, pool=pool, graphs=graphs)
    o = oracle_run(pb)
    assert_same_histories(c.get_histories(), o.histories())
    gb, ob = c.get_bank(), o.bank()
    assert np.array_equal(gb["parent"], ob["parent"]) and np.array_equal(gb["xyz"], ob["xyz"])
    for t in range(len(pb["tallies"])):
        gm, gs = c.get_tally(t)
        om, osd = o.tally(t)
        assert gm.shape == om.shape
        assert rel_close(gm, om, SUM_RTOL, 1e-300)
        assert rel_close(gs, osd, 1e-6, 1e-14)
    cg, co = c.get_counters(), o.counters()
    for key in ["histories", "collisions", "crossings", "leaks", "lost", "generations",
                "time_cut"]:
        assert cg[key] == co[key], key
    return c, o


@pytest.mark.parametrize("mode,pool,graphs", MODES)
def test_two_group_pulse_parity(mcgb, mode, pool, graphs):
    m = _mat([0.4, 1.0], [[0.1, 0.2], [0.0, 0.6]], [0.0, 0.5], [1.0, 0.0])
    edges = np.array([0.0, 1e-7, 3e-7, 1e-6, 3e-6, 1e-5, 3e-5, 1e-4, 2e-4])
    pb = W.time_pulse_mg(m, [1.0, 0.0], [1e-7, 1e-5], t_cut=2e-4, t_edges=edges, n=6_000)
    c, o = _parity(pb, mode, pool, graphs)
    assert c.get_counters()["time_cut"] > 0


@pytest.mark.parametrize("mode,pool,graphs", MODES)
def test_multiplying_pulse_parity(mcgb, mode, pool, graphs):
    m = _mat([0.5], [[0.25]], [0.4], [1.0])
    edges = np.array([0.0, 2e-6, 4e-6, 6e-6, 8e-6, 1e-5, 1.2e-5])   # the last bin lies past the cutoff
    pb = W.time_pulse_mg(m, [1.0], [1e-6], t_cut=1.0e-5, t_edges=edges, n=3_000)
    c, o = _parity(pb, mode, pool, graphs)
    gm, _ = c.get_tally(0)
    assert np.all(gm[0, 0, 5:] == 0.0) and np.all(gm[0, 0, :5] > 0.0)


@pytest.mark.parametrize("mode,pool,graphs", [(0, 0, 0), (1, 0, 0), (2, 0, 0)])
def test_ce_scattering_pulse_parity(mcgb, mode, pool, graphs):
    E = np.geomspace(W.E_MIN, W.E_MAX, 2000)
    pb = W.time_pulse_ce(1.0, 1.0e6, t_cut=5.0e-5, t_edges=np.linspace(0.0, 5.0e-5, 6), A=1.0,
                         sig_s=20.0, density=0.05, n=4_000)
    nuc = pb["nuclides"][0]
    nuc["E"], nuc["sig_s"] = E, np.full_like(E, 20.0)
    nuc["sig_c"], nuc["sig_f"] = 1.0 / np.sqrt(E), np.zeros_like(E)
    _parity(pb, mode, pool, graphs)


@pytest.mark.parametrize("mode,pool,graphs", [(0, 0, 0), (1, 0, 0), (2, 0, 0), (1, -1, 0)])
def test_free_gas_thermal_parity(mcgb, mode, pool, graphs):
    E = np.geomspace(W.E_MIN, W.E_MAX, 2000)
    pb = W.time_pulse_ce(1.0, 0.0253, t_cut=5.0e-5, t_edges=np.linspace(0.0, 5.0e-5, 6),
                         A=1.0, sig_s=20.0, density=0.05, n=4_000)
    nuc = pb["nuclides"][0]
    nuc["E"], nuc["sig_s"] = E, np.full_like(E, 20.0)
    nuc["sig_c"], nuc["sig_f"] = 1.0 / np.sqrt(E), np.zeros_like(E)
    pb["free_gas"] = {"kT": 0.0253}
    c, o = _parity(pb, mode, pool, graphs)
    assert c.get_counters()["collisions"] > 2 * pb["run"]["n"]


@pytest.mark.parametrize("mode,pool,graphs", [(0, 0, 0), (1, 0, 0), (1, -1, 0)])
def test_ce_time_pin_parity(mcgb, mode, pool, graphs):
    pb = W.ce_time_pin(n=1_500, npts=5_000, nres=40, t_cut=2e-6, ntbins=12, batches=5)
    c, o = _parity(pb, mode, pool, graphs)
    h = c.get_histories()
    assert np.any(h["fate"] == 5)


def test_time_runs_reject_eigen_and_derivatives(mcgb):
    pb = W.pin_cell_mg(n=500, inactive=1, active=1)
    pb["time"] = {"t0": 0.0, "t_cut": 1e-5, "inv_v": np.full(pb["G"], 1e-6)}
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    with pytest.raises(mcgb.McgbError):
        c.run_eigenvalue(500, 1, 1, 1)
    pb = W.diff_slab(n=1000, batches=2)
    pb["time"] = {"t0": 0.0, "t_cut": 1e-5, "inv_v": np.full(pb["G"], 1e-6)}
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    with pytest.raises(mcgb.McgbError):
        c.forward_fixed(1000, 1, pb["detector_cell"])


def test_ce_time_pin_full_size_sampled(mcgb):
    """1e6 source histories of the time-dependent pin (the bench leg runs 1e7 of
    the same): sampled generation-0 histories recomputed one by one by the
    oracle are identical; every history ends absorbed or at the cutoff."""
    from oracle import Oracle
    pb = W.ce_time_pin(n=1_000_000)
    c = mcgb.load_problem(mcgb.Context(mode=1, record_histories=True, bank_factor=8.0), pb)
    c.run()
    h = c.get_histories()
    assert len(h["n_coll"]) == 1_000_000
    idx = np.sort(np.random.default_rng(5).choice(1_000_000, 300, replace=False))
    ho = Oracle(pb, strict=True).histories_by_index(idx)
    assert_same_histories({k: v[idx] for k, v in h.items()}, ho)
    assert set(np.unique(h["fate"]).tolist()) <= {0, 5}
    cnt = c.get_counters()
    assert cnt["time_cut"] > 0 and cnt["leaks"] == 0 and cnt["lost"] == 0


@pytest.mark.parametrize("pool", [0, -1])
def test_batch_mixing_time_and_static_problems(mcgb, pool):
    """A batch with a time-dependent problem runs every problem through the
    time-aware kernels; the static problems must give their standalone (and
    oracle) results, and the time-dependent one its own."""
    from oracle import Oracle
    m = _mat([0.4, 1.0], [[0.1, 0.2], [0.0, 0.6]], [0.0, 0.5], [1.0, 0.0])
    timed = W.time_pulse_mg(m, [1.0, 0.0], [1e-7, 1e-5], t_cut=2e-4,
                            t_edges=np.array([0.0, 1e-6, 1e-5, 1e-4, 2e-4]), n=3_000)
    probs = W.batch_boxes(nproblems=3, nmin=500, nmax=2000)[:2] + [timed]
    b = mcgb.Batch(pool=pool)
    ctxs = []
    for p in probs:
        c = mcgb.load_problem(mcgb.Context(), p)
        ctxs.append(c)
        b.add_problem(c, p["run"]["n"], p["run"]["batches"], p["run"]["seed"])
    b.run()
    for i, (c, p) in enumerate(zip(ctxs, probs)):
        c.run()
        bm, _ = b.tally(i)
        cm, _ = c.get_tally()
        om, _ = Oracle(p, strict=True).run().tally()
        assert bm.shape == cm.shape == om.shape, i
        assert rel_close(bm, cm, SUM_RTOL, 1e-300) and rel_close(bm, om, SUM_RTOL, 1e-300), i
