"""The GPU's production path against the oracle in its plain mode.

The plain oracle evaluates every step by its definition (libm log, true
division, no fused multiply-add, nuclide sums at the particle's energy); the
library keeps its own faster rounding conventions.  So the two are compared at
the tolerances the method's statement of parity sets, not bit for bit:

* random-number streams bit-exact (every history that agrees ends in the same
  generator state; stream words are compared directly elsewhere);
* per-history collision counts identical on at least 99.9% of histories;
* every tally bin within |z| < 4, z = (a - b) / sqrt(sd_a^2 + sd_b^2), and k
  within 3 combined standard deviations;
* fission-bank sizes: their differences are reported (a history that takes
  another branch changes M, and every later cycle resamples from another bank).

The launch configuration is the benchmark's: persistent pool kernel, cycles
after the first replayed as CUDA graphs.  The strict-mode comparisons in the
other GPU test files stay bit-exact.
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests.gpu_util import gpu_run

pytestmark = pytest.mark.gpu
MIN_SAME = 0.999


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _same(hg, ho, idx=None):
    """fraction of histories with equal collision counts, and the mask of
    histories equal in every recorded field"""
    a = {k: np.asarray(v) if idx is None else np.asarray(v)[idx] for k, v in hg.items()}
    coll = a["n_coll"] == np.asarray(ho["n_coll"])
    full = coll.copy()
    for k in ["n_cross", "n_fis", "fate", "g_end", "rng_end"]:
        full &= a[k] == np.asarray(ho[k])
    return coll.mean(), full


def _check_tallies(c, o, ntallies):
    worst = 0.0
    for t in range(ntallies):
        gm, gs = c.get_tally(t)
        om, osd = o.tally(t)
        gm, gs, om, osd = (np.asarray(x, float).ravel() for x in (gm, gs, om, osd))
        s = np.sqrt(gs ** 2 + osd ** 2)
        pos = s > 0
        z = np.abs(gm[pos] - om[pos]) / s[pos]
        assert np.all(z < 4.0), (t, z.max())
        # bins neither side scored in any batch agree exactly (both zero)
        assert np.array_equal(gm[~pos], om[~pos]), t
        worst = max(worst, float(z.max()) if z.size else 0.0)
    return worst


def _check_k(c, o):
    gk, ok = c.get_k(), o.k()
    for key, sdk in [("k", "k_sd"), ("k_col", "k_col_sd"), ("k_analog", "k_analog_sd")]:
        s = np.hypot(gk[sdk], ok[sdk])
        assert abs(gk[key] - ok[key]) <= 3.0 * s + 1e-12 * abs(ok[key]), (key, gk, ok)


def _eigen_vs_plain(mcgb, pb):
    ncyc = pb["run"]["inactive"] + pb["run"]["active"]
    c = gpu_run(pb, mode=1)
    o = Oracle(pb).run()
    mg, mo = c.get_cycle_k(ncyc)[2], o.cycle_k(ncyc)[2]
    diff = np.nonzero(mg != mo)[0]
    print(f"\n{pb['name']}: bank sizes differ in {len(diff)} of {ncyc} cycles"
          + (f", first at cycle {diff[0]} ({mg[diff[0]]} vs {mo[diff[0]]})" if len(diff) else ""))
    if len(diff) == 0:
        # same banks every cycle: the last cycle's histories are comparable
        frac, full = _same(c.get_histories(), o.histories())
        print(f"  last cycle: {frac:.6f} of histories with equal collision counts")
        assert frac >= MIN_SAME
        hg, ho = c.get_histories(), o.histories()
        assert np.array_equal(np.asarray(hg["rng_end"])[full], np.asarray(ho["rng_end"])[full])
    _check_k(c, o)
    z = _check_tallies(c, o, len(pb["tallies"]))
    print(f"  k {c.get_k()['k']:.6f} vs {o.k()['k']:.6f}; largest tally |z| {z:.3f}")
    return c, o


def _first_cycle(mcgb, pb):
    """first cycle only: sources are identical by construction"""
    one = W.with_run(pb, inactive=0, active=1)
    c = gpu_run(one, mode=1)
    o = Oracle(one).run()
    frac, _ = _same(c.get_histories(), o.histories())
    print(f"\n{pb['name']} first cycle: {frac:.6f} of {len(o.histories()['n_coll'])} histories "
          f"with equal collision counts; bank {c.get_cycle_k(1)[2][0]} vs {o.cycle_k(1)[2][0]}")
    assert frac >= MIN_SAME


def test_pin_cell_full_config(mcgb):
    """the pin cell at its full size: 1e4 per cycle, 10 inactive + 20 active"""
    pb = W.pin_cell_mg()
    _first_cycle(mcgb, pb)
    _eigen_vs_plain(mcgb, pb)


def test_lattice_4000_per_cycle(mcgb):
    """the C5G7-shaped lattice at 4000 per cycle, its full 50 + 100 cycles"""
    pb = W.c5g7_like_lattice(n=4000)
    _first_cycle(mcgb, pb)
    _eigen_vs_plain(mcgb, pb)


def test_ce_pin_reduced(mcgb):
    """the continuous-energy pin (full 5e4-point grids, 200 resonances per
    nuclide) at 3000 per cycle, 5 inactive + 10 active"""
    pb = W.ce_pin_cell(n=3000, inactive=5, active=10)
    _first_cycle(mcgb, pb)
    _eigen_vs_plain(mcgb, pb)


@pytest.mark.parametrize("name", ["lattice", "ce"])
def test_full_size_first_cycle_sampled(mcgb, name):
    """1e6 particles, first cycle: a sample of histories recomputed one by one
    by the plain oracle"""
    pb = W.c5g7_like_lattice(n=1_000_000, inactive=0, active=1) if name == "lattice" else \
        W.ce_pin_cell(n=1_000_000, inactive=0, active=1)
    c = gpu_run(pb, mode=1)
    h = c.get_histories()
    idx = np.sort(np.random.default_rng(11).choice(1_000_000, 3000 if name == "lattice" else 1000,
                                                   replace=False))
    ho = Oracle(pb).histories_by_index(idx)
    frac, full = _same(h, ho, idx)
    print(f"\n{name} 1e6 first cycle, {len(idx)} sampled: {frac:.6f} equal collision counts")
    assert frac >= MIN_SAME
    assert np.array_equal(np.asarray(h["rng_end"])[idx][full], np.asarray(ho["rng_end"])[full])


def test_fixed_source_slab_and_boxes(mcgb):
    for pb in [W.diff_slab(n=20000, batches=20)] + W.batch_boxes(nproblems=4, nmin=2000,
                                                                  nmax=6000)[:4]:
        c = gpu_run(pb, mode=1)
        o = Oracle(pb).run()
        frac, _ = _same(c.get_histories(), o.histories())
        assert frac >= MIN_SAME, pb["name"]
        _check_tallies(c, o, len(pb["tallies"]))


def test_derivatives_against_plain_oracle(mcgb):
    """replay-backward derivatives on the slab against the plain oracle's
    stored-score estimator on the same seeds"""
    pb = W.diff_slab(n=10, shield_len=8.0)
    n, seed, det = 4000, 77, pb["detector_cell"]
    nm = len(pb["materials"])
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    tally = c.forward_fixed(n, seed, det)
    g = c.backward_fixed(np.ones(pb["G"]), nm)
    o = Oracle(pb).grad(n=n, seed=seed, cell=det)
    assert np.allclose(tally, o["tally"], rtol=1e-9, atol=1e-300)
    for key in ["sigma_t", "sigma_s", "nu_sigma_f"]:
        a, b = np.asarray(g[key]).ravel(), np.asarray(o[key]).ravel()
        scale = max(np.abs(b).max(), 1e-300)
        assert np.all(np.abs(a - b) <= 1e-8 * np.abs(b) + 1e-12 * scale), key
