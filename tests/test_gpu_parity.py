"""GPU vs oracle parity, element by element, through the C ABI.

Every history draws from its own random stream and both implementations
evaluate the same IEEE double expressions without contraction, so random
streams, histories (collision and crossing counts, end states, fates), fission
banks and per-cycle bank sizes must be bit-identical.  Tallies and k are sums
over histories taken in different orders (atomics on the GPU), so they agree to
a relative 1e-9 (rounding of ~1e6 additions of O(1) terms is ~1e-10).
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests.gpu_util import assert_same_histories, gpu_run, oracle_run, rel_close

pytestmark = pytest.mark.gpu
SUM_RTOL = 1e-9


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def test_rng_streams_bit_exact(mcgb, orc):
    c = mcgb.Context()
    ids = [0, 5, 152916, (3 << 32) + 7, (200 << 32) + 123456]
    for first in ids:
        st = c.rng_states(12345, first, 64, 200)
        for i in [0, 1, 33, 63]:
            s = orc.rng_stream(12345, first + i)
            for k in range(200):
                s = orc.rng_next(s)
                assert int(st[i, k]) == s
    big = c.rng_states(1, 0, 1000, 1000)
    s = orc.rng_stream(1, 999)
    for k in range(1000):
        s = orc.rng_next(s)
    assert int(big[999, 999]) == s


def test_log_bit_exact(mcgb, orc):
    c = mcgb.Context()
    s = 99
    xs = []
    for _ in range(50000):
        s = orc.rng_next(s)
        xs.append(orc.rng_xi(s))
    xs += [1.0, 0.5, 2.0**-53, 1 - 2.0**-53, 0.75]
    xs = np.array(xs)
    got = c.log(xs)
    ref = np.array([orc.log(float(x)) for x in xs])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("name", ["pin", "lattice", "slab", "box"])
def test_geometry_probe_bit_exact(mcgb, name):
    pb = {"pin": W.pin_cell_mg(n=10), "lattice": W.c5g7_like_lattice(n=10),
          "slab": W.diff_slab(n=10), "box": W.batch_boxes(nproblems=2)[1]}[name]
    c = mcgb.load_problem(mcgb.Context(), pb)
    o = Oracle(pb, strict=True)
    xs = [s["coef"][0] for s in pb["surfaces"] if s["type"] == "px"]
    ys = [s["coef"][0] for s in pb["surfaces"] if s["type"] == "py"]
    zs = [s["coef"][0] for s in pb["surfaces"] if s["type"] == "pz"] or [-3.0, 3.0]
    rng = np.random.default_rng(4)
    n = 3000
    pos = np.stack([rng.uniform(min(xs), max(xs), n), rng.uniform(min(ys), max(ys), n),
                    rng.uniform(min(zs), max(zs), n)], 1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    path, dist, kind = c.probe(pos, d)
    for i in range(0, n, 7):
        op, od, ok = o.probe(pos[i], d[i])
        assert list(path[i]) == [int(v) for v in op]
        assert dist[i] == od and kind[i] == ok


def test_ce_lookup_bit_exact(mcgb):
    pb = W.ce_pin_cell(n=10, npts=5000, nres=30)
    c = mcgb.load_problem(mcgb.Context(), pb)
    o = Oracle(pb, strict=True)
    rng = np.random.default_rng(8)
    E = np.exp(rng.uniform(np.log(1e-5), np.log(2e7), 4000))
    E = np.concatenate([E, pb["nuclides"][3]["E"][::97], [1e-5, 2e7]])
    for mat in (0, 1):
        out = c.ce_lookup(mat, E)
        for i in range(0, len(E), 3):
            assert np.array_equal(out[i], o.ce_lookup(mat, float(E[i])))


# execution variants (mode, pool, graphs): one kernel per event; persistent with
# sorted pools (default 256, 512/1024 per 256-thread block, 256 per 128-thread
# block, 64 per warp), cycles replayed as CUDA graphs or launched one by one;
# one particle per thread in registers; the monolithic segment kernel (mode 2)
VARIANTS = [(0, 0, 0), (1, 0, 0), (1, 0, -1), (1, 512, 0), (1, 1024, 0), (1, 2256, 0),
            (1, 64, 0), (1, -1, 0), (2, 0, 0)]
FEW = [(0, 0, 0), (1, 0, 0), (1, -1, -1), (2, 0, 0)]


def _eigen_parity(mcgb, pb, mode, pool=0, graphs=0):
    ncyc = pb["run"]["inactive"] + pb["run"]["active"]
    c = gpu_run(pb, mode=mode, pool=pool, graphs=graphs)
    o = oracle_run(pb)
    gk, gc, gm = c.get_cycle_k(ncyc)
    ok, oc, om = o.cycle_k(ncyc)
    assert gm.tolist() == om.tolist()
    assert rel_close(gk, ok, SUM_RTOL) and rel_close(gc, oc, SUM_RTOL)
    assert_same_histories(c.get_histories(), o.histories())
    gb, ob = c.get_bank(), o.bank()
    assert np.array_equal(gb["parent"], ob["parent"]) and np.array_equal(gb["child"], ob["child"])
    assert np.array_equal(gb["xyz"], ob["xyz"]) and np.array_equal(gb["mat"], ob["mat"])
    for t in range(len(pb["tallies"])):
        gmean, gsd = c.get_tally(t)
        omean, osd = o.tally(t)
        assert rel_close(gmean, omean, SUM_RTOL, 1e-300)
        assert rel_close(gsd, osd, 1e-6, 1e-14)
    gkk, okk = c.get_k(), o.k()
    for key in ["k", "k_col", "k_analog"]:
        assert abs(gkk[key] - okk[key]) <= SUM_RTOL * abs(okk[key])
    cnt_g, cnt_o = c.get_counters(), o.counters()
    for key in ["collisions", "crossings", "leaks", "lost", "capped"]:
        assert cnt_g[key] == cnt_o[key], key
    return c, o


@pytest.mark.parametrize("mode,pool,graphs", VARIANTS)
def test_pin_cell_eigen_parity(mcgb, mode, pool, graphs):
    _eigen_parity(mcgb, W.pin_cell_mg(n=3000, inactive=3, active=5), mode, pool, graphs)


@pytest.mark.parametrize("mode,pool,graphs", FEW)
def test_lattice_eigen_parity(mcgb, mode, pool, graphs):
    _eigen_parity(mcgb, W.c5g7_like_lattice(n=4000, inactive=2, active=3), mode, pool, graphs)


@pytest.mark.parametrize("mode,pool,graphs", FEW)
def test_ce_pin_eigen_parity(mcgb, mode, pool, graphs):
    _eigen_parity(mcgb, W.ce_pin_cell(n=600, inactive=1, active=2, npts=5000, nres=40), mode,
                  pool, graphs)


def test_stepwise_cycles_equal_one_call(mcgb):
    """begin + cycles in several calls (graphs and launches mixed) = one run call."""
    pb = W.pin_cell_mg(n=3000, inactive=2, active=4)
    import paper_2501_05440_gb300 as m
    ref = gpu_run(pb, mode=1)
    c = m.load_problem(m.Context(mode=1, record_histories=True), pb)
    c.eigen_begin(3000, 2, 4, pb["run"]["seed"])
    for k in (1, 2, 3):
        c.eigen_cycles(k)
    c.eigen_finish()
    assert c.get_cycle_k(6)[2].tolist() == ref.get_cycle_k(6)[2].tolist()
    assert_same_histories(c.get_histories(), ref.get_histories())
    assert c.get_k()["k"] == pytest.approx(ref.get_k()["k"], rel=1e-12)


def _fixed_parity(mcgb, pb, mode, pool=0, graphs=0):
    c = gpu_run(pb, mode=mode, pool=pool, graphs=graphs)
    o = oracle_run(pb)
    assert_same_histories(c.get_histories(), o.histories())
    gb, ob = c.get_bank(), o.bank()
    assert np.array_equal(gb["parent"], ob["parent"]) and np.array_equal(gb["xyz"], ob["xyz"])
    for t in range(len(pb["tallies"])):
        gmean, gsd = c.get_tally(t)
        omean, osd = o.tally(t)
        assert rel_close(gmean, omean, SUM_RTOL, 1e-300)
        assert rel_close(gsd, osd, 1e-6, 1e-14)
    cg, co = c.get_counters(), o.counters()
    for key in ["histories", "collisions", "crossings", "leaks", "lost", "generations"]:
        assert cg[key] == co[key], key


@pytest.mark.parametrize("mode,pool,graphs", FEW)
def test_slab_fixed_source_parity(mcgb, mode, pool, graphs):
    _fixed_parity(mcgb, W.diff_slab(n=5000, batches=10), mode, pool, graphs)


@pytest.mark.parametrize("mode,pool,graphs", FEW)
def test_box_fixed_source_parity(mcgb, mode, pool, graphs):
    for pb in W.batch_boxes(nproblems=4, nmin=500, nmax=3000)[:4]:
        _fixed_parity(mcgb, pb, mode, pool, graphs)


def test_one_collision_and_absorber_parity(mcgb):
    for pb in [W.one_collision_slab(n=5000), W.absorbing_slab_beam(n=5000)]:
        _fixed_parity(mcgb, pb, 0)


@pytest.mark.parametrize("mode,pool,graphs", FEW)
def test_ce_infinite_medium_eigen_parity(mcgb, mode, pool, graphs):
    E = np.array([W.E_MIN, 1.0, W.E_MAX])
    nuc = lambda A, sc, cc, sf, nu: {"A": A, "E": E, "sig_s": np.full(3, sc), "sig_c": np.full(3, cc),
                                     "sig_f": np.full(3, sf), "nu": nu}
    pb = W.ce_infinite_eigen([nuc(235.0, 4.0, 1.0, 2.0, 2.43), nuc(1.0, 3.0, 0.5, 0.0, 0.0)],
                             [0.02, 0.04], n=3000, inactive=2, active=3)
    _eigen_parity(mcgb, pb, mode, pool, graphs)


@pytest.mark.parametrize("mode,pool,graphs", FEW + [(1, 64, 0), (1, 512, 0)])
def test_ce_free_gas_eigen_parity(mcgb, mode, pool, graphs):
    """Free-gas thermal scattering in a k-eigenvalue run without time
    dependence (the pool instantiations without the particle clock; the
    other free-gas cases are time dependent): a fissile nuclide in hydrogen
    whose neutrons slow down into the thermal range."""
    E = np.array([W.E_MIN, 1.0, W.E_MAX])
    nuc = lambda A, sc, cc, sf, nu: {"A": A, "E": E, "sig_s": np.full(3, sc), "sig_c": np.full(3, cc),
                                     "sig_f": np.full(3, sf), "nu": nu}
    pb = W.ce_infinite_eigen([nuc(235.0, 4.0, 0.2, 0.4, 2.43), nuc(1.0, 20.0, 0.01, 0.0, 0.0)],
                             [0.002, 0.06], n=2000, inactive=1, active=2)
    pb["free_gas"] = {"kT": 0.0253}
    c, o = _eigen_parity(mcgb, pb, mode, pool, graphs)
    del pb["free_gas"]
    cold = oracle_run(pb).histories()
    assert np.any(cold["rng_end"] != c.get_histories()["rng_end"]), "free gas never sampled"


@pytest.mark.parametrize("mode,pool,graphs", FEW)
def test_ce_fixed_energy_eigen_parity(mcgb, mode, pool, graphs):
    """The problem of the oracle's fixed-energy closed form (nuclides of mass
    ~1e9 with cross sections that vary over the fission spectrum's energies):
    histories, banks, tallies and k equal to the oracle's."""
    from tests.test_oracle_ce_fixed_energy import _nuclides
    E = np.geomspace(W.E_MIN, W.E_MAX, 4001)
    pb = W.ce_infinite_eigen(_nuclides(E), [0.02, 0.03], n=3000, inactive=1, active=2, seed=11)
    _eigen_parity(mcgb, pb, mode, pool, graphs)


@pytest.mark.parametrize("radius", [0.6299, 0.63])
@pytest.mark.parametrize("mode,pool,graphs", [(0, 0, 0), (1, 0, 0)])
def test_lattice_tight_pins_parity(mcgb, radius, mode, pool, graphs):
    """Pins nearly filling their element (r = 0.6299 of a 0.63 half pitch: the
    fuel cell is proven inside, so its flights skip the lattice walls and root
    planes) and touching it (r = 0.63: nothing skipped) -- histories equal the
    oracle's, which always evaluates every surface."""
    pb = W.c5g7_like_lattice(n=4000, inactive=2, active=3)
    pb["surfaces"][4]["coef"][2] = radius
    _eigen_parity(mcgb, pb, mode, pool, graphs)


# Root boundaries that reach inside the lattice's elements: z-planes bounding a
# lattice of finite height, and a reflective x-plane through the first column's
# pin centres.  A particle in a fuel pin can reach them before it leaves the
# pin.  Radius 0.54: the fuel cell is inside its element, so its flights skip
# the lattice walls (and root surfaces only where none of them cuts an
# element); radius 0.63 touches the element and nothing is skipped.
SMALL_LATTICES = {
    "z-planes": dict(z_planes=(-3.0, 3.0, "reflect", "vacuum")),
    "x-plane-through-pins": dict(x_plane=(0.63, "reflect")),
    "both": dict(x_plane=(0.63, "reflect"), z_planes=(-2.0, 2.0, "vacuum", "reflect")),
}


@pytest.mark.parametrize("radius", [0.54, 0.63])
@pytest.mark.parametrize("name", sorted(SMALL_LATTICES))
@pytest.mark.parametrize("mode,pool,graphs", [(0, 0, 0), (1, 0, 0), (2, 0, 0)])
def test_lattice_root_boundaries_inside_elements(mcgb, name, radius, mode, pool, graphs):
    pb = W.small_lattice(n=4000, inactive=2, active=3, r=radius, **SMALL_LATTICES[name])
    _eigen_parity(mcgb, pb, mode, pool, graphs)
