"""GPU checks beyond the small parity cases: derivatives, batching, autograd,
full-size runs sampled history by history, error paths and degenerate inputs."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests.gpu_util import assert_same_histories, gpu_run, rel_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcgb():
    import paper_2501_05440_gb300 as m
    m.build()
    return m


def _close_vec(a, b, rtol):
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    scale = max(np.abs(b).max(), 1e-300)
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + 1e-12 * scale)


@pytest.mark.parametrize("mode,pool", [(0, 0), (1, 0), (1, -1)])
def test_replay_derivatives_match_oracle(mcgb, mode, pool):
    pb = W.diff_slab(n=10, shield_len=8.0)
    n, seed, det = 4000, 77, pb["detector_cell"]
    G, nm = pb["G"], len(pb["materials"])
    w = np.random.default_rng(1).uniform(0.5, 2.0, G)
    c = mcgb.load_problem(mcgb.Context(mode=mode, pool=pool), pb)
    tally = c.forward_fixed(n, seed, det)
    g = c.backward_fixed(w, nm)
    o = Oracle(pb, strict=True).grad(n=n, seed=seed, cell=det, weights=w)
    assert rel_close(tally, o["tally"], 1e-9, 1e-300)
    for key in ["sigma_t", "sigma_s", "nu_sigma_f"]:
        assert _close_vec(g[key], o[key], 1e-8), key
    # zero-valued parameters take no score on both sides
    for m in range(nm):
        zero = pb["materials"][m]["sigma_s"] == 0
        assert np.all(g["sigma_s"][m][zero] == 0.0)
    # a second backward with other weights on the same forward pass
    w2 = np.ones(G)
    g2 = c.backward_fixed(w2, nm)
    o2 = Oracle(pb, strict=True).grad(n=n, seed=seed, cell=det, weights=w2)
    assert _close_vec(g2["sigma_t"], o2["sigma_t"], 1e-8)


def test_absorbing_slab_derivative_closed_form_on_gpu(mcgb):
    import math
    sig, x, L = 0.7, 3.0, 2.0
    pb = W.absorbing_slab_beam(sigma_t=sig, thickness=x, det_len=L)
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    n = 400000
    c.forward_fixed(n, 3, 1)
    g = c.backward_fixed([1.0], 2)
    exact = -x * L * math.exp(-sig * x)
    p = math.exp(-sig * x)
    sd = x * L * math.sqrt(p * (1 - p) / n)
    assert abs(g["sigma_t"][0, 0] - exact) < 5 * sd


def test_autograd_function(mcgb):
    import torch

    from paper_2501_05440_gb300.autograd import detector_tally
    pb = W.diff_slab(n=10, shield_len=8.0)
    n, seed, det = 3000, 5, pb["detector_cell"]
    st = torch.tensor(np.array([m["sigma_t"] for m in pb["materials"]]), requires_grad=True)
    ss = torch.tensor(np.array([m["sigma_s"] for m in pb["materials"]]), requires_grad=True)
    nf = torch.tensor(np.array([m["nu_sigma_f"] for m in pb["materials"]]), requires_grad=True)
    y = detector_tally(pb, st, ss, nf, n, seed, det)
    c = torch.linspace(0.5, 1.5, pb["G"], dtype=torch.float64)
    (y * c).sum().backward()
    o = Oracle(pb, strict=True).grad(n=n, seed=seed, cell=det, weights=c.numpy())
    assert rel_close(y.detach().numpy(), o["tally"], 1e-9, 1e-300)
    assert _close_vec(st.grad.numpy(), o["sigma_t"], 1e-8)
    assert _close_vec(ss.grad.numpy(), o["sigma_s"], 1e-8)
    assert _close_vec(nf.grad.numpy(), o["nu_sigma_f"], 1e-8)


def test_autograd_function_cuda_tensors(mcgb):
    """CUDA tensors take the device-pointer calls (no host copies of any array)
    and give the host-array path's results; a second forward with changed
    cross sections uses the updated device tables."""
    import torch

    from paper_2501_05440_gb300.autograd import detector_tally
    pb = W.diff_slab(n=10, shield_len=8.0)
    n, seed, det = 3000, 5, pb["detector_cell"]
    dev = torch.device("cuda", 0)
    st0 = np.array([m["sigma_t"] for m in pb["materials"]])
    ss0 = np.array([m["sigma_s"] for m in pb["materials"]])
    nf0 = np.array([m["nu_sigma_f"] for m in pb["materials"]])
    c = torch.linspace(0.5, 1.5, pb["G"], dtype=torch.float64)
    eng = None
    for scale in (1.0, 1.1):
        st = torch.tensor(st0 * scale, device=dev, requires_grad=True)
        ss = torch.tensor(ss0, device=dev, requires_grad=True)
        nf = torch.tensor(nf0, device=dev, requires_grad=True)
        if eng is None:
            eng = mcgb.load_problem(mcgb.Context(mode=1), pb)
        y = detector_tally(pb, st, ss, nf, n, seed, det, engine=eng)
        assert y.is_cuda
        (y * c.to(dev)).sum().backward()
        assert st.grad.is_cuda and ss.grad.is_cuda and nf.grad.is_cuda
        p2 = copy.deepcopy(pb)
        for m in range(len(pb["materials"])):
            p2["materials"][m]["sigma_t"] = st0[m] * scale
        o = Oracle(p2, strict=True).grad(n=n, seed=seed, cell=det, weights=c.numpy())
        assert rel_close(y.detach().cpu().numpy(), o["tally"], 1e-9, 1e-300), scale
        assert _close_vec(st.grad.cpu().numpy(), o["sigma_t"], 1e-8), scale
        assert _close_vec(ss.grad.cpu().numpy(), o["sigma_s"], 1e-8), scale
        assert _close_vec(nf.grad.cpu().numpy(), o["nu_sigma_f"], 1e-8), scale


def test_device_material_update_rejects_invalid(mcgb):
    import torch
    pb = W.diff_slab(n=10, shield_len=8.0)
    G, nm = pb["G"], len(pb["materials"])
    eng = mcgb.load_problem(mcgb.Context(mode=1), pb)
    st = torch.tensor(np.array([m["sigma_t"] for m in pb["materials"]]), device="cuda")
    ss = torch.tensor(np.array([m["sigma_s"] for m in pb["materials"]]), device="cuda")
    nf = torch.tensor(np.array([m["nu_sigma_f"] for m in pb["materials"]]), device="cuda")
    st[1, 2] = 0.5 * ss[1, 2].sum()          # scattering above total
    eng.update_material_mg_dev(0, nm, st.data_ptr(), ss.data_ptr(), nf.data_ptr())
    out = torch.empty(G, dtype=torch.float64, device="cuda")
    with pytest.raises(mcgb.McgbError) as e:
        eng.forward_fixed_dev(1000, 1, pb["detector_cell"], out.data_ptr())
    assert e.value.code == -1
    # the flag is cleared: valid tables run
    st[1, 2] = 2.0 * ss[1, 2].sum() + 0.1
    eng.update_material_mg_dev(0, nm, st.data_ptr(), ss.data_ptr(), nf.data_ptr())
    eng.forward_fixed_dev(1000, 1, pb["detector_cell"], out.data_ptr())
    assert torch.all(out >= 0)


@pytest.mark.parametrize("pool", [0, -1])
def test_batch_equals_standalone_runs(mcgb, pool):
    probs = W.batch_boxes(nproblems=6, nmin=300, nmax=4000)
    b = mcgb.Batch(pool=pool)
    ctxs = []
    for p in probs:
        c = mcgb.load_problem(mcgb.Context(), p)
        ctxs.append(c)
        b.add_problem(c, p["run"]["n"], p["run"]["batches"], p["run"]["seed"])
    b.run()
    for i, (c, p) in enumerate(zip(ctxs, probs)):
        c.run()
        bm, bs = b.tally(i)
        cm, cs = c.get_tally()
        om, osd = Oracle(p, strict=True).run().tally()
        assert rel_close(bm, cm, 1e-9, 1e-300) and rel_close(bm, om, 1e-9, 1e-300), i
    cnt = b.counters()
    assert cnt["histories"] >= sum(p["run"]["n"] for p in probs)


def test_batch_autotune_and_cache(mcgb, tmp_path, monkeypatch):
    probs = W.batch_boxes(nproblems=4, nmin=300, nmax=2000)
    b = mcgb.Batch()
    for p in probs:
        c = mcgb.load_problem(mcgb.Context(), p)
        b.add_problem(c, p["run"]["n"], p["run"]["batches"], p["run"]["seed"])
    t = b.autotune(budget_ms=3000)
    assert t["pool"] in (-1, 32, 64, 128, 256, 512, 1024, 2256, 2512) and t["blocks_per_sm"] >= 1 and t["ms"] > 0
    t2 = b.autotune(budget_ms=3000)      # served from the cache
    assert t2 == t
    b.run(t)


@pytest.mark.parametrize("name", ["lattice", "ce"])
def test_full_size_first_cycle_sampled(mcgb, name):
    """Full configuration size (1e6 particles), first cycle: sampled histories
    recomputed one by one by the oracle must be identical."""
    pb = W.c5g7_like_lattice(n=1_000_000, inactive=0, active=1) if name == "lattice" else \
        W.ce_pin_cell(n=1_000_000, inactive=0, active=1)
    c = gpu_run(pb, mode=1)
    h = c.get_histories()
    assert len(h["n_coll"]) == 1_000_000
    idx = np.sort(np.random.default_rng(3).choice(1_000_000, 1500 if name == "lattice" else 400,
                                                  replace=False))
    ho = Oracle(pb, strict=True).histories_by_index(idx)
    assert_same_histories({k: v[idx] for k, v in h.items()}, ho)
    # properties at full size: the bank holds exactly the sites the histories counted
    assert int(h["n_fis"].sum()) == c.get_cycle_k(1)[2][0]
    assert np.all(h["fate"] >= 0)


def test_error_paths(mcgb):
    # bank overflow is reported, not written out of bounds
    pb = W.pin_cell_mg(n=5000, inactive=1, active=1)
    c = mcgb.load_problem(mcgb.Context(mode=1, bank_factor=0.01), pb)
    with pytest.raises(mcgb.McgbError) as e:
        c.run()
    assert e.value.code == -5
    # a gap in the geometry loses particles
    gap = W.pin_cell_mg(n=2000, inactive=0, active=1)
    gap["cells"] = gap["cells"][:1]          # drop the moderator cell
    gap["source"]["box"] = [-0.3, 0.3, -0.3, 0.3, 0.0, 0.0]
    c = mcgb.load_problem(mcgb.Context(), gap)
    with pytest.raises(mcgb.McgbError) as e:
        c.run()
    assert e.value.code == -6
    # no fissile cell for a fissile-only source
    nf = W.pin_cell_mg(n=100, inactive=0, active=1)
    for m in nf["materials"]:
        m["nu_sigma_f"] = np.zeros(nf["G"])
    c = mcgb.load_problem(mcgb.Context(), nf)
    with pytest.raises(mcgb.McgbError) as e:
        c.run()
    assert e.value.code == -2
    # invalid arguments
    c = mcgb.Context()
    with pytest.raises(mcgb.McgbError) as e:
        c.add_surface(9, [0.0], 0)
    assert e.value.code == -1
    with pytest.raises(mcgb.McgbError) as e:
        mcgb.Context(pool=300)
    assert e.value.code == -1
    c = mcgb.load_problem(mcgb.Context(), W.pin_cell_mg(n=10))
    with pytest.raises(mcgb.McgbError) as e:
        c.run_eigenvalue(-5, 1, 1, 1)
    assert e.value.code == -1


def test_degenerate_sizes(mcgb):
    from oracle import OracleError
    # tiny eigenvalue runs: either both implementations finish identically, or
    # both stop on an empty fission bank (MCGB_E_STATE)
    for n, seed in [(1, 1), (1, 2), (3, 5), (7, 11)]:
        for mode in (0, 1):
            pb = W.pin_cell_mg(n=n, inactive=0, active=2)
            pb["run"]["seed"] = seed
            g_err = o_err = None
            try:
                c = gpu_run(pb, mode=mode)
            except mcgb.McgbError as e:
                g_err = e.code
            try:
                o = Oracle(pb, strict=True).run()
            except OracleError:
                o_err = -2
            assert g_err == o_err, (n, seed, mode, g_err, o_err)
            if g_err is None:
                assert c.get_cycle_k(2)[2].tolist() == o.cycle_k(2)[2].tolist()
                assert_same_histories(c.get_histories(), o.histories())
    # one source history, fixed source
    pb = W.diff_slab(n=1, batches=1)
    c = gpu_run(pb, mode=1)
    o = Oracle(pb, strict=True).run()
    assert_same_histories(c.get_histories(), o.histories())
    # no tallies at all
    pb = W.pin_cell_mg(n=500, inactive=0, active=2)
    pb["tallies"] = []
    c = gpu_run(pb, mode=1)
    assert c.get_k()["k"] > 0


def test_full_size_graph_cycles_equal_launches(mcgb):
    """The bench's launch configuration at full size: cycles replayed as CUDA
    graphs give the bank sizes, last-cycle histories and bank of cycles
    launched one by one (which the smaller parity tests pin to the oracle)."""
    pb = W.c5g7_like_lattice(n=1_000_000, inactive=1, active=2)
    runs = []
    for graphs in (0, -1):
        c = mcgb.load_problem(mcgb.Context(mode=1, record_histories=True, graphs=graphs), pb)
        c.run()
        runs.append(c)
    g, l = runs
    assert g.get_cycle_k(3)[2].tolist() == l.get_cycle_k(3)[2].tolist()
    assert_same_histories(g.get_histories(), l.get_histories())
    bg, bl = g.get_bank(), l.get_bank()
    assert np.array_equal(bg["parent"], bl["parent"]) and np.array_equal(bg["xyz"], bl["xyz"])
    assert abs(g.get_k()["k"] - l.get_k()["k"]) <= 1e-12 * abs(l.get_k()["k"])


def test_event_mode_flight_timing(mcgb):
    """Event mode reports the device time of each cycle's first flight launch
    and the state bytes one particle moves in it (lattice, multigroup, no
    z-planes, no time: 121 B loaded, 53 B stored); other modes report none."""
    pb = W.c5g7_like_lattice(n=20_000, inactive=1, active=2)
    c = mcgb.load_problem(mcgb.Context(mode=0), pb)
    c.run()
    t = c.get_event_timing()
    assert t["launches"] == 3 and t["particles"] == 3 * 20_000
    assert t["advance_ms"] > 0.0
    assert t["bytes_per_particle"] == 174.0
    c = mcgb.load_problem(mcgb.Context(mode=1), pb)
    c.run()
    assert c.get_event_timing()["launches"] == 0


def test_bench_batch_at_full_size(mcgb):
    """The benchmark's 64-problem batch (1e3-1e6 histories each, 8.7e6 in all)
    in its autotuned persistent launch equals 64 standalone runs problem by
    problem, and sampled generation-0 histories of the 16 largest problems
    equal the oracle's, one by one."""
    probs = W.batch_boxes()
    b = mcgb.Batch()
    ctxs = []
    for p in probs:
        c = mcgb.load_problem(mcgb.Context(mode=1, record_histories=True), p)
        ctxs.append(c)
        b.add_problem(c, p["run"]["n"], p["run"]["batches"], p["run"]["seed"])
    t = b.autotune(budget_ms=3000)
    b.run(t)
    big = set(np.argsort([p["run"]["n"] for p in probs])[-16:].tolist())
    rng = np.random.default_rng(17)
    for i, (c, p) in enumerate(zip(ctxs, probs)):
        c.run()
        bm, bs = b.tally(i)
        cm, cs = c.get_tally()
        assert rel_close(bm, cm, 1e-9, 1e-300), i
        assert rel_close(bs, cs, 1e-6, 1e-14), i
        if i in big:
            n = p["run"]["n"]
            idx = np.sort(rng.choice(n, 150, replace=False))
            h = c.get_histories()
            ho = Oracle(p, strict=True).histories_by_index(idx)
            assert_same_histories({k: np.asarray(v)[idx] for k, v in h.items()}, ho)
    assert b.counters()["histories"] >= sum(p["run"]["n"] for p in probs)
