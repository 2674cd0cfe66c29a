"""Pins of the oracle's transport against closed forms and exact enumeration.

* infinite medium: k = dominant eigenvalue of (diag Sigma_t - Sigma_s^T)^-1 chi nuSigma_f^T
  and the flux per source neutron is (diag Sigma_t - Sigma_s^T)^-1 chi;
* one group: k = nuSigma_f / Sigma_a;
* absorbing slab: uncollided transmission exp(-Sigma_t x), detector track length
  L exp(-Sigma_t x) and its Sigma_t derivative -x L exp(-Sigma_t x);
* one-collision slab: the joint law of (region, outcome, fission count) of the
  first collision, enumerated exactly;
* CE lookup: values at grid points are the table values, and linear in E between.
"""
import math

import numpy as np
import pytest
from scipy import stats

import workloads as W
from oracle import Oracle


def _fuel(seed=1):
    return W.pin_cell_mg(seed=seed)["materials"][0]


def test_kinf_seven_groups(orc):
    mat = _fuel()
    A = np.diag(mat["sigma_t"]) - mat["sigma_s"].T
    F = np.outer(mat["chi"], mat["nu_sigma_f"])
    kinf = max(abs(np.linalg.eigvals(np.linalg.solve(A, F))))
    o = Oracle(W.infinite_medium_mg(mat, n=20000, inactive=5, active=40)).run()
    k = o.k()
    assert abs(k["k"] - kinf) < 5 * k["k_sd"], (k, kinf)
    assert abs(k["k_col"] - kinf) < 5 * k["k_col_sd"]
    assert abs(k["k_analog"] - kinf) < 5 * k["k_analog_sd"]
    # flux per source neutron (material filter: both bins hold the same material)
    mean, sd = o.tally(0)
    phi = mean.sum(axis=0)
    phisd = np.sqrt((sd ** 2).sum(axis=0))
    exact = np.linalg.solve(A, mat["chi"])
    z = (phi - exact) / phisd
    assert np.all(np.abs(z) < 5), z


def test_kinf_one_group(orc):
    mat = {"sigma_t": np.array([1.0]), "sigma_s": np.array([[0.6]]),
           "nu_sigma_f": np.array([0.5]), "chi": np.array([1.0])}
    o = Oracle(W.infinite_medium_mg(mat, n=20000, inactive=3, active=30)).run()
    k = o.k()
    assert abs(k["k"] - 0.5 / 0.4) < 5 * k["k_sd"]
    # one group: every collision yields mu = 0.5 exactly, so k_C is exact
    assert abs(k["k_col"] - 1.25) < 5 * k["k_col_sd"] + 1e-12


def test_absorbing_slab_transmission(orc):
    sig, x, L, n = 0.7, 3.0, 2.0, 200000
    pb = W.absorbing_slab_beam(sigma_t=sig, thickness=x, det_len=L, n=n)
    o = Oracle(pb).run()
    p = math.exp(-sig * x)
    leaks = o.counters()["leaks"]
    assert abs(leaks - n * p) < 5 * math.sqrt(n * p * (1 - p))
    mean, sd = o.tally(0)
    det = mean[1, 0]
    assert abs(det - L * p) < 5 * sd[1, 0]
    h = o.histories()
    # every history either leaks after 2 crossings or is absorbed in the slab
    assert np.all((h["n_cross"] == 2) | ((h["n_coll"] == 1) & (h["n_cross"] == 0)))


def test_absorbing_slab_derivative(orc):
    sig, x, L = 0.7, 3.0, 2.0
    pb = W.absorbing_slab_beam(sigma_t=sig, thickness=x, det_len=L)
    exact = -x * L * math.exp(-sig * x)
    vals = []
    for seed in range(8):
        g = Oracle(pb).grad(n=20000, seed=100 + seed, cell=1)
        vals.append(g["sigma_t"][0, 0])
        assert g["sigma_t"][1, 0] == 0.0          # void: zero-valued parameter takes no score
    vals = np.array(vals)
    # per history the estimator is -x L * [transmitted]
    p = math.exp(-sig * x)
    sd = x * L * math.sqrt(p * (1 - p) / (20000 * 8))
    assert abs(vals.mean() - exact) < 5 * sd, (vals.mean(), exact)


def test_one_collision_enumeration(orc):
    pb = W.one_collision_slab(n=200000)
    m0, m1 = pb["materials"]
    o = Oracle(pb).run()
    h = o.histories()
    # exact joint law of the first (only) collision for a group-0 beam
    s0, s1 = m0["sigma_t"][0], m1["sigma_t"][0]
    P = {}
    pr = {0: 1 - math.exp(-s0 * 1.0), 1: math.exp(-s0) * (1 - math.exp(-s1 * 1.5))}
    P[("esc", -1, 0)] = math.exp(-s0 - 1.5 * s1)
    for r, m in ((0, m0), (1, m1)):
        st = m["sigma_t"][0]
        mu = m["nu_sigma_f"][0] / st
        fl, fr = math.floor(mu), mu - math.floor(mu)
        nfis = {fl: 1 - fr, fl + 1: fr} if fr > 0 else {fl: 1.0}
        outs = {("abs", -1): 1 - m["sigma_s"][0].sum() / st}
        for gp in range(2):
            outs[("sc", gp)] = m["sigma_s"][0][gp] / st
        for (kind, gp), po in outs.items():
            for nf, pn in nfis.items():
                P[(f"{kind}{r}", gp, nf)] = pr[r] * po * pn
    assert abs(sum(P.values()) - 1) < 1e-12
    keys = list(P)
    counts = dict.fromkeys(keys, 0)
    for nc, nx, fate, g, nf in zip(h["n_coll"], h["n_cross"], h["fate"], h["g_end"], h["n_fis"]):
        if nc == 0:
            k = ("esc", -1, 0)
        else:
            r = int(nx)
            k = (f"abs{r}", -1, int(nf)) if fate == 0 else (f"sc{r}", int(g), int(nf))
        counts[k] += 1
    obs = np.array([counts[k] for k in keys], float)
    exp = np.array([P[k] for k in keys]) * len(h["n_coll"])
    keep = exp > 0
    assert obs[~keep].sum() == 0
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4, (chi2, dict(zip(keys, obs)), P)


def test_ce_lookup_grid_points_and_linearity(orc):
    pb = W.ce_pin_cell(n=10, npts=2000, nres=20)
    # one-nuclide materials so that the macroscopic value is N sigma_i
    nuc = pb["nuclides"][3]
    pb = dict(pb, materials=[{"nuclides": [3], "density": [2.0]}, {"nuclides": [0], "density": [1.0]}])
    o = Oracle(pb)
    idx = np.linspace(0, len(nuc["E"]) - 1, 57).astype(int)
    for j in idx:
        E = nuc["E"][j]
        st, nusf, ss, sf = o.ce_lookup(0, float(E))
        assert st == 2.0 * ((nuc["sig_s"][j] + nuc["sig_c"][j]) + nuc["sig_f"][j])
        assert ss == 2.0 * nuc["sig_s"][j]
    rng = np.random.default_rng(2)
    for E in np.exp(rng.uniform(math.log(1e-5), math.log(2e7), 300)):
        st, nusf, ss, sf = o.ce_lookup(0, float(E))
        ref_s = np.interp(E, nuc["E"], nuc["sig_s"])
        ref_f = np.interp(E, nuc["E"], nuc["sig_f"])
        assert abs(ss - 2.0 * ref_s) <= 1e-12 * abs(2.0 * ref_s)
        assert abs(nusf - 2.0 * nuc["nu"] * ref_f) <= 1e-12 * abs(2.0 * nuc["nu"] * ref_f)


def test_absorbing_slab_self_tally_derivative(orc):
    """Tally on the absorbing slab itself: E[T] = (1 - e^{-S x})/S, so
    dE[T]/dS = x e^{-S x}/S - (1 - e^{-S x})/S^2.  Per history the estimator
    is (1/S - s) s for a collision at depth s and -x^2 for transmission."""
    sig, x = 0.7, 3.0
    pb = W.absorbing_slab_beam(sigma_t=sig, thickness=x, det_len=2.0)
    e = math.exp(-sig * x)
    t_exact = (1 - e) / sig
    d_exact = x * e / sig - (1 - e) / sig ** 2
    vals, tals = [], []
    for seed in range(8):
        g = Oracle(pb).grad(n=20000, seed=300 + seed, cell=0)
        vals.append(g["sigma_t"][0, 0])
        tals.append(g["tally"][0])
    vals, tals = np.array(vals), np.array(tals)
    assert abs(tals.mean() - t_exact) < 5 * tals.std(ddof=1) / math.sqrt(8)
    assert abs(vals.mean() - d_exact) < 5 * vals.std(ddof=1) / math.sqrt(8), (vals.mean(), d_exact)
