"""Pins of the oracle's time-dependent fixed-source mode against closed forms.

A pulse of neutrons at t = 0 in an infinite medium has the population
N(t) = expm(A t) q, A = (Sigma_s^T + chi nuSigma_f^T - diag Sigma_t) V,
V = diag(v_g): reactions of group g' happen at rate Sigma v_g' N_g' (one group: exp(v (nuSigma_f - Sigma_a) t)).  A tally with time
bins scores the mean population per source neutron in each bin, so its exact
value is the bin average A^-1 (expm(A b) - expm(A a)) q / (b - a).  Speeds in
continuous energy are checked against the 2200 m/s thermal-neutron value
(v(E) = 2.2e5 cm/s sqrt(E / 0.0253 eV)), independent of the constants the
oracle uses.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as W

pytestmark = pytest.mark.usefixtures("orc")


def _mat(sigma_t, sigma_s, nu_sigma_f, chi):
    return {"sigma_t": np.asarray(sigma_t, float), "sigma_s": np.asarray(sigma_s, float),
            "nu_sigma_f": np.asarray(nu_sigma_f, float), "chi": np.asarray(chi, float)}


def _bin_average(A, q, edges):
    """Exact bin averages of expm(A t) q over consecutive edges (A invertible)."""
    Ainv = np.linalg.inv(A)
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        out.append(Ainv @ (scipy.linalg.expm(A * b) - scipy.linalg.expm(A * a)) @ q / (b - a))
    return np.array(out).T          # [group, time bin]


def _check(mean, sd, exact, nsig=5.0):
    mean, sd, exact = (np.asarray(x, float) for x in (mean, sd, exact))
    assert np.all(np.abs(mean - exact) <= nsig * sd + 1e-12 * np.abs(exact).max()), \
        (mean, exact, sd)


def _run(orc, pb):
    o = orc.Oracle(pb)
    o.run()
    mean, sd = o.tally(0)
    return o, mean[0], sd[0]          # the single material bin: [group or E bin, time bin]


def test_one_group_decay(orc):
    m = _mat([0.5], [[0.2]], [0.0], [1.0])
    v = 1.0e6
    edges = np.linspace(0.0, 1.0e-5, 11)
    pb = W.time_pulse_mg(m, [1.0], [1.0 / v], t_cut=1.0e-5, t_edges=edges, n=20_000)
    o, mean, sd = _run(orc, pb)
    exact = _bin_average(np.array([[-0.3 * v]]), np.array([1.0]), edges)
    _check(mean, sd, exact)
    c = o.counters()
    # survivors to the cutoff: binomial with p = exp(-Sigma_a v t_cut)
    p = np.exp(-3.0)
    n = pb["run"]["n"]
    assert abs(c["time_cut"] / n - p) < 5 * np.sqrt(p * (1 - p) / n)
    assert c["leaks"] == 0 and c["lost"] == 0


def test_one_group_multiplying(orc):
    # nuSigma_f 0.4 > Sigma_a 0.25: N(t) = exp(v (0.4 - 0.25) t)
    m = _mat([0.5], [[0.25]], [0.4], [1.0])
    v = 1.0e6
    edges = np.linspace(0.0, 1.0e-5, 6)
    pb = W.time_pulse_mg(m, [1.0], [1.0 / v], t_cut=1.0e-5, t_edges=edges, n=10_000)
    o, mean, sd = _run(orc, pb)
    exact = _bin_average(np.array([[0.15 * v]]), np.array([1.0]), edges)
    _check(mean, sd, exact)
    assert o.counters()["generations"] > 3


def test_two_groups_distinct_speeds(orc):
    sig_t = [0.4, 1.0]
    sig_s = [[0.1, 0.2], [0.0, 0.6]]
    nusf = [0.0, 0.5]
    chi = [1.0, 0.0]
    v = np.array([1.0e7, 1.0e5])
    edges = np.array([0.0, 1e-7, 3e-7, 1e-6, 3e-6, 1e-5, 3e-5, 1e-4, 2e-4])
    pb = W.time_pulse_mg(_mat(sig_t, sig_s, nusf, chi), [1.0, 0.0], 1.0 / v, t_cut=2e-4,
                         t_edges=edges, n=20_000)
    o, mean, sd = _run(orc, pb)
    M = np.array(sig_s).T + np.outer(chi, nusf) - np.diag(sig_t)
    A = M @ np.diag(v)
    exact = _bin_average(A, np.array([1.0, 0.0]), edges)
    _check(mean, sd, exact)
    # swapping the group speeds must be detectable at this sample size
    wrong = _bin_average(M @ np.diag(v[::-1]), np.array([1.0, 0.0]), edges)
    assert np.any(np.abs(mean - wrong) > 8 * sd)


def test_cutoff_ends_scores(orc):
    m = _mat([0.5], [[0.2]], [0.0], [1.0])
    edges = np.linspace(0.0, 2.0e-5, 9)
    pb = W.time_pulse_mg(m, [1.0], [1.0e-6], t_cut=1.0e-5, t_edges=edges, n=4_000)
    o, mean, sd = _run(orc, pb)
    assert np.all(mean[0, 4:] == 0.0) and np.all(mean[0, :4] > 0.0)
    c = o.counters()
    assert c["time_cut"] > 0
    h = o.histories()
    assert set(np.unique(h["fate"]).tolist()) <= {0, 5}        # absorbed or reached the cutoff


def _v_thermal_anchor(E):
    return 2.2e5 * np.sqrt(E / 0.0253)


def test_ce_speed_pure_capture(orc):
    sig_c, dens, E0 = 2.0, 0.05, 1.0
    lam = dens * sig_c * _v_thermal_anchor(E0)
    edges = np.linspace(0.0, 2.0e-5, 9)
    pb = W.time_pulse_ce(sig_c, E0, t_cut=2.0e-5, t_edges=edges, density=dens, n=20_000)
    o, mean, sd = _run(orc, pb)
    exact = _bin_average(np.array([[-lam]]), np.array([1.0]), edges)
    # the anchor and the physical constants agree to 2e-4: far inside the statistics
    _check(mean, sd, exact)


def test_ce_one_over_v_capture_with_scattering(orc):
    """1/v capture makes Sigma_c v constant, so the population decays as
    exp(-N a v(1 eV) t) whatever the scattering does to the energies."""
    a, dens = 1.0, 0.05                       # sigma_c(E) = a / sqrt(E / 1 eV) barns
    E = np.geomspace(W.E_MIN, W.E_MAX, 4000)
    pb = W.time_pulse_ce(1.0, 1.0e6, t_cut=5.0e-5, t_edges=np.linspace(0.0, 5.0e-5, 6),
                         A=1.0, sig_s=20.0, density=dens, n=10_000)
    nuc = pb["nuclides"][0]
    nuc["E"], nuc["sig_s"] = E, np.full_like(E, 20.0)
    nuc["sig_c"], nuc["sig_f"] = a / np.sqrt(E), np.zeros_like(E)
    o, mean, sd = _run(orc, pb)
    lam = dens * a * _v_thermal_anchor(1.0)
    edges = np.asarray(pb["tallies"][0]["time_edges"])
    exact = _bin_average(np.array([[-lam]]), np.array([1.0]), edges)
    _check(mean, sd, exact)
    assert o.counters()["collisions"] > 10 * pb["run"]["n"]


def test_ce_one_over_v_capture_with_free_gas(orc):
    """Free-gas scattering (upscatter included) leaves Sigma_c v constant under
    1/v capture: the same exponential decay holds from a thermal source."""
    a, dens = 1.0, 0.05
    E = np.geomspace(W.E_MIN, W.E_MAX, 4000)
    pb = W.time_pulse_ce(1.0, 0.0253, t_cut=5.0e-5, t_edges=np.linspace(0.0, 5.0e-5, 6),
                         A=1.0, sig_s=20.0, density=dens, n=10_000)
    nuc = pb["nuclides"][0]
    nuc["E"], nuc["sig_s"] = E, np.full_like(E, 20.0)
    nuc["sig_c"], nuc["sig_f"] = a / np.sqrt(E), np.zeros_like(E)
    pb["free_gas"] = {"kT": 0.0253}
    o, mean, sd = _run(orc, pb)
    lam = dens * a * _v_thermal_anchor(1.0)
    edges = np.asarray(pb["tallies"][0]["time_edges"])
    _check(mean, sd, _bin_average(np.array([[-lam]]), np.array([1.0]), edges))


def test_time_is_fixed_source_only(orc):
    pb = W.pin_cell_mg(n=100, inactive=1, active=1)
    pb["time"] = {"t0": 0.0, "t_cut": 1e-5, "inv_v": np.full(pb["G"], 1e-6)}
    o = orc.Oracle(pb)
    with pytest.raises(orc.OracleError):
        o.run()
