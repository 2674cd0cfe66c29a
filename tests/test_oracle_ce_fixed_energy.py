"""Pin of the oracle's continuous-energy eigenvalue transport with energy-
dependent cross sections (Sec. 4's continuous-energy physics, Sec. 1's power
iteration), by a closed form that holds for any tabulated data.

Every nuclide is made so heavy (A ~ 1e9) that an elastic scattering leaves
the neutron's energy unchanged to ~1e-8, so a history keeps the energy it was
born with.  Its expected number of fission sites is then, over its
collisions, nuSigma_f(E) / Sigma_a(E) (the collisions until absorption
number Sigma_t / Sigma_a on average, each banking nuSigma_f / Sigma_t), and
the births of every generation follow the fission spectrum, so every
estimate of k has the expectation

    k = int chi(E) g(E) dE,   g(E) = sum_i N_i nu_i sigma_f,i(E) / sum_i N_i (sigma_c,i + sigma_f,i)(E),

chi the Maxwellian of temperature 1.33 MeV conditioned on E <= 20 MeV (the
oracle's reading of the spectrum), the sigma's lin-lin interpolated in E
between the tabulated points.  The integral is taken by Gauss-Legendre
quadrature on every interval of the table (a ratio of two linear functions
times the Maxwellian: exact to rounding at 16 nodes).  The fission cross
section grows in proportion to E over 0.1-10 MeV, where the spectrum lives,
beside a larger capture cross section with a bump at 0.5 MeV, so that a wrong spectrum
temperature, a nu taken from the other nuclide, absorption without fission,
or a fission yield per total instead of per absorption cross section moves k
by many standard deviations (checked below).
"""
import numpy as np
import pytest

import workloads as W

T_FIS = 1.33e6


def _nuclides(E):
    lE = np.log(E / 5.0e5)
    fis = {"A": 1.0e9, "E": E, "nu": 2.43,
           "sig_s": np.full_like(E, 4.0),
           "sig_f": 0.05 + 1.0 * (E / 1.0e6),
           "sig_c": 3.0 + 2.0 * np.exp(-(lE / 0.3) ** 2)}
    mod = {"A": 2.0e9, "E": E, "nu": 2.9,
           "sig_s": np.full_like(E, 8.0),
           "sig_f": np.zeros_like(E),
           "sig_c": 0.3 * (1.0e6 / E) ** 0.2}
    return [fis, mod]


def _spectrum_mean(E, num, den, T):
    """int chi g / int chi over [E_0, E_n] for g = num / den, num and den
    piecewise linear on the grid E, chi(E) ~ sqrt(E) exp(-E / T)."""
    x, w = np.polynomial.legendre.leggauss(16)
    a, b = E[:-1, None], E[1:, None]
    e = 0.5 * (b - a) * x[None, :] + 0.5 * (b + a)
    ww = 0.5 * (b - a) * w[None, :]
    t = (e - a) / (b - a)
    g = ((1 - t) * num[:-1, None] + t * num[1:, None]) / ((1 - t) * den[:-1, None] + t * den[1:, None])
    chi = np.sqrt(e) * np.exp(-e / T)
    return float(np.sum(ww * chi * g) / np.sum(ww * chi))


def _expected(nucs, dens, T=T_FIS, nu_swap=False, per_total=False, no_fission_absorption=False):
    E = nucs[0]["E"]
    nus = [n["nu"] for n in nucs][::-1] if nu_swap else [n["nu"] for n in nucs]
    num = sum(d * nu * n["sig_f"] for d, nu, n in zip(dens, nus, nucs))
    if per_total:
        den = sum(d * (n["sig_s"] + n["sig_c"] + n["sig_f"]) for d, n in zip(dens, nucs))
    elif no_fission_absorption:
        den = sum(d * n["sig_c"] for d, n in zip(dens, nucs))
    else:
        den = sum(d * (n["sig_c"] + n["sig_f"]) for d, n in zip(dens, nucs))
    return _spectrum_mean(E, num, den, T)


@pytest.mark.parametrize("strict", [False, True])
def test_ce_fixed_energy_k_closed_form(orc, strict):
    E = np.geomspace(W.E_MIN, W.E_MAX, 4001)
    nucs, dens = _nuclides(E), [0.02, 0.03]
    pb = W.ce_infinite_eigen(nucs, dens, n=20_000, inactive=1, active=20, seed=11)
    k = orc.Oracle(pb, strict=strict).run().k()
    want = _expected(nucs, dens)
    for key in ("k", "k_col", "k_analog"):
        assert abs(k[key] - want) < 4.0 * k[key + "_sd"], (key, k[key], k[key + "_sd"], want)
    # the pin tells these readings apart: each is > 8 standard deviations off
    sd = max(k["k_sd"], k["k_col_sd"], k["k_analog_sd"])
    for wrong in (_expected(nucs, dens, T=1.2895e6), _expected(nucs, dens, nu_swap=True),
                  _expected(nucs, dens, per_total=True),
                  _expected(nucs, dens, no_fission_absorption=True)):
        assert abs(wrong - want) > 8.0 * sd, (wrong, want, sd)


def test_quadrature_against_sampling():
    """The quadrature itself, against a direct average of g over Maxwellian
    energies drawn by numpy (Gamma(3/2, T)) and rejected above 20 MeV."""
    E = np.geomspace(W.E_MIN, W.E_MAX, 4001)
    nucs, dens = _nuclides(E), [0.02, 0.03]
    num = sum(d * n["nu"] * n["sig_f"] for d, n in zip(dens, nucs))
    den = sum(d * (n["sig_c"] + n["sig_f"]) for d, n in zip(dens, nucs))
    rng = np.random.default_rng(3)
    e = rng.gamma(1.5, T_FIS, 4_000_000)
    e = e[e <= W.E_MAX]
    g = np.interp(e, E, num) / np.interp(e, E, den)
    want = _spectrum_mean(E, num, den, T_FIS)
    assert abs(g.mean() - want) < 5.0 * g.std() / np.sqrt(len(g))
