"""Pins of the oracle's free-gas elastic scattering (constant cross section).

Reference distribution, derived independently of the sampling steps: a
collision picks the target velocity with density proportional to the relative
speed r(x, mu) times the Maxwellian x^2 exp(-x^2) (speeds in units of the
target's thermal speed, mu the cosine between target and neutron directions,
uniform a priori); for isotropic scattering in the centre-of-mass frame the
lab energy is then uniform between E (|V| - w)^2 / y^2 and E (|V| + w)^2 / y^2,
with V the centre-of-mass velocity and w = A r / (A + 1).  The outgoing-energy
CDF is that mixture integrated by quadrature; for A = 1 it must equal the
Wigner-Wilkins proton-gas kernel in closed form, which pins the quadrature.
"""
import numpy as np
import pytest
from scipy import integrate, special, stats

pytestmark = pytest.mark.usefixtures("orc")
KT = 0.0253


def _ww_cdf(E, kT):
    """Wigner-Wilkins kernel (A = 1), normalised per collision, as a CDF in E'."""
    I = lambda a, b: integrate.quad(lambda e: special.erf(np.sqrt(e / kT)), a, b)[0]
    IE = I(0.0, E)
    tot = IE + kT * special.erf(np.sqrt(E / kT))

    def F(Ep):
        if Ep <= E:
            return I(0.0, Ep) / tot
        return (IE + kT * special.erf(np.sqrt(E / kT)) * (1.0 - np.exp((E - Ep) / kT))) / tot
    return F


def _quad_cdf(E, A, kT, nx=1500, nmu=400):
    """Outgoing-energy CDF from the target-velocity mixture (independent quadrature)."""
    y = np.sqrt(A * E / kT)
    x, wx = np.polynomial.legendre.leggauss(nx)
    x = 3.5 * (x + 1.0)                 # [0, 7]
    wx = 3.5 * wx
    mu, wmu = np.polynomial.legendre.leggauss(nmu)
    X, MU = np.meshgrid(x, mu, indexing="ij")
    r = np.sqrt(np.maximum(X * X + y * y - 2.0 * X * y * MU, 0.0))
    dens = r * X * X * np.exp(-X * X) * np.outer(wx, wmu)
    dens /= dens.sum()
    V = np.sqrt(np.maximum(y * y + (A * X) ** 2 + 2.0 * A * X * y * MU, 0.0)) / (A + 1.0)
    w = A * r / (A + 1.0)
    lo, hi = E * (V - w) ** 2 / y ** 2, E * (V + w) ** 2 / y ** 2
    span = np.maximum(hi - lo, 1e-300)

    def F(Ep):
        return float((dens * np.clip((Ep - lo) / span, 0.0, 1.0)).sum())
    return F


def _tabulated(F, E):
    """F on a fine log grid of E', interpolated (the CDF is smooth)."""
    grid = np.concatenate([[0.0], np.geomspace(1e-6 * E, 60.0 * max(E, KT), 1500)])
    vals = np.array([F(g) for g in grid])
    return lambda x: np.interp(x, grid, vals)


def _samples(orc, E, A, kT, n, seed=3):
    s = orc.rng_stream(seed, 0)
    d = np.array([0.0, 0.0, 1.0])
    Ep = np.empty(n)
    mu = np.empty(n)
    for i in range(n):
        out, s = orc.free_gas(E, A, kT, d, s)
        Ep[i] = out[0]
        mu[i] = out[3]
        assert abs(out[1] ** 2 + out[2] ** 2 + out[3] ** 2 - 1.0) < 1e-12
    return Ep, mu


@pytest.mark.parametrize("E", [0.3 * KT, KT, 5.0 * KT])
def test_quadrature_matches_wigner_wilkins(E):
    Fq, Fw = _quad_cdf(E, 1.0, KT), _ww_cdf(E, KT)
    for Ep in np.geomspace(0.01 * KT, 20 * KT, 25):
        assert abs(Fq(Ep) - Fw(Ep)) < 2e-4, (E, Ep)


@pytest.mark.parametrize("A,E", [(1.0, 0.3 * KT), (1.0, 3.0 * KT), (16.0, KT), (235.0, 2 * KT)])
def test_outgoing_energy_distribution(orc, A, E):
    Ep, _ = _samples(orc, E, A, KT, 40_000)
    F = _tabulated(_quad_cdf(E, A, KT, nx=800, nmu=200), E)
    res = stats.kstest(Ep, F)
    assert res.pvalue > 1e-3, (A, E, res)


def test_fast_limit_is_target_at_rest(orc):
    # E >> kT: mean E'/E -> (A^2 + 1)/(A + 1)^2, mean mu_lab -> 2 / (3A)
    for A in (1.0, 16.0):
        E = 300.0 * KT
        Ep, mu = _samples(orc, E, A, KT, 20_000, seed=5)
        assert abs(Ep.mean() / E - (A * A + 1) / (A + 1) ** 2) < 0.01
        assert abs(mu.mean() - 2.0 / (3.0 * A)) < 0.015


def test_thermal_neutrons_gain_energy(orc):
    # far below kT the target's motion dominates: upscatter on average
    Ep, _ = _samples(orc, 0.05 * KT, 1.0, KT, 5_000, seed=7)
    assert Ep.mean() > 5 * 0.05 * KT
