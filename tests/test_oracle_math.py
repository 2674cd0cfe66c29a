"""Pins of the oracle's elementary sampling steps against closed forms."""
import math

import numpy as np
import pytest

from scipy import special, stats


def xi_samples(orc, n, seed=77):
    s = seed
    out = np.empty(n)
    for i in range(n):
        s = orc.rng_next(s)
        out[i] = orc.rng_xi(s)
    return out


def test_log_against_libm(orc):
    xs = xi_samples(orc, 20000)
    extra = np.array([1.0, 0.5, 0.25, 2.0**-53, 2.0**-52, 1 - 2.0**-53, 0.75, 0.999, 1e-3, 3.0**-20])
    extra = np.round(extra * 2.0**53) / 2.0**53
    for x in np.concatenate([xs, extra]):
        got = orc.log(float(x))
        ref = math.log(x)
        # relative 2.5 ulp where |ln xi| >= 1, absolute 2 ulp of 1 nearer to 0
        tol = 2.5 * np.spacing(abs(ref)) if abs(ref) >= 1.0 else 2.0 * np.spacing(1.0)
        assert abs(got - ref) <= tol, (x, got, ref)
    assert orc.log(1.0) == 0.0
    assert orc.log(0.5) == -math.log(2.0)
    assert abs(orc.log(2.0**-53) + 53 * math.log(2.0)) <= 2 * np.spacing(37.0)


def test_isotropic_direction(orc):
    n = 20000
    s = 5
    d = np.empty((n, 3))
    for i in range(n):
        d[i], s = orc.iso_dir(s)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=4e-16)
    for k in range(3):
        # each cosine is U(-1, 1) on the unit sphere (Archimedes)
        assert stats.kstest(d[:, k], stats.uniform(-1, 2).cdf).pvalue > 1e-4
    # azimuth uniform
    phi = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-4


@pytest.mark.parametrize("A", [1.0, 16.0, 90.0, 235.0])
def test_elastic_target_at_rest(orc, A):
    n = 20000
    s = 11
    E = 1.0e6
    ratios, mulab = np.empty(n), np.empty(n)
    rng = np.random.default_rng(3)
    for i in range(n):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        out, s = orc.elastic(E, A, v, s)
        ratios[i] = out[0] / E
        mulab[i] = float(np.dot(out[1:], v))
        assert abs(np.linalg.norm(out[1:]) - 1.0) < 1e-12
    alpha = ((A - 1) / (A + 1)) ** 2
    assert ratios.min() >= alpha * (1 - 1e-12) and ratios.max() <= 1 + 1e-12
    # isotropic centre-of-mass scattering: E'/E ~ U(alpha, 1), mean (A^2+1)/(A+1)^2
    mean = (A * A + 1) / (A + 1) ** 2
    assert abs(ratios.mean() - mean) < 5 * (1 - alpha) / math.sqrt(12 * n)
    if A > 1:
        assert stats.kstest(ratios, stats.uniform(alpha, 1 - alpha).cdf).pvalue > 1e-4
    # mean lab cosine 2/(3A)
    assert abs(mulab.mean() - 2 / (3 * A)) < 5 * mulab.std() / math.sqrt(n)
    # the rotation puts the new direction exactly at mu_lab from the old one
    mucm = (ratios * (A + 1) ** 2 - (A * A + 1)) / (2 * A)
    pred = (1 + A * mucm) / np.sqrt(A * A + 2 * A * mucm + 1)
    ok = np.isfinite(pred) & (ratios > 1e-9)
    assert np.allclose(mulab[ok], pred[ok], atol=2e-6)


def test_maxwell_spectrum(orc):
    n = 20000
    s = 21
    e = np.empty(n)
    for i in range(n):
        e[i], s = orc.maxwell(s)
    T = 1.33e6
    assert e.min() >= 1e-5 and e.max() <= 2e7
    # chi(E) ~ sqrt(E) exp(-E/T): CDF is the regularised lower gamma P(3/2, E/T)
    assert stats.kstest(e, lambda x: special.gammainc(1.5, x / T)).pvalue > 1e-4
    assert abs(e.mean() - 1.5 * T) < 5 * math.sqrt(1.5) * T / math.sqrt(n)
