"""Pins of the oracle's random-number stream against the generator's algebra.

The paper (Sec. 1) requires replicable streams on CPU and GPU without naming a
generator; the oracle uses the 63-bit LCG s' = (g s + 1) mod 2^63 with Brown's
skip-ahead.  These checks use exact Python integers, independent of the C code.
"""
import random

import numpy as np

G = 2806196910506780709
M = 1 << 63


def lcg_closed_form(s, n):
    """s_n = g^n s + (g^n - 1)/(g - 1) mod 2^63, the geometric sum taken exactly."""
    mod = (G - 1) * M
    gn = pow(G, n, mod)
    geo = (gn - 1) // (G - 1)
    return (gn % M * s + geo) % M


def test_next_matches_definition(orc):
    rnd = random.Random(1)
    for _ in range(2000):
        s = rnd.randrange(M)
        assert orc.rng_next(s) == (G * s + 1) % M


def test_skip_equals_sequential_steps(orc):
    s0 = 12345
    s = s0
    for n in range(1, 20001):
        s = orc.rng_next(s)
        if n % 997 == 0 or n < 50:
            assert orc.rng_skip(s0, n) == s


def test_skip_closed_form_large_strides(orc):
    rnd = random.Random(7)
    for _ in range(500):
        s = rnd.randrange(M)
        n = rnd.randrange(1 << 62)
        assert orc.rng_skip(s, n) == lcg_closed_form(s, n)
    # the period is 2^63
    assert orc.rng_skip(99, M) == 99
    assert orc.rng_skip(99, 0) == 99


def test_stream_start_and_composition(orc):
    seed = 1
    for i in [0, 1, 2, 17, 152916, (3 << 32) + 5]:
        assert orc.rng_stream(seed, i) == lcg_closed_form(seed, i * 152917 % M)
    a, b = 10**12 + 3, 7 * 10**15
    assert orc.rng_skip(orc.rng_skip(5, a), b) == orc.rng_skip(5, a + b)


def test_uniform_is_exact_and_in_unit_interval(orc):
    s = 2024
    xs = []
    for _ in range(20000):
        s = orc.rng_next(s)
        xi = orc.rng_xi(s)
        n = (s >> 10) + 1
        assert xi == n / 2.0**53
        xs.append(xi)
    xs = np.array(xs)
    assert xs.min() > 0.0 and xs.max() <= 1.0
    # first two moments of U(0,1) within 5 sigma
    assert abs(xs.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(xs))
    assert abs((xs ** 2).mean() - 1 / 3) < 5 * np.sqrt(4 / 45 / len(xs))
    assert orc.rng_xi(M - 1) == 1.0 and orc.rng_xi(0) == 2.0**-53
