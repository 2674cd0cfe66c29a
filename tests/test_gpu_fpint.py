"""The transport's float64 square root, quotient and reciprocal, computed on
the integer and float32 pipes, against numpy's IEEE operations.

The library evaluates every square root and division of a history (surface
distances, isotropic directions, direction reciprocals, collision kinematics)
with its own correctly rounded routines instead of the hardware's.  IEEE 754
fixes the round-to-nearest result of both operations uniquely, so the values
must be bit-identical to numpy's (which calls the host's IEEE instructions) on
every input: random significands over the whole exponent range, significands
next to the ends of their binade, inputs with exact results, and the special
operands (zero, subnormal, infinite, NaN) that take the hardware path.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2501_05440_gb300 as m
    m.build()
    return m.Context()


def _random_doubles(rng, n, emin=1, emax=2046):
    """Bit patterns with random exponents and significands, an eighth of them
    with all-zero, all-one or near-end significands."""
    e = rng.integers(emin, emax + 1, size=n, dtype=np.uint64)
    m = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    kind = rng.integers(0, 16, size=n)
    small = rng.integers(0, 16, size=n, dtype=np.uint64)
    full = np.uint64((1 << 52) - 1)
    m = np.where(kind == 0, np.uint64(0), m)
    m = np.where(kind == 1, full, m)
    m = np.where(kind == 2, small, m)
    m = np.where(kind == 3, full - small, m)
    bits = (e << np.uint64(52)) | m
    return bits.view(np.float64)


def _same(got, want):
    """Bit-identical, NaN payloads aside."""
    g, w = np.asarray(got), np.asarray(want)
    nan = np.isnan(w)
    assert np.array_equal(np.isnan(g), nan)
    gb, wb = g.view(np.uint64), w.view(np.uint64)
    bad = np.nonzero((gb != wb) & ~nan)[0]
    assert len(bad) == 0, (len(bad), g[bad[:4]], w[bad[:4]])


def _check(ctx, a, b):
    out = ctx.fpint_ops(a, b)
    with np.errstate(all="ignore"):
        _same(out[:, 0], np.sqrt(a))
        _same(out[:, 1], a / b)
        _same(out[:, 2], 1.0 / b)


def test_random_significands_whole_range(ctx):
    rng = np.random.default_rng(20250105)
    for _ in range(4):
        n = 1 << 22
        a = _random_doubles(rng, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
        b = _random_doubles(rng, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
        _check(ctx, np.abs(a), b)
        _check(ctx, a, b)


def test_transport_ranges(ctx):
    """Magnitudes the transport meets: direction cosines, squared distances
    and discriminants of a pin-sized cylinder, cross sections."""
    rng = np.random.default_rng(7)
    n = 1 << 22
    u = rng.uniform(-1.0, 1.0, n)
    disc = rng.uniform(0.0, 0.5, n) ** 3
    sig = 10.0 ** rng.uniform(-3, 3, n)
    _check(ctx, disc, u)
    _check(ctx, sig, disc + 1e-300)
    _check(ctx, 1.0 - u * u, sig)


def test_exact_and_near_binade_ends(ctx):
    """Perfect squares, exact quotients, powers of two, and significands at
    both ends of a binade (where the root's significand rounds up to the next
    binade and the quotient's normalisation shift changes)."""
    k = np.arange(1, 200001, dtype=np.float64)
    _check(ctx, k * k, k)
    _check(ctx, 3.0 * k, 3.0 * np.ones_like(k))
    p2 = np.ldexp(1.0, np.arange(-1022, 1024))
    _check(ctx, p2, p2[::-1].copy())
    top = np.nextafter(np.ldexp(1.0, np.arange(-1020, 1023)), 0.0)   # largest of each binade
    _check(ctx, top, np.ldexp(1.0, np.arange(-1020, 1023)) * 1.0000000000000002)
    _check(ctx, top, top)


def test_special_operands(ctx):
    """Zero, subnormal, infinite and NaN operands, and quotients that
    overflow or are subnormal, take the hardware operation and agree too."""
    tiny = np.float64(5e-324)
    vals = np.array([0.0, -0.0, tiny, -tiny, 2.2250738585072014e-308, 2.225073858507201e-308,
                     1.7976931348623157e308, np.inf, -np.inf, np.nan, 1.0, -1.0, 0.5, 2.0,
                     1e-300, 1e300, 3.0, -7.5], dtype=np.float64)
    a = np.repeat(vals, len(vals))
    b = np.tile(vals, len(vals))
    _check(ctx, a, b)


def test_empty_input(ctx):
    out = ctx.fpint_ops(np.zeros(0), np.zeros(0))
    assert out.shape == (0, 3)
