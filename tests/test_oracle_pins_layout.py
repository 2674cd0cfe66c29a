"""Pins of oracle functions that the closed-form transport checks cannot see.

* Systematic resampling (power iteration, Sec. 4): the site of source j is
  floor((j + xi) M / N), clamped to M - 1, checked against exact rationals.
* The lattice-filter tally bin ix + nx * iy (the per-pin tallies of the
  paper's C5G7 runs, Sec. 4): a beam through a void lattice.
* Continuous-energy tally bins: energies exactly on the edges, the top edge
  closing the last bin.
* The strict logarithm's table: ln(1 + j/256) correctly rounded.

Each pin is also run against a plausible mistake (computed here in Python) to
show that the mistake would fail it.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.usefixtures("orc")


def _exact_site(j, n, M, N):
    k = math.floor((Fraction(j) + Fraction(n, 2 ** 53)) * M / N)
    return min(k, M - 1)


def _cases():
    rng = np.random.default_rng(12)
    out = []
    for _ in range(400):
        N = int(rng.integers(1, 3_000_000))
        M = int(rng.integers(1, 3 * N + 1))          # M < N and M > N both occur
        j = int(rng.integers(0, N))
        n = int(rng.integers(1, 2 ** 53 + 1))
        out.append((j, n, M, N))
    # xi = 1 (n = 2^53): the last source reaches M itself, clamped to M - 1
    for M, N in [(5, 7), (7, 5), (1, 1), (1000, 999), (999, 1000), (3, 3)]:
        out.append((N - 1, 2 ** 53, M, N))
        out.append((0, 2 ** 53, M, N))
    # (j + xi) M / N an exact integer just below and at a site boundary
    out += [(3, 2 ** 52, 2, 7), (6, 2 ** 53, 4, 7), (1, 2 ** 52, 2, 3)]
    return out


def test_resampling_site_exact(orc):
    cases = _cases()
    got = [orc.site_index(*c) for c in cases]
    want = [_exact_site(*c) for c in cases]
    assert got == want
    assert all(0 <= g < c[2] for g, c in zip(got, cases))
    # mistakes this pin catches: M and N swapped, no clamp
    swapped = [min(math.floor((Fraction(j) + Fraction(n, 2 ** 53)) * N / M), M - 1)
               for j, n, M, N in cases]
    assert swapped != want
    unclamped = [math.floor((Fraction(j) + Fraction(n, 2 ** 53)) * M / N) for j, n, M, N in cases]
    assert unclamped != want


def test_resampling_site_counts(orc):
    """Systematic sampling with xi < 1 takes each of the M sites floor(N/M) or
    ceil(N/M) times, and every site when M <= N.  (At xi = 1 exactly, a draw of
    probability 2^-53, every index moves up by M/N and the clamp gives the last
    site to the last source as well.)"""
    for M, N, n in [(7, 20, 123456789), (20, 7, 2 ** 40), (1000, 1000, 2 ** 53 - 1), (3, 1000, 1)]:
        sites = np.array([orc.site_index(j, n, M, N) for j in range(N)])
        counts = np.bincount(sites, minlength=M)
        assert counts.sum() == N
        assert counts.min() >= N // M and counts.max() <= -(-N // M)
        if M <= N:
            assert counts.min() >= 1
        assert np.all(np.diff(sites) >= 0)
    at_one = [orc.site_index(j, 2 ** 53, 1000, 1000) for j in range(1000)]
    assert at_one[:3] == [1, 2, 3] and at_one[-2:] == [999, 999]


@pytest.mark.parametrize("strict", [False, True])
@pytest.mark.parametrize("row", [0, 1])
def test_lattice_tally_bin_layout(orc, strict, row):
    nx, ny, pitch = 3, 2, 1.25
    pb = W.void_lattice_beam(nx=nx, ny=ny, pitch=pitch, row=row)
    mean, sd = orc.Oracle(pb, strict=strict).run().tally(0)
    assert mean.shape == (nx * ny, 1)
    want = np.zeros(nx * ny)
    for ix in range(nx):
        want[ix + nx * row] = pitch
    assert np.allclose(mean[:, 0], want, rtol=1e-12, atol=0.0)
    # the transposed layout ix * ny + iy would put the track elsewhere
    transposed = np.zeros(nx * ny)
    for ix in range(nx):
        transposed[ix * ny + row] = pitch
    assert not np.allclose(transposed, want)


@pytest.mark.parametrize("strict", [False, True])
def test_ce_energy_bin_edges(orc, strict):
    edges = np.array([1.0e-3, 1.0, 1.0e3, 1.0e6])
    L = 2.0
    cases = [(1.0e-3, 0), (1.0, 1), (1.0e3, 2), (1.0e6, 2), (0.5, 0), (2.0e5, 2),
             (1.0e-4, None), (1.5e6, None)]
    for E, b in cases:
        mean, _ = orc.Oracle(W.ce_void_beam(E, edges, length=L), strict=strict).run().tally(0)
        want = np.zeros(len(edges) - 1)
        if b is not None:
            want[b] = L
        # E = 1e6 on the top edge: an open top edge would score nothing
        assert np.allclose(mean[0], want, rtol=1e-12, atol=0.0), (E, mean[0])


def test_log_table_correctly_rounded(orc):
    """The strict logarithm's table holds ln(1 + j/256) in 57 fraction bits,
    rounded to the nearest integer (checked against 200-bit mpmath)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    scale = mpmath.mpf(2) ** 57
    for j in range(256):
        want = int(mpmath.nint(mpmath.log(1 + mpmath.mpf(j) / 256) * scale))
        assert orc.log_table_q57(j) == want, j
    # rounding down instead of to nearest would differ
    assert any(int(mpmath.floor(mpmath.log(1 + mpmath.mpf(j) / 256) * scale)) != orc.log_table_q57(j)
               for j in range(256))