"""The oracle's two arithmetic modes differ only in rounding.

The plain mode evaluates each definition as written; the strict mode adopts
the CUDA library's rounding conventions.  Both take the same random draws, so
a history can differ only where a rounding difference flips a discrete
decision (a flight ending within an ulp of a surface, say): nearly every
history, every bank size here, and the estimates must agree.  Every pin of
the other test files runs in the plain mode; the ones below run both.
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.usefixtures("orc")


def _same_fraction(a, b):
    keys = ["n_coll", "n_cross", "n_fis", "fate", "g_end", "rng_end"]
    same = np.ones(len(a["n_coll"]), bool)
    for k in keys:
        same &= np.asarray(a[k]) == np.asarray(b[k])
    return same.mean()


@pytest.mark.parametrize("make", [lambda: W.pin_cell_mg(n=4000, inactive=2, active=4),
                                  lambda: W.c5g7_like_lattice(n=3000, inactive=1, active=2),
                                  lambda: W.ce_pin_cell(n=400, inactive=1, active=2, npts=4000,
                                                        nres=30)])
def test_plain_and_strict_histories_agree(make):
    pb = make()
    ncyc = pb["run"]["inactive"] + pb["run"]["active"]
    p = Oracle(pb).run()
    s = Oracle(pb, strict=True).run()
    mp, ms = p.cycle_k(ncyc)[2], s.cycle_k(ncyc)[2]
    assert mp.tolist() == ms.tolist()
    assert _same_fraction(p.histories(), s.histories()) >= 0.999
    kp, ks = p.k(), s.k()
    assert abs(kp["k"] - ks["k"]) <= 1e-9 * abs(ks["k"])


def test_plain_mode_differs_in_rounding_only():
    """The modes are not the same program: on the lattice their flight
    distances, and so the k track-length estimates, differ in the last bits."""
    pb = W.c5g7_like_lattice(n=3000, inactive=0, active=1)
    kp = Oracle(pb).run().cycle_k(1)[0][0]
    ks = Oracle(pb, strict=True).run().cycle_k(1)[0][0]
    assert kp != ks and abs(kp - ks) <= 1e-12 * abs(ks)


@pytest.mark.parametrize("strict", [False, True])
def test_kinf_both_modes(strict):
    mat = W.pin_cell_mg(seed=1)["materials"][0]
    A = np.diag(mat["sigma_t"]) - mat["sigma_s"].T
    F = np.outer(mat["chi"], mat["nu_sigma_f"])
    kinf = max(abs(np.linalg.eigvals(np.linalg.solve(A, F))))
    o = Oracle(W.infinite_medium_mg(mat, n=20000, inactive=5, active=30), strict=strict).run()
    k = o.k()
    assert abs(k["k"] - kinf) < 5 * k["k_sd"], (k, kinf)
