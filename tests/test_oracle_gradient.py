"""Pin of the oracle's likelihood-ratio derivatives against common-random-number
central finite differences (statistical: both estimators are unbiased for the
same derivative, so their difference is tested against both variances)."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle

PARAMS = [("sigma_t", 1, (0,)), ("sigma_t", 0, (2,)), ("sigma_s", 1, (0, 0)),
          ("sigma_s", 1, (0, 1)), ("nu_sigma_f", 0, (0,)), ("sigma_t", 2, (3,))]


def _small_slab():
    return W.diff_slab(n=10, shield_len=6.0, source_len=3.0, det_len=3.0)


def test_lr_matches_crn_finite_differences(orc):
    pb = _small_slab()
    n, seeds, h = 20000, 6, 5e-3
    det = pb["detector_cell"]
    lr = {p: [] for p in PARAMS}
    fd = {p: [] for p in PARAMS}
    for k in range(seeds):
        seed = 1000 + k
        g = Oracle(pb).grad(n=n, seed=seed, cell=det)
        for p in PARAMS:
            key, m, idx = p
            lr[p].append(g[key][(m,) + idx])
            theta = pb["materials"][m][key][idx]
            tp = Oracle(W.scaled(pb, m, key, idx, 1 + h)).grad(n=n, seed=seed, cell=det)["tally"].sum()
            tm = Oracle(W.scaled(pb, m, key, idx, 1 - h)).grad(n=n, seed=seed, cell=det)["tally"].sum()
            fd[p].append((tp - tm) / (2 * h * theta))
    for p in PARAMS:
        a, b = np.array(lr[p]), np.array(fd[p])
        z = (a.mean() - b.mean()) / np.sqrt(a.var(ddof=1) / seeds + b.var(ddof=1) / seeds)
        assert abs(z) < 5, (p, a.mean(), b.mean(), z)
        # the derivative is resolved: not just two noisy zeros
        assert abs(a.mean()) > 2 * a.std(ddof=1) / np.sqrt(seeds), (p, a)
