"""Pin of the oracle's continuous-energy k-eigenvalue path (fission banking,
nuclide and reaction selection, resampling) against a closed form.

In an infinite medium whose cross sections do not depend on energy, every
collision banks nu sigma_f / sigma_t sites on average (nuclide picked with
probability N_i sigma_t,i / Sigma_t) and the history survives it with
probability Sigma_s / Sigma_t, so a history banks Sum N nu sigma_f /
Sum N (sigma_c + sigma_f) sites on average whatever the energies the
scatterings and the fission spectrum give: that ratio is k_inf, and the
analog, collision and track-length estimators all converge to it.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.usefixtures("orc")


def _nuc(A, s, c, f, nu):
    E = np.array([W.E_MIN, 1.0, W.E_MAX])
    return {"A": float(A), "E": E, "sig_s": np.full(3, float(s)), "sig_c": np.full(3, float(c)),
            "sig_f": np.full(3, float(f)), "nu": float(nu)}


def _infinite_ce(nucs, dens, n=20_000, inactive=2, active=30, seed=5):
    return W.ce_infinite_eigen(nucs, dens, n=n, inactive=inactive, active=active, seed=seed)


@pytest.mark.parametrize("A_mod", [1.0, 16.0])
def test_ce_infinite_medium_k(orc, A_mod):
    nucs = [_nuc(235.0, 4.0, 1.0, 2.0, 2.43), _nuc(A_mod, 3.0, 0.5, 0.0, 0.0)]
    dens = [0.02, 0.04]
    k_inf = (0.02 * 2.43 * 2.0) / (0.02 * (1.0 + 2.0) + 0.04 * 0.5)
    o = orc.Oracle(_infinite_ce(nucs, dens))
    o.run()
    k = o.k()
    for est, sd in (("k", "k_sd"), ("k_col", "k_col_sd"), ("k_analog", "k_analog_sd")):
        assert k[sd] > 0
        assert abs(k[est] - k_inf) <= 4.0 * k[sd], (est, k[est], k_inf, k[sd])


def test_ce_infinite_medium_k_sees_each_nuclides_nu(orc):
    # the fissile nuclide's nu is the only one that counts: doubling the
    # non-fissile nuclide's nu (it has no fission) leaves k unchanged, while
    # a k computed with a density-weighted mean nu would move by ~30%
    nucs = [_nuc(235.0, 4.0, 1.0, 2.0, 2.43), _nuc(16.0, 3.0, 0.5, 0.0, 5.0)]
    dens = [0.02, 0.04]
    k_inf = (0.02 * 2.43 * 2.0) / (0.02 * 3.0 + 0.04 * 0.5)
    o = orc.Oracle(_infinite_ce(nucs, dens, active=20))
    o.run()
    k = o.k()
    assert abs(k["k_analog"] - k_inf) <= 4.0 * k["k_analog_sd"]
