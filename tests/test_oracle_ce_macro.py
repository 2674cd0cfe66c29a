"""Pin of the macroscopic flight cross sections of a continuous-energy
material: interpolating the tabulated sums on the material's union grid must
give sum_i N_i sigma_i(E) with each nuclide interpolated lin-lin on its own
grid (np.interp here), up to rounding, at any energy and at the grid points."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.usefixtures("orc")


def _reference(pb, mat, E):
    m = pb["materials"][mat]
    st = np.zeros_like(E)
    nf = np.zeros_like(E)
    for nuc, dens in zip(m["nuclides"], m["density"]):
        u = pb["nuclides"][nuc]
        tot = np.asarray(u["sig_s"]) + np.asarray(u["sig_c"]) + np.asarray(u["sig_f"])
        st += dens * np.interp(E, u["E"], tot)
        nf += dens * u["nu"] * np.interp(E, u["E"], np.asarray(u["sig_f"]))
    return st, nf


@pytest.mark.parametrize("strict", [False, True])
def test_macro_table_equals_nuclide_sum(orc, strict):
    """strict: the per-material macroscopic table; plain: the nuclide sum at E"""
    pb = W.ce_pin_cell(n=100, npts=3000, nres=30)
    o = orc.Oracle(pb, strict=strict)
    rng = np.random.default_rng(4)
    E = np.exp(rng.uniform(np.log(W.E_MIN), np.log(W.E_MAX), 3000))
    E = np.concatenate([E, pb["nuclides"][3]["E"][::7], pb["nuclides"][0]["E"][::11]])
    for mat in (0, 1):
        st_ref, nf_ref = _reference(pb, mat, E)
        out = np.array([o.ce_lookup(mat, float(e)) for e in E])
        assert np.allclose(out[:, 0], st_ref, rtol=1e-11, atol=0), mat
        assert np.allclose(out[:, 1], nf_ref, rtol=1e-11, atol=1e-300), mat
