"""Seeded synthetic problem descriptions for event-based Monte Carlo transport.

This module only *describes* problems: geometry, cross-section tables, sources,
tallies and run settings, as plain Python dicts of numbers and numpy arrays.  It
holds none of the transport arithmetic.  Both the CPU oracle and the CUDA
library read the same descriptions through their own loaders.

The paper (Sec. 4) times a 3D C5G7 multigroup k-eigenvalue benchmark and a
continuous-energy infinite pin cell driven by OpenMC nuclear data.  Neither the
C5G7 geometry/cross sections nor the nuclear data are available here, so the
generators below build seeded stand-ins with the same structure: a 7-group
pin cell, a 51x51 lattice of 2x2 fuel assemblies plus a reflector band, and a
pin cell of four synthetic nuclides with 1/v capture and Breit-Wigner
resonances.  Two further workloads exercise batching of many small fixed-source
problems and cross-section derivatives on a slab.

Vocabulary (strings, so neither side shares enum values with the other):
  surface types  'px' 'py' 'pz' (coef[0] = plane position), 'plane'
                 (a, b, c, d for a x + b y + c z = d), 'cylz' (x0, y0, R),
                 'sphere' (x0, y0, z0, R)
  boundaries     'none' 'vacuum' 'reflect'
  cell fills     'material' or 'lattice'; cells list (surface, sense) pairs,
                 sense +1 for the side where the surface function is positive
  tally filters  'cell' (innermost cell), 'lattice' (element ix + nx*iy),
                 'material'; energy bins are the groups (MG) or 'edges' (CE)
"""
from __future__ import annotations

import copy
import math

import numpy as np

__all__ = [
    "mg_material", "kinf_mg", "pin_cell_mg", "c5g7_like_lattice", "ce_pin_cell",
    "batch_boxes", "diff_slab", "infinite_medium_mg", "absorbing_slab_beam",
    "one_collision_slab", "infinite_medium_fixed", "scaled", "with_run", "CONFIG_NAMES",
    "time_pulse_mg", "time_pulse_ce", "ce_time_pin", "void_lattice_beam", "ce_void_beam",
    "small_lattice",
]

CONFIG_NAMES = {
    0: "mg-pin-cell-7g-keff",
    1: "mg-c5g7-like-lattice-51x51-7g-keff",
    2: "ce-pin-cell-4nuclides-keff",
    3: "batch-64-fixed-source-boxes",
    4: "diff-slab-3region-7g-fixed-source",
}


# ----------------------------------------------------------------------------
# cross-section data
# ----------------------------------------------------------------------------
def kinf_mg(sigma_t, sigma_s, nu_sigma_f, chi):
    """Infinite-medium multiplication factor of one multigroup material.

    The balance (diag Sigma_t - Sigma_s^T) phi = chi (nuSigma_f . phi) / k has a
    rank-one fission operator, so k = nuSigma_f . (diag Sigma_t - Sigma_s^T)^-1 chi.
    Used here only to scale generated data into a target range.
    """
    a = np.diag(np.asarray(sigma_t, float)) - np.asarray(sigma_s, float).T
    return float(np.asarray(nu_sigma_f, float) @ np.linalg.solve(a, np.asarray(chi, float)))


def mg_material(rng, G, *, fissile, kinf=None, sigt=(0.2, 2.0), ratio=(0.5, 0.98),
                upscatter=True):
    """One seeded multigroup material.

    Sigma_t ~ U[sigt]; the scattering row sum is U[ratio] * Sigma_t; each row
    goes mostly to its own and lower-energy groups with geometric decay, and
    only the last two groups (groups 6-7 of 7) may scatter up, into groups
    G-3 .. g-1.  A fissile material gets chi on the first three groups and
    nuSigma_f scaled so that its infinite-medium k equals `kinf`.
    """
    sigma_t = rng.uniform(*sigt, size=G)
    r = rng.uniform(*ratio, size=G)
    sigma_s = np.zeros((G, G))
    for g in range(G):
        decay = rng.uniform(0.2, 0.6)
        w = np.zeros(G)
        for gp in range(g, G):
            w[gp] = decay ** (gp - g)
        if upscatter and G >= 4 and g >= G - 2:
            for gp in range(G - 3, g):
                w[gp] = rng.uniform(0.01, 0.1)
        sigma_s[g] = w / w.sum() * r[g] * sigma_t[g]
    nu_sigma_f = np.zeros(G)
    chi = np.zeros(G)
    if fissile:
        nf = min(3, G)
        chi[:nf] = rng.uniform(0.2, 1.0, size=nf)
        chi /= chi.sum()
        nu_sigma_f = rng.uniform(0.5, 1.5, size=G) * (sigma_t - sigma_s.sum(axis=1))
        if kinf is not None:
            nu_sigma_f *= kinf / kinf_mg(sigma_t, sigma_s, nu_sigma_f, chi)
    return {"sigma_t": sigma_t, "sigma_s": sigma_s, "nu_sigma_f": nu_sigma_f, "chi": chi}


# ----------------------------------------------------------------------------
# geometry helpers
# ----------------------------------------------------------------------------
def _surf(kind, coef, bc="none"):
    c = list(map(float, coef)) + [0.0] * (4 - len(coef))
    return {"type": kind, "coef": c, "bc": bc}


def _cell(universe, halfspaces, fill_kind, fill):
    return {"universe": int(universe), "surfs": [int(s) for s, _ in halfspaces],
            "senses": [int(x) for _, x in halfspaces], "fill_kind": fill_kind, "fill": int(fill)}


def _pin_geometry(half=0.63, r=0.54, bc="reflect"):
    """Square box [-half, half]^2 (infinite in z) around a z-cylinder at the origin."""
    surfaces = [_surf("cylz", [0.0, 0.0, r]),
                _surf("px", [-half], bc), _surf("px", [half], bc),
                _surf("py", [-half], bc), _surf("py", [half], bc)]
    box = [(1, +1), (2, -1), (3, +1), (4, -1)]
    cells = [_cell(0, [(0, -1)] + box, "material", 0),
             _cell(0, [(0, +1)] + box, "material", 1)]
    return surfaces, cells


def _eigen_run(n, inactive, active, seed):
    return {"mode": "eigen", "n": int(n), "inactive": int(inactive), "active": int(active),
            "seed": int(seed)}


def _fixed_run(n, seed, batches=50):
    return {"mode": "fixed", "n": int(n), "seed": int(seed), "batches": int(batches)}


# ----------------------------------------------------------------------------
# configuration 0: multigroup pin cell, k-eigenvalue
# ----------------------------------------------------------------------------
def pin_cell_mg(seed=1, n=10_000, inactive=10, active=20, G=7):
    """Cylinder r=0.54 in a 1.26x1.26 box, reflective on all sides, infinite in z.

    Two materials (fuel-like with k_inf in [1.0, 1.4], moderator-like), G groups,
    track-length flux tally per cell and group.
    """
    rng = np.random.default_rng([seed, 0])
    fuel = mg_material(rng, G, fissile=True, kinf=rng.uniform(1.0, 1.4))
    mod = mg_material(rng, G, fissile=False)
    surfaces, cells = _pin_geometry()
    return {
        "name": CONFIG_NAMES[0], "G": G, "surfaces": surfaces, "cells": cells, "lattices": [],
        "materials": [fuel, mod],
        "source": {"kind": "box", "box": [-0.63, 0.63, -0.63, 0.63, 0.0, 0.0],
                   "accept": "fissile", "energy": "chi", "direction": "iso"},
        "tallies": [{"filter": "cell"}],
        "run": _eigen_run(n, inactive, active, seed),
    }


def infinite_medium_mg(material, seed=3, n=20_000, inactive=5, active=20):
    """The pin-cell geometry with one material in both cells: an infinite medium."""
    G = len(material["sigma_t"])
    surfaces, cells = _pin_geometry()
    return {
        "name": "mg-infinite-medium", "G": G, "surfaces": surfaces, "cells": cells,
        "lattices": [], "materials": [copy.deepcopy(material), copy.deepcopy(material)],
        "source": {"kind": "box", "box": [-0.63, 0.63, -0.63, 0.63, 0.0, 0.0],
                   "accept": "fissile", "energy": "chi", "direction": "iso"},
        "tallies": [{"filter": "material"}],
        "run": _eigen_run(n, inactive, active, seed),
    }


# ----------------------------------------------------------------------------
# configuration 1: C5G7-shaped lattice, k-eigenvalue
# ----------------------------------------------------------------------------
def c5g7_like_lattice(seed=1, n=1_000_000, inactive=50, active=100, G=7, guide_per_assembly=25):
    """51x51 lattice (pitch 1.26): 2x2 fuel assemblies of 17x17 pins + 17-pin reflector band.

    Reflective on x=0 and y=0, vacuum on x=y=64.26, infinite in z.  Seven
    seeded materials: four fuels (k_inf in [1.0, 1.4]), a guide-tube filler, a
    moderator and a reflector.  Assembly (0,0) holds fuel 0, (1,0) fuel 1,
    (0,1) fuel 2, (1,1) fuel 3; each assembly has `guide_per_assembly` seeded
    guide/instrument positions.  Tally: per-pin (lattice element) per-group flux.
    """
    rng = np.random.default_rng([seed, 1])
    mats = [mg_material(rng, G, fissile=True, kinf=rng.uniform(1.0, 1.4)) for _ in range(4)]
    mats.append(mg_material(rng, G, fissile=False))                      # 4: guide tube
    mats.append(mg_material(rng, G, fissile=False, ratio=(0.9, 0.98)))   # 5: moderator
    mats.append(mg_material(rng, G, fissile=False, ratio=(0.9, 0.98)))   # 6: reflector
    pitch, nx = 1.26, 51
    width = pitch * nx
    surfaces = [_surf("px", [0.0], "reflect"), _surf("px", [width], "vacuum"),
                _surf("py", [0.0], "reflect"), _surf("py", [width], "vacuum"),
                _surf("cylz", [0.0, 0.0, 0.54])]
    cells = [_cell(0, [(0, +1), (1, -1), (2, +1), (3, -1)], "lattice", 0)]
    # universes 1..4: fuel pins, 5: guide tube pin, 6: reflector block
    for u, m in enumerate([0, 1, 2, 3, 4], start=1):
        cells.append(_cell(u, [(4, -1)], "material", m))
        cells.append(_cell(u, [(4, +1)], "material", 5))
    cells.append(_cell(6, [], "material", 6))
    univ = np.full((nx, nx), 6, dtype=np.int64)          # [iy, ix]
    for ay in range(2):
        for ax in range(2):
            fuel_u = 1 + (ax + 2 * ay)
            block = np.full(17 * 17, fuel_u)
            guides = rng.choice(17 * 17, size=guide_per_assembly, replace=False)
            block[guides] = 5
            univ[17 * ay:17 * ay + 17, 17 * ax:17 * ax + 17] = block.reshape(17, 17)
    lattice = {"x0": 0.0, "y0": 0.0, "pitch": pitch, "nx": nx, "ny": nx,
               "universes": univ.reshape(-1).tolist()}
    return {
        "name": CONFIG_NAMES[1], "G": G, "surfaces": surfaces, "cells": cells,
        "lattices": [lattice], "materials": mats,
        "source": {"kind": "box", "box": [0.0, 34 * pitch, 0.0, 34 * pitch, 0.0, 0.0],
                   "accept": "fissile", "energy": "chi", "direction": "iso"},
        "tallies": [{"filter": "lattice"}],
        "run": _eigen_run(n, inactive, active, seed),
    }


# ----------------------------------------------------------------------------
# configuration 2: continuous-energy pin cell, k-eigenvalue
# ----------------------------------------------------------------------------
E_MIN, E_MAX = 1.0e-5, 2.0e7          # eV
FUEL_235 = (3.5e-3, 4.5e-3)           # atom density ranges of the fuel (atoms/b-cm)
FUEL_90 = (1.0e-3, 2.0e-3)


def _ce_nuclide(rng, A, npts, fissile, sig_pot, a_c, a_f=0.0, nu=0.0, nres=200,
                split=(2.0, 2.0, 2.0)):
    """Pointwise cross sections on a log grid with a seeded sub-interval phase.

    Smooth part: constant potential scattering and 1/v capture (and 1/v fission
    for a fissile nuclide).  Resonances: `nres` single-level Breit-Wigner lines,
    E0 log-uniform in [1 eV, 1e5 eV], total width U[0.02, 0.5] eV * (E0/1 eV)^0.25,
    peak log-uniform in [10, 1e4] b, split into neutron / capture (/ fission) widths.
    """
    phase = rng.uniform(0.05, 0.95)
    k = np.arange(1, npts - 1, dtype=float)
    lo, hi = math.log(E_MIN), math.log(E_MAX)
    E = np.empty(npts)
    E[0], E[-1] = E_MIN, E_MAX
    E[1:-1] = np.exp(lo + (hi - lo) * (k - 1 + phase) / (npts - 2))
    sqrtE = np.sqrt(E)
    sig_s = np.full(npts, sig_pot)
    sig_c = a_c / sqrtE
    sig_f = a_f / sqrtE if fissile else np.zeros(npts)
    E0 = np.exp(rng.uniform(math.log(1.0), math.log(1.0e5), size=nres))
    gam = rng.uniform(0.02, 0.5, size=nres) * E0 ** 0.25
    peak = np.exp(rng.uniform(math.log(10.0), math.log(1.0e4), size=nres))
    parts = rng.dirichlet(list(split[:3]) if fissile else list(split[:2]), size=nres)
    for i in range(nres):
        x = 2.0 * (E - E0[i]) / gam[i]
        shape = peak[i] / (1.0 + x * x)
        sig_s += parts[i, 0] * shape
        sig_c += parts[i, 1] * shape * np.sqrt(E0[i] / E)
        if fissile:
            sig_f += parts[i, 2] * shape * np.sqrt(E0[i] / E)
    return {"A": float(A), "E": E, "sig_s": sig_s, "sig_c": sig_c, "sig_f": sig_f,
            "nu": float(nu)}


def ce_pin_cell(seed=1, n=1_000_000, inactive=20, active=50, npts=50_000, nres=200, nbins=10):
    """Infinite pin cell (reflective box 1.26 x 1.26, cylinder r=0.54), four synthetic nuclides.

    Nuclides: A=1 (hydrogen-like), 16, 90, 235 (fissile, nu-bar 2.43).  Fuel =
    235 + 16 + 90, moderator = 1 + 16, with seeded atom densities (atoms/b-cm).
    Tally: track-length flux per cell on `nbins` log-spaced energy bins.
    """
    rng = np.random.default_rng([seed, 2])
    nucs = [
        _ce_nuclide(rng, 1.0, npts, False, 20.0, 0.02, nres=nres, split=(30.0, 0.005)),
        _ce_nuclide(rng, 16.0, npts, False, 3.8, 0.0003, nres=nres, split=(30.0, 0.005)),
        _ce_nuclide(rng, 90.0, npts, False, 6.0, 0.03, nres=nres, split=(6.0, 1.0)),
        _ce_nuclide(rng, 235.0, npts, True, 10.0, 10.0, a_f=93.0, nu=2.43, nres=nres,
                    split=(2.0, 0.5, 2.5)),
    ]
    fuel = {"nuclides": [3, 1, 2],
            "density": [rng.uniform(FUEL_235[0], FUEL_235[1]), 4.6e-2,
                        rng.uniform(FUEL_90[0], FUEL_90[1])]}
    mod = {"nuclides": [0, 1], "density": [rng.uniform(6.0e-2, 7.0e-2), 3.3e-2]}
    surfaces, cells = _pin_geometry()
    edges = np.geomspace(E_MIN, E_MAX, nbins + 1)
    return {
        "name": CONFIG_NAMES[2], "G": 0, "surfaces": surfaces, "cells": cells, "lattices": [],
        "nuclides": nucs, "materials": [fuel, mod],
        "source": {"kind": "box", "box": [-0.63, 0.63, -0.63, 0.63, 0.0, 0.0],
                   "accept": "fissile", "energy": "maxwell", "direction": "iso"},
        "tallies": [{"filter": "cell", "edges": edges}],
        "run": _eigen_run(n, inactive, active, seed),
    }


# ----------------------------------------------------------------------------
# configuration 3: 64 independent fixed-source problems
# ----------------------------------------------------------------------------
def _box_problem(rng, n, max_cells=400):
    """A 3D box split by planes into a grid of cells, some holding a sphere or cylinder."""
    G = int(rng.integers(2, 8))
    target = int(round(math.exp(rng.uniform(0.0, math.log(max_cells * 0.8)))))
    dims = [1, 1, 1]
    while dims[0] * dims[1] * dims[2] * 1.25 < target:
        dims[int(rng.integers(0, 3))] += 1
    nx, ny, nz = dims
    L = rng.uniform(5.0, 40.0, size=3)
    xs = [np.sort(np.concatenate([[0.0, L[a]], rng.uniform(0.15, 0.85, size=d - 1) * L[a]]))
          for a, d in enumerate(dims)]
    # keep planes apart so inner spheres fit
    for a in range(3):
        xs[a] = np.linspace(0.0, L[a], dims[a] + 1) * 0.5 + xs[a] * 0.5
    surfaces = []
    idx = {}
    for a, name in enumerate(["px", "py", "pz"]):
        for i, v in enumerate(xs[a]):
            edge = i == 0 or i == len(xs[a]) - 1
            idx[(a, i)] = len(surfaces)
            surfaces.append(_surf(name, [v], "vacuum" if edge else "none"))
    nmat = int(rng.integers(1, 5))
    mats = []
    for m in range(nmat):
        fis = bool(rng.uniform() < 0.6)
        mats.append(mg_material(rng, G, fissile=fis, kinf=rng.uniform(0.2, 0.8) if fis else None))
    cells = []
    n_inner = 0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                box = [(idx[(0, i)], +1), (idx[(0, i + 1)], -1), (idx[(1, j)], +1),
                       (idx[(1, j + 1)], -1), (idx[(2, k)], +1), (idx[(2, k + 1)], -1)]
                m_out = int(rng.integers(0, nmat))
                room = len(cells) + 2 <= max_cells
                if room and rng.uniform() < 0.2:
                    c = [(xs[0][i] + xs[0][i + 1]) / 2, (xs[1][j] + xs[1][j + 1]) / 2,
                         (xs[2][k] + xs[2][k + 1]) / 2]
                    if rng.uniform() < 0.5:
                        r = 0.3 * min(xs[0][i + 1] - xs[0][i], xs[1][j + 1] - xs[1][j],
                                      xs[2][k + 1] - xs[2][k])
                        s = len(surfaces)
                        surfaces.append(_surf("sphere", [c[0], c[1], c[2], r]))
                        cells.append(_cell(0, [(s, -1)], "material", int(rng.integers(0, nmat))))
                    else:
                        r = 0.3 * min(xs[0][i + 1] - xs[0][i], xs[1][j + 1] - xs[1][j])
                        s = len(surfaces)
                        surfaces.append(_surf("cylz", [c[0], c[1], r]))
                        cells.append(_cell(0, [(s, -1), box[4], box[5]], "material",
                                           int(rng.integers(0, nmat))))
                    cells.append(_cell(0, [(s, +1)] + box, "material", m_out))
                    n_inner += 1
                else:
                    cells.append(_cell(0, box, "material", m_out))
    pdf = rng.uniform(0.1, 1.0, size=G)
    pdf[0] += 2.0
    if rng.uniform() < 0.5:
        p = [rng.uniform(0.1, 0.9) * L[0], rng.uniform(0.1, 0.9) * L[1], rng.uniform(0.1, 0.9) * L[2]]
        src = {"kind": "point", "point": p, "energy": "pdf", "pdf": pdf / pdf.sum(),
               "direction": "iso"}
    else:
        src = {"kind": "box", "box": [0.0, L[0], 0.0, L[1], 0.0, L[2]], "accept": "any",
               "energy": "pdf", "pdf": pdf / pdf.sum(), "direction": "iso"}
    return {"name": "box", "G": G, "surfaces": surfaces, "cells": cells, "lattices": [],
            "materials": mats, "source": src, "tallies": [{"filter": "cell"}],
            "run": _fixed_run(n, int(rng.integers(1, 2 ** 40)), batches=10)}


def batch_boxes(seed=1, nproblems=64, nmin=1_000, nmax=1_000_000, max_cells=400):
    """`nproblems` independent fixed-source box problems with log-uniform sizes in [nmin, nmax]."""
    rng = np.random.default_rng([seed, 3])
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nproblems)).astype(np.int64)
    out = []
    for p in range(nproblems):
        prob = _box_problem(rng, int(sizes[p]), max_cells)
        prob["name"] = f"{CONFIG_NAMES[3]}[{p}]"
        out.append(prob)
    return out


# ----------------------------------------------------------------------------
# configuration 4: differentiation slab
# ----------------------------------------------------------------------------
def diff_slab(seed=1, n=10_000_000, G=7, source_len=5.0, shield_len=20.0, det_len=5.0,
              batches=50):
    """Three-region slab along x: source [0,5], scattering shield [5,25], detector [25,30].

    Vacuum at both x ends, reflective planes at y=+-1 and z=+-1.  Source:
    uniform isotropic in the source region, group 1.  Three seeded subcritical
    materials (k_inf < 0.8).  Tally: detector-cell track-length flux per group.
    """
    rng = np.random.default_rng([seed, 4])
    src_mat = mg_material(rng, G, fissile=True, kinf=rng.uniform(0.3, 0.8))
    shield = mg_material(rng, G, fissile=True, kinf=rng.uniform(0.1, 0.5), sigt=(0.1, 0.4),
                         ratio=(0.85, 0.98))
    det = mg_material(rng, G, fissile=True, kinf=rng.uniform(0.1, 0.5), sigt=(0.1, 0.4))
    x1, x2, x3 = source_len, source_len + shield_len, source_len + shield_len + det_len
    surfaces = [_surf("px", [0.0], "vacuum"), _surf("px", [x1]), _surf("px", [x2]),
                _surf("px", [x3], "vacuum"),
                _surf("py", [-1.0], "reflect"), _surf("py", [1.0], "reflect"),
                _surf("pz", [-1.0], "reflect"), _surf("pz", [1.0], "reflect")]
    yz = [(4, +1), (5, -1), (6, +1), (7, -1)]
    cells = [_cell(0, [(0, +1), (1, -1)] + yz, "material", 0),
             _cell(0, [(1, +1), (2, -1)] + yz, "material", 1),
             _cell(0, [(2, +1), (3, -1)] + yz, "material", 2)]
    pdf = np.zeros(G)
    pdf[0] = 1.0
    return {
        "name": CONFIG_NAMES[4], "G": G, "surfaces": surfaces, "cells": cells, "lattices": [],
        "materials": [src_mat, shield, det],
        "source": {"kind": "box", "box": [0.0, x1, -1.0, 1.0, -1.0, 1.0], "accept": "any",
                   "energy": "pdf", "pdf": pdf, "direction": "iso"},
        "tallies": [{"filter": "cell"}],
        "detector_cell": 2,
        "run": _fixed_run(n, seed, batches),
    }


def absorbing_slab_beam(sigma_t=0.7, thickness=3.0, det_len=2.0, G=1, n=100_000, seed=5,
                        batches=20):
    """Normal beam on a purely absorbing slab followed by a void detector.

    Beam at x=0 along +x into [0, thickness] (Sigma_s = nuSigma_f = 0), then a
    void detector [thickness, thickness + det_len], vacuum beyond.  The
    uncollided fraction is exp(-Sigma_t x); the detector track length per source
    particle is det_len * exp(-Sigma_t x) and its Sigma_t derivative is
    -x * det_len * exp(-Sigma_t x).
    """
    z = np.zeros(G)
    shield = {"sigma_t": np.full(G, float(sigma_t)), "sigma_s": np.zeros((G, G)),
              "nu_sigma_f": z.copy(), "chi": z.copy()}
    void = {"sigma_t": np.zeros(G), "sigma_s": np.zeros((G, G)), "nu_sigma_f": z.copy(),
            "chi": z.copy()}
    surfaces = [_surf("px", [0.0], "vacuum"), _surf("px", [thickness]),
                _surf("px", [thickness + det_len], "vacuum")]
    cells = [_cell(0, [(0, +1), (1, -1)], "material", 0),
             _cell(0, [(1, +1), (2, -1)], "material", 1)]
    pdf = np.zeros(G)
    pdf[0] = 1.0
    return {
        "name": "absorbing-slab-beam", "G": G, "surfaces": surfaces, "cells": cells,
        "lattices": [], "materials": [shield, void],
        "source": {"kind": "point", "point": [0.0, 0.0, 0.0], "energy": "pdf", "pdf": pdf,
                   "direction": "beam", "beam": [1.0, 0.0, 0.0]},
        "tallies": [{"filter": "cell"}],
        "detector_cell": 1,
        "run": _fixed_run(n, seed, batches),
    }


def one_collision_slab(seed=7, n=200_000, batches=20):
    """Two-region, two-group slab for exact enumeration of first-collision outcomes.

    A beam in group 0 enters a slab [0, 1] (material 0) then [1, 2.5] (material
    1), vacuum on both ends.  With the run option max_collisions = 1 every
    history ends at its first collision, so the joint law of (region of first
    collision, outcome, fission count) has a closed form.
    """
    m0 = {"sigma_t": np.array([0.8, 1.3]), "sigma_s": np.array([[0.2, 0.3], [0.0, 0.6]]),
          "nu_sigma_f": np.array([0.5, 0.9]), "chi": np.array([1.0, 0.0])}
    m1 = {"sigma_t": np.array([0.35, 0.9]), "sigma_s": np.array([[0.1, 0.15], [0.05, 0.5]]),
          "nu_sigma_f": np.array([0.0, 0.0]), "chi": np.array([0.0, 0.0])}
    surfaces = [_surf("px", [0.0], "vacuum"), _surf("px", [1.0]), _surf("px", [2.5], "vacuum")]
    cells = [_cell(0, [(0, +1), (1, -1)], "material", 0),
             _cell(0, [(1, +1), (2, -1)], "material", 1)]
    return {
        "name": "one-collision-slab", "G": 2, "surfaces": surfaces, "cells": cells,
        "lattices": [], "materials": [m0, m1],
        "source": {"kind": "point", "point": [0.0, 0.0, 0.0], "energy": "pdf",
                   "pdf": np.array([1.0, 0.0]), "direction": "beam", "beam": [1.0, 0.0, 0.0]},
        "tallies": [{"filter": "cell"}],
        "run": dict(_fixed_run(n, seed, batches), max_collisions=1),
    }


# ----------------------------------------------------------------------------
# small helpers
# ----------------------------------------------------------------------------
def with_run(problem, **kw):
    """A copy of `problem` with run settings replaced (n, inactive, active, seed, ...)."""
    p = copy.deepcopy(problem)
    p["run"].update(kw)
    return p


def scaled(problem, material, key, index, factor):
    """A copy of `problem` with one cross-section entry multiplied by `factor`."""
    p = copy.deepcopy(problem)
    arr = np.array(p["materials"][material][key], dtype=float)
    arr[index] *= factor
    p["materials"][material][key] = arr
    return p


def infinite_medium_fixed(material, pdf, seed=9, n=20_000, half=1.0, batches=20):
    """One reflective cube [-half, half]^3 of one material with a uniform volume source.

    In this infinite medium the volume-integrated flux per source neutron is
    phi = (diag Sigma_t - Sigma_s^T - chi nuSigma_f^T)^-1 q for source spectrum q,
    which gives closed forms for the tally and all its cross-section derivatives.
    """
    G = len(material["sigma_t"])
    surfaces = [_surf("px", [-half], "reflect"), _surf("px", [half], "reflect"),
                _surf("py", [-half], "reflect"), _surf("py", [half], "reflect"),
                _surf("pz", [-half], "reflect"), _surf("pz", [half], "reflect")]
    cells = [_cell(0, [(0, +1), (1, -1), (2, +1), (3, -1), (4, +1), (5, -1)], "material", 0)]
    return {
        "name": "mg-infinite-medium-fixed-source", "G": G, "surfaces": surfaces, "cells": cells,
        "lattices": [], "materials": [copy.deepcopy(material)],
        "source": {"kind": "box", "box": [-half, half, -half, half, -half, half], "accept": "any",
                   "energy": "pdf", "pdf": np.asarray(pdf, float) / np.sum(pdf), "direction": "iso"},
        "tallies": [{"filter": "cell"}],
        "detector_cell": 0,
        "run": _fixed_run(n, seed, batches),
    }


# ----------------------------------------------------------------------------
# time-dependent fixed source (Sec. 1: time-dependent transport; Sec. 4 runs
# its continuous-energy pin cell in this mode)
# ----------------------------------------------------------------------------
def time_pulse_mg(material, pdf, inv_v, t_cut, t_edges, seed=11, n=20_000, batches=20,
                  half=1.0):
    """A pulse of `n` neutrons at t = 0 in an infinite medium (reflective cube).

    One material tally with time bins: the mean neutron population per source
    neutron in each bin, per group.  With one group the population is
    exp(v (nuSigma_f - Sigma_a) t); with several, N(t) = expm(A t) q with
    A = (Sigma_s^T + chi nuSigma_f^T - diag Sigma_t) V, V = diag(1 / inv_v).
    """
    pb = infinite_medium_fixed(material, pdf, seed=seed, n=n, half=half, batches=batches)
    pb["name"] = "mg-infinite-medium-time-pulse"
    pb["time"] = {"t0": 0.0, "t_cut": float(t_cut), "inv_v": np.asarray(inv_v, float)}
    pb["tallies"] = [{"filter": "material", "time_edges": np.asarray(t_edges, float)}]
    return pb


def time_pulse_ce(sig_c, E0, t_cut, t_edges, A=1.0, sig_s=0.0, density=0.05, seed=12,
                  n=20_000, batches=20, half=1.0):
    """A pulse of `n` neutrons of energy E0 (eV) in an infinite medium of one
    nuclide with constant cross sections (barns); energy-integrated population
    tally with time bins.  Without scattering the population is
    exp(-N sigma_c v(E0) t), v(E) = 2.2e5 cm/s sqrt(E / 0.0253 eV)."""
    nuc = {"A": float(A), "E": np.array([E_MIN, E_MAX]), "sig_s": np.array([sig_s, sig_s]),
           "sig_c": np.array([sig_c, sig_c]), "sig_f": np.zeros(2), "nu": 0.0}
    surfaces = [_surf("px", [-half], "reflect"), _surf("px", [half], "reflect"),
                _surf("py", [-half], "reflect"), _surf("py", [half], "reflect"),
                _surf("pz", [-half], "reflect"), _surf("pz", [half], "reflect")]
    cells = [_cell(0, [(0, +1), (1, -1), (2, +1), (3, -1), (4, +1), (5, -1)], "material", 0)]
    return {
        "name": "ce-infinite-medium-time-pulse", "G": 0, "surfaces": surfaces, "cells": cells,
        "lattices": [], "nuclides": [nuc], "materials": [{"nuclides": [0], "density": [density]}],
        "source": {"kind": "box", "box": [-half, half, -half, half, -half, half], "accept": "any",
                   "energy": "fixed", "E": float(E0), "direction": "iso"},
        "tallies": [{"filter": "material", "edges": np.array([E_MIN, E_MAX]),
                     "time_edges": np.asarray(t_edges, float)}],
        "time": {"t0": 0.0, "t_cut": float(t_cut)},
        "run": _fixed_run(n, seed, batches),
    }


def ce_infinite_eigen(nuclides, density, n=20_000, inactive=2, active=30, seed=5, half=1.0):
    """k-eigenvalue in an infinite medium (reflective cube) of one continuous-
    energy material: `nuclides` (dicts as in ce_pin_cell) at atom densities
    `density`; fission-spectrum source; one material tally."""
    surfaces = [_surf("px", [-half], "reflect"), _surf("px", [half], "reflect"),
                _surf("py", [-half], "reflect"), _surf("py", [half], "reflect"),
                _surf("pz", [-half], "reflect"), _surf("pz", [half], "reflect")]
    cells = [_cell(0, [(0, +1), (1, -1), (2, +1), (3, -1), (4, +1), (5, -1)], "material", 0)]
    return {
        "name": "ce-infinite-medium-eigen", "G": 0, "surfaces": surfaces, "cells": cells,
        "lattices": [], "nuclides": list(nuclides),
        "materials": [{"nuclides": list(range(len(nuclides))), "density": list(density)}],
        "source": {"kind": "box", "box": [-half, half, -half, half, -half, half],
                   "accept": "fissile", "energy": "maxwell", "direction": "iso"},
        "tallies": [{"filter": "material", "edges": np.array([E_MIN, E_MAX])}],
        "run": _eigen_run(n, inactive, active, seed),
    }


def ce_time_pin(seed=1, n=10_000_000, t_cut=1.0e-5, ntbins=40, npts=50_000, nres=200,
                batches=20):
    """Stand-in for the paper's continuous-energy benchmark (Sec. 4): the infinite
    pin cell of ce_pin_cell driven by a uniform 14 MeV source, time-dependent
    fixed source, free-gas elastic scattering (kT = 0.0253 eV) below 400 kT;
    tally: neutron population per cell in `ntbins` log-spaced time bins on
    [1e-9 s, t_cut] (energy-integrated)."""
    pb = ce_pin_cell(seed=seed, n=n, npts=npts, nres=nres, nbins=1)
    pb["name"] = "ce-pin-cell-4nuclides-time-14mev"
    pb["source"] = {"kind": "box", "box": [-0.63, 0.63, -0.63, 0.63, 0.0, 0.0], "accept": "any",
                    "energy": "fixed", "E": 14.0e6, "direction": "iso"}
    t_edges = np.concatenate([[0.0], np.geomspace(1.0e-9, t_cut, ntbins)])
    pb["tallies"] = [{"filter": "cell", "edges": np.array([E_MIN, E_MAX]), "time_edges": t_edges}]
    pb["time"] = {"t0": 0.0, "t_cut": float(t_cut)}
    # the paper's model: free-gas elastic scattering, here at 293.6 K
    pb["free_gas"] = {"kT": 0.0253}
    pb["run"] = _fixed_run(n, seed, batches)
    return pb


# ----------------------------------------------------------------------------
# pins of tally layouts and lattice boundaries
# ----------------------------------------------------------------------------
def void_lattice_beam(nx=3, ny=2, pitch=1.25, row=1, n=200, seed=21):
    """A void nx x ny lattice of pitch `pitch` from the origin, vacuum outside,
    with a beam along +x entering at x = 0 through the middle of row `row`.
    Every history crosses the row's elements one after the other, each over a
    track of exactly one pitch, and leaks; the lattice-filter tally must hold
    `pitch` in bins ix + nx * row and 0 elsewhere."""
    G = 1
    void = {"sigma_t": np.zeros(G), "sigma_s": np.zeros((G, G)), "nu_sigma_f": np.zeros(G),
            "chi": np.zeros(G)}
    X, Y = nx * pitch, ny * pitch
    surfaces = [_surf("px", [0.0], "vacuum"), _surf("px", [X], "vacuum"),
                _surf("py", [0.0], "vacuum"), _surf("py", [Y], "vacuum")]
    cells = [_cell(0, [(0, +1), (1, -1), (2, +1), (3, -1)], "lattice", 0),
             _cell(1, [], "material", 0)]
    lattice = {"x0": 0.0, "y0": 0.0, "pitch": float(pitch), "nx": int(nx), "ny": int(ny),
               "universes": np.ones(nx * ny, dtype=np.int32)}
    return {
        "name": "void-lattice-beam", "G": G, "surfaces": surfaces, "cells": cells,
        "lattices": [lattice], "materials": [void],
        "source": {"kind": "point", "point": [0.0, (row + 0.5) * pitch, 0.0], "energy": "pdf",
                   "pdf": np.ones(G), "direction": "beam", "beam": [1.0, 0.0, 0.0]},
        "tallies": [{"filter": "lattice"}],
        "run": _fixed_run(n, seed, 4),
    }


def ce_void_beam(E, edges, length=2.0, n=200, seed=22):
    """Continuous energy: a beam of fixed energy E along +x through a slab of
    a material whose nuclide has zero cross sections, vacuum at both faces.
    Each history streams `length` at energy E and leaks; the cell tally with
    energy edges `edges` must hold `length` in the bin E falls in (the largest
    b with edges[b] <= E, the top edge closing the last bin) and nothing when E
    is outside [edges[0], edges[-1]]."""
    grid = np.array([E_MIN, 1.0, E_MAX])
    nuc = {"A": 1.0, "E": grid, "sig_s": np.zeros(3), "sig_c": np.zeros(3), "sig_f": np.zeros(3),
           "nu": 0.0}
    surfaces = [_surf("px", [0.0], "vacuum"), _surf("px", [length], "vacuum")]
    cells = [_cell(0, [(0, +1), (1, -1)], "material", 0)]
    return {
        "name": "ce-void-beam", "G": 0, "surfaces": surfaces, "cells": cells, "lattices": [],
        "nuclides": [nuc], "materials": [{"nuclides": [0], "density": [1.0]}],
        "source": {"kind": "point", "point": [0.0, 0.0, 0.0], "energy": "fixed", "E": float(E),
                   "direction": "beam", "beam": [1.0, 0.0, 0.0]},
        "tallies": [{"filter": "cell", "edges": np.asarray(edges, float)}],
        "run": _fixed_run(n, seed, 4),
    }


def small_lattice(seed=31, n=4000, inactive=2, active=3, nx=4, ny=4, pitch=1.26, r=0.54,
                  z_planes=None, x_plane=None, G=7):
    """A small k-eigenvalue lattice of pin cells (fuel cylinder of radius r in
    moderator, every element alike) with root boundaries that reach inside the
    lattice's elements.  z_planes = (zlo, zhi, bc_lo, bc_hi): the root cell is
    also bounded by z-planes (the lattice is finite in height).  x_plane =
    (x, bc): the root cell's low-x boundary is a plane at x (through the first
    column's pin centres for x = pitch / 2) instead of the lattice's edge.
    Otherwise the outer boundary is reflective at low x and y and vacuum at
    high x and y."""
    rng = np.random.default_rng([seed, 5])
    fuel = mg_material(rng, G, fissile=True, kinf=1.3)
    mod = mg_material(rng, G, fissile=False)
    X, Y = nx * pitch, ny * pitch
    xlo, xbc = (0.0, "reflect") if x_plane is None else (float(x_plane[0]), x_plane[1])
    surfaces = [_surf("px", [xlo], xbc), _surf("px", [X], "vacuum"),
                _surf("py", [0.0], "reflect"), _surf("py", [Y], "vacuum"),
                _surf("cylz", [0.0, 0.0, r])]
    root = [(0, +1), (1, -1), (2, +1), (3, -1)]
    zlo = zhi = None
    if z_planes is not None:
        zlo, zhi, blo, bhi = z_planes
        surfaces += [_surf("pz", [zlo], blo), _surf("pz", [zhi], bhi)]
        root += [(5, +1), (6, -1)]
    cells = [_cell(0, root, "lattice", 0),
             _cell(1, [(4, -1)], "material", 0),
             _cell(1, [(4, +1)], "material", 1)]
    lattice = {"x0": 0.0, "y0": 0.0, "pitch": float(pitch), "nx": int(nx), "ny": int(ny),
               "universes": np.ones(nx * ny, dtype=np.int32)}
    box = [xlo, X, 0.0, Y, zlo if zlo is not None else 0.0, zhi if zhi is not None else 0.0]
    return {
        "name": "small-lattice", "G": G, "surfaces": surfaces, "cells": cells,
        "lattices": [lattice], "materials": [fuel, mod],
        "source": {"kind": "box", "box": box, "accept": "fissile", "energy": "chi",
                   "direction": "iso"},
        "tallies": [{"filter": "lattice"}, {"filter": "cell"}],
        "run": _eigen_run(n, inactive, active, seed),
    }
