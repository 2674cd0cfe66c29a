"""Independent numpy point classification of a problem's CSG geometry.

Used only by tests: it evaluates every cell's half-spaces at sample points
(no distance formulas), so ray marching with bisection on "the containing cell
changes" gives brute-force distances to the nearest boundary.
"""
import numpy as np


def surface_values(pb, pts):
    """f_s(p) for every surface s (rows) and point p (columns)."""
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    out = np.empty((len(pb["surfaces"]), len(pts)))
    for i, s in enumerate(pb["surfaces"]):
        c = s["coef"]
        t = s["type"]
        if t == "px":
            out[i] = x - c[0]
        elif t == "py":
            out[i] = y - c[0]
        elif t == "pz":
            out[i] = z - c[0]
        elif t == "plane":
            out[i] = c[0] * x + c[1] * y + c[2] * z - c[3]
        elif t == "cylz":
            out[i] = (x - c[0]) ** 2 + (y - c[1]) ** 2 - c[2] ** 2
        else:
            out[i] = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 - c[3] ** 2
    return out


def _cells_of(pb, universe):
    return [i for i, c in enumerate(pb["cells"]) if c["universe"] == universe]


def _member(pb, fv, cells):
    """index into `cells` of the (unique) cell holding each point, -1 if none."""
    res = np.full(fv.shape[1], -1)
    for k, ci in enumerate(cells):
        c = pb["cells"][ci]
        ok = np.ones(fv.shape[1], dtype=bool)
        for s, sense in zip(c["surfs"], c["senses"]):
            ok &= (fv[s] > 0) if sense > 0 else (fv[s] < 0)
        res[ok & (res == -1)] = ci
    return res


def classify(pb, pts):
    """Integer code of (root cell, lattice element, universe cell) per point; -1 outside."""
    pts = np.atleast_2d(pts)
    fv = surface_values(pb, pts)
    root = _member(pb, fv, _cells_of(pb, 0))
    code = np.full(len(pts), -1, dtype=np.int64)
    nc = len(pb["cells"])
    for r in np.unique(root[root >= 0]):
        sel = root == r
        cell = pb["cells"][r]
        if cell["fill_kind"] != "lattice":
            code[sel] = r * (nc + 1) * 10**7
            continue
        L = pb["lattices"][cell["fill"]]
        p = pts[sel]
        ix = np.floor((p[:, 0] - L["x0"]) / L["pitch"]).astype(int)
        iy = np.floor((p[:, 1] - L["y0"]) / L["pitch"]).astype(int)
        ix = np.clip(ix, 0, L["nx"] - 1)
        iy = np.clip(iy, 0, L["ny"] - 1)
        loc = p.copy()
        loc[:, 0] -= L["x0"] + (ix + 0.5) * L["pitch"]
        loc[:, 1] -= L["y0"] + (iy + 0.5) * L["pitch"]
        fl = surface_values(pb, loc)
        uc = np.full(len(p), -1)
        univ = np.asarray(L["universes"])[ix + L["nx"] * iy]
        for U in np.unique(univ):
            m = univ == U
            uc[m] = _member(pb, fl[:, m], _cells_of(pb, int(U)))
        sub = ((r * (nc + 1) + uc + 1) * 10**7 + (ix * 3000 + iy))
        sub[uc < 0] = -1
        code[np.where(sel)[0]] = sub
    return code


def brute_distance(pb, pos, direction, tmax, h):
    """Smallest t in (0, tmax] where the classification changes (bisection to 1e-13)."""
    ts = np.arange(1, int(np.ceil(tmax / h)) + 1) * h
    pts = pos[None, :] + ts[:, None] * direction[None, :]
    c0 = classify(pb, pos[None, :] + 1e-13 * direction[None, :])[0]
    codes = classify(pb, pts)
    ch = np.nonzero(codes != c0)[0]
    if len(ch) == 0:
        return np.inf
    hi = ts[ch[0]]
    lo = hi - h
    while hi - lo > 1e-13:
        mid = 0.5 * (lo + hi)
        if classify(pb, (pos + mid * direction)[None, :])[0] == c0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
