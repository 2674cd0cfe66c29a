"""Python access to the plain CPU oracle (``mcoracle.c``).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The CUDA library never
uses it.  This module only marshals arguments; all arithmetic is in the C file.

``Oracle(problem)`` evaluates every step by its plain definition (libm log,
true division, no fused multiply-add, nuclide sums at the particle's energy).
``Oracle(problem, strict=True)`` adopts the CUDA library's rounding
conventions instead, for bit-for-bit comparisons of histories.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcoracle.c")
_HDR = os.path.join(_HERE, "mcoracle.h")
_LIB = os.path.join(_HERE, "_build", "libmcoracle.so")
_lock = threading.Lock()
_lib = None

SURF = {"px": 0, "py": 1, "pz": 2, "plane": 3, "cylz": 4, "sphere": 5}
BC = {"none": 0, "vacuum": 1, "reflect": 2}
FILL = {"material": 0, "lattice": 1}
FILTER = {"cell": 0, "lattice": 1, "material": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double, no contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64, u64, d, i32 = C.c_int64, C.c_uint64, C.c_double, C.c_int
            P = C.c_void_p
            L.orc_create.restype = P
            L.orc_destroy.argtypes = [P]
            L.orc_error.restype = C.c_char_p
            L.orc_error.argtypes = [P]
            L.orc_run_eigen.argtypes = [P, i64, i32, i32, u64, i32]
            L.orc_run_fixed.argtypes = [P, i64, i32, u64, i32]
            L.orc_add_lattice.argtypes = [P, d, d, d, i32, i32, P]
            L.orc_add_nuclide.argtypes = [P, d, i32, P, P, P, P, d]
            L.orc_grad_fixed.argtypes = [P, i64, u64, i32, P, P, P, P, P]
            L.orc_histories_by_index.argtypes = [P, u64, i64, P, P, P, P, P, P, P]
            L.orc_rng_skip.restype = u64
            L.orc_rng_skip.argtypes = [u64, u64]
            L.orc_rng_stream.restype = u64
            L.orc_rng_stream.argtypes = [u64, u64]
            L.orc_rng_next.restype = u64
            L.orc_rng_next.argtypes = [u64]
            L.orc_rng_xi.restype = d
            L.orc_rng_xi.argtypes = [u64]
            L.orc_log.restype = d
            L.orc_log.argtypes = [d]
            L.orc_log_table_q57.restype = C.c_int64
            L.orc_log_table_q57.argtypes = [i32]
            L.orc_site_index.restype = i64
            L.orc_site_index.argtypes = [i64, u64, i64, i64]
            L.orc_maxwell.restype = d
            L.orc_maxwell.argtypes = [P, i32]
            L.orc_elastic.argtypes = [d, d, P, P, P, i32]
            L.orc_free_gas.argtypes = [d, d, d, P, P, P, i32]
            L.orc_iso_dir.argtypes = [P, P, i32]
            L.orc_set_arith.restype = i32
            L.orc_set_arith.argtypes = [P, i32]
            L.orc_set_free_gas.restype = i32
            L.orc_set_free_gas.argtypes = [P, d, d]
            L.orc_history_count.restype = i64
            L.orc_history_count.argtypes = [P]
            L.orc_bank_count.restype = i64
            L.orc_bank_count.argtypes = [P]
            L.orc_set_time.restype = i32
            L.orc_set_time.argtypes = [P, d, d]
            L.orc_set_inverse_speeds.restype = i32
            L.orc_set_inverse_speeds.argtypes = [P, i32, P]
            L.orc_set_tally_time_bins.restype = i32
            L.orc_set_tally_time_bins.argtypes = [P, i32, i32, P]
            for name in ["orc_add_surface", "orc_add_cell", "orc_set_groups", "orc_add_material_mg",
                         "orc_add_material_ce", "orc_set_source", "orc_add_tally",
                         "orc_set_max_collisions", "orc_get_k", "orc_get_cycle_k",
                         "orc_tally_size", "orc_get_tally", "orc_get_counters",
                         "orc_get_histories", "orc_get_bank", "orc_iso_dir", "orc_probe",
                         "orc_ce_lookup"]:
                getattr(L, name).restype = i32
            _lib = L
        return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class OracleError(RuntimeError):
    pass


class Oracle:
    """One problem loaded into the CPU oracle."""

    def __init__(self, problem: dict, strict: bool = False):
        self.L = lib()
        self.problem = problem
        self.strict = bool(strict)
        self.ctx = C.c_void_p(self.L.orc_create())
        self._keep = []
        self._chk(self.L.orc_set_arith(self.ctx, 1 if strict else 0))
        self._load(problem)

    def __del__(self):
        if getattr(self, "ctx", None):
            self.L.orc_destroy(self.ctx)
            self.ctx = None

    def _chk(self, r):
        if r < 0:
            raise OracleError(self.L.orc_error(self.ctx).decode())
        return r

    def _load(self, pb):
        L, c = self.L, self.ctx
        for s in pb["surfaces"]:
            coef = _f64(s["coef"])
            self._chk(L.orc_add_surface(c, SURF[s["type"]], _p(coef), BC[s["bc"]]))
        for cell in pb["cells"]:
            surf, sense = _i32(cell["surfs"]), _i32(cell["senses"])
            self._chk(L.orc_add_cell(c, cell["universe"], len(cell["surfs"]), _p(surf), _p(sense),
                                     FILL[cell["fill_kind"]], cell["fill"]))
        for lat in pb["lattices"]:
            u = _i32(lat["universes"])
            self._chk(L.orc_add_lattice(c, lat["x0"], lat["y0"], lat["pitch"], lat["nx"],
                                        lat["ny"], _p(u)))
        if pb["G"] > 0:
            self._chk(L.orc_set_groups(c, pb["G"]))
            for m in pb["materials"]:
                a = [_f64(m[k]) for k in ("sigma_t", "sigma_s", "nu_sigma_f", "chi")]
                self._chk(L.orc_add_material_mg(c, *[_p(x) for x in a]))
        else:
            for nu in pb["nuclides"]:
                arrs = [_f64(nu[k]) for k in ("E", "sig_s", "sig_c", "sig_f")]
                self._chk(L.orc_add_nuclide(c, nu["A"], len(arrs[0]), *[_p(x) for x in arrs],
                                            nu["nu"]))
            for m in pb["materials"]:
                nucs, dens = _i32(m["nuclides"]), _f64(m["density"])
                self._chk(L.orc_add_material_ce(c, len(nucs), _p(nucs), _p(dens)))
        src = pb["source"]
        if src["kind"] == "box":
            kind, params = 0, _f64(src["box"])
        else:
            kind, params = 1, _f64(src["point"])
        accept = 1 if src.get("accept") == "fissile" else 0
        ek = {"chi": 0, "pdf": 1, "fixed": 2, "maxwell": 3}[src["energy"]]
        edata = _f64(src["pdf"] if ek == 1 else ([src.get("E", 0.0)] if ek == 2 else [0.0]))
        dk = 1 if src["direction"] == "beam" else 0
        beam = _f64(src.get("beam", [0.0, 0.0, 1.0]))
        self._keep += [params, edata, beam]
        self._chk(L.orc_set_source(c, kind, _p(params), accept, ek, _p(edata), len(edata), dk,
                                   _p(beam)))
        for t in pb["tallies"]:
            edges = _f64(t.get("edges", [0.0]))
            ne = len(edges) if "edges" in t else 0
            self._chk(L.orc_add_tally(c, FILTER[t["filter"]], ne, _p(edges)))
        if "free_gas" in pb:
            fg = pb["free_gas"]
            self._chk(L.orc_set_free_gas(c, float(fg["kT"]), float(fg.get("cut", 0.0))))
        if "time" in pb:
            tm = pb["time"]
            self._chk(L.orc_set_time(c, float(tm.get("t0", 0.0)), float(tm["t_cut"])))
            if pb["G"] > 0:
                inv_v = _f64(tm["inv_v"])
                self._keep.append(inv_v)
                self._chk(L.orc_set_inverse_speeds(c, len(inv_v), _p(inv_v)))
        for i, t in enumerate(pb["tallies"]):
            if "time_edges" in t:
                te = _f64(t["time_edges"])
                self._keep.append(te)
                self._chk(L.orc_set_tally_time_bins(c, i, len(te), _p(te)))
        self._chk(L.orc_set_max_collisions(c, int(pb["run"].get("max_collisions", 0))))

    # ---------------------------------------------------------------- runs
    def run(self, threads: int = 0, **over):
        r = dict(self.problem["run"], **over)
        if r["mode"] == "eigen":
            self._chk(self.L.orc_run_eigen(self.ctx, r["n"], r["inactive"], r["active"],
                                           r["seed"], threads))
        else:
            self._chk(self.L.orc_run_fixed(self.ctx, r["n"], r["batches"], r["seed"], threads))
        return self

    def k(self):
        out = np.zeros(6)
        self.L.orc_get_k(self.ctx, _p(out))
        return {"k": out[0], "k_sd": out[1], "k_col": out[2], "k_col_sd": out[3],
                "k_analog": out[4], "k_analog_sd": out[5]}

    def cycle_k(self, ncyc):
        ktl, kc, m = np.zeros(ncyc), np.zeros(ncyc), np.zeros(ncyc, dtype=np.int64)
        self.L.orc_get_cycle_k(self.ctx, ncyc, _p(ktl), _p(kc), _p(m))
        return ktl, kc, m

    def tally(self, t: int = 0):
        """Means and sds per (bin, group or energy bin), with a trailing time-bin
        axis when the tally has time bins."""
        nb, ne, nt = C.c_int(), C.c_int(), C.c_int()
        self._chk(self.L.orc_tally_size(self.ctx, t, C.byref(nb), C.byref(ne), C.byref(nt)))
        mean = np.zeros(nb.value * ne.value * nt.value)
        sd = np.zeros_like(mean)
        self._chk(self.L.orc_get_tally(self.ctx, t, _p(mean), _p(sd)))
        shape = (nb.value, ne.value)
        if "time_edges" in self.problem["tallies"][t]:
            shape = shape + (nt.value,)
        return mean.reshape(shape), sd.reshape(shape)

    def counters(self):
        out = np.zeros(8, dtype=np.int64)
        self.L.orc_get_counters(self.ctx, _p(out))
        keys = ["histories", "collisions", "crossings", "leaks", "lost", "capped", "generations",
                "time_cut"]
        return dict(zip(keys, out.tolist()))

    def histories(self):
        n = self.L.orc_history_count(self.ctx)
        nc, nx, nf, fate, g = (np.zeros(n, dtype=np.int32) for _ in range(5))
        rng = np.zeros(n, dtype=np.uint64)
        self.L.orc_get_histories(self.ctx, _p(nc), _p(nx), _p(rng), _p(nf), _p(fate), _p(g))
        return {"n_coll": nc, "n_cross": nx, "rng_end": rng, "n_fis": nf, "fate": fate, "g_end": g}

    def histories_by_index(self, idx, seed=None):
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        n = len(idx)
        nc, nx, nf, fate, g = (np.zeros(n, dtype=np.int32) for _ in range(5))
        rng = np.zeros(n, dtype=np.uint64)
        seed = self.problem["run"]["seed"] if seed is None else seed
        self._chk(self.L.orc_histories_by_index(self.ctx, seed, n, _p(idx), _p(nc), _p(nx), _p(rng),
                                                _p(nf), _p(fate), _p(g)))
        return {"n_coll": nc, "n_cross": nx, "rng_end": rng, "n_fis": nf, "fate": fate, "g_end": g}

    def bank(self):
        n = self.L.orc_bank_count(self.ctx)
        xyz = np.zeros((n, 3))
        parent = np.zeros(n, dtype=np.int64)
        child, mat = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
        self.L.orc_get_bank(self.ctx, _p(xyz), _p(parent), _p(child), _p(mat))
        return {"xyz": xyz, "parent": parent, "child": child, "mat": mat}

    def grad(self, n: int, seed: int, cell: int, weights=None):
        G = self.problem["G"]
        nm = len(self.problem["materials"])
        w = _f64(np.ones(G) if weights is None else weights)
        dst, dss, dnf = np.zeros(nm * G), np.zeros(nm * G * G), np.zeros(nm * G)
        tal = np.zeros(G)
        self._chk(self.L.orc_grad_fixed(self.ctx, n, seed, cell, _p(w), _p(dst), _p(dss), _p(dnf),
                                        _p(tal)))
        return {"sigma_t": dst.reshape(nm, G), "sigma_s": dss.reshape(nm, G, G),
                "nu_sigma_f": dnf.reshape(nm, G), "tally": tal}

    def probe(self, pos, direction):
        path = np.zeros(5, dtype=np.int32)
        d = C.c_double()
        kind = C.c_int()
        pos, direction = _f64(pos), _f64(direction)
        self._chk(self.L.orc_probe(self.ctx, _p(pos), _p(direction), _p(path), C.byref(d),
                                   C.byref(kind)))
        return path, d.value, kind.value

    def ce_lookup(self, material, E):
        out = np.zeros(4)
        self._chk(self.L.orc_ce_lookup(self.ctx, material, C.c_double(E), _p(out)))
        return out


# -------------------------------------------------------------------- building blocks
def rng_skip(s, n):
    return lib().orc_rng_skip(s, n)


def rng_stream(seed, i):
    return lib().orc_rng_stream(seed, i)


def rng_next(s):
    return lib().orc_rng_next(s)


def rng_xi(s):
    return lib().orc_rng_xi(s)


def log(xi):
    """ln xi by the strict mode's table-driven method"""
    return lib().orc_log(xi)


def log_table_q57(j):
    """entry j of the strict logarithm's table: ln(1 + j/256) 2^57 rounded to
    the nearest integer"""
    return lib().orc_log_table_q57(j)


def site_index(j, n, M, N):
    """bank site taken by source j of N after M sites, resampling draw n 2^-53"""
    return lib().orc_site_index(j, n, M, N)


def iso_dir(state, strict=False):
    s = C.c_uint64(state)
    out = np.zeros(3)
    lib().orc_iso_dir(C.byref(s), _p(out), 1 if strict else 0)
    return out, s.value


def elastic(E, A, direction, state, strict=False):
    s = C.c_uint64(state)
    d = _f64(direction)
    out = np.zeros(4)
    lib().orc_elastic(E, A, _p(d), C.byref(s), _p(out), 1 if strict else 0)
    return out, s.value


def free_gas(E, A, kT, direction, state, strict=False):
    s = C.c_uint64(state)
    d = _f64(direction)
    out = np.zeros(4)
    lib().orc_free_gas(E, A, kT, _p(d), C.byref(s), _p(out), 1 if strict else 0)
    return out, s.value


def maxwell(state, strict=False):
    s = C.c_uint64(state)
    e = lib().orc_maxwell(C.byref(s), 1 if strict else 0)
    return e, s.value
