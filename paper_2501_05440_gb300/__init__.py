"""GB300 event-based Monte Carlo neutral-particle transport (libmcgb).

Thin ctypes binding of the C ABI declared in include/mcgb.h: the methods carry
the C names without the ``mcgb_`` prefix and only marshal arguments; every
transport step runs in the CUDA kernels of libmcgb.so.  There is no CPU
fallback: importing works anywhere, but creating a context needs the built
library and a CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = ["lib", "build", "McgbError", "Context", "Batch", "load_problem", "library_path",
           "bank_offsets_noalloc", "kernel_source_hash", "MODE_EVENT", "MODE_PERSISTENT",
           "MODE_SEGMENT"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "_build", "libmcgb.so")
_lock = threading.Lock()
_lib = None

MODE_EVENT, MODE_PERSISTENT, MODE_SEGMENT = 0, 1, 2
SURF = {"px": 0, "py": 1, "pz": 2, "plane": 3, "cylz": 4, "sphere": 5}
BC = {"none": 0, "vacuum": 1, "reflect": 2}
FILL = {"material": 0, "lattice": 1}
FILTER = {"cell": 0, "lattice": 1, "material": 2}
ENERGY = {"chi": 0, "pdf": 1, "fixed": 2, "maxwell": 3}


class McgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mcgb error {code}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("device", C.c_int), ("mode", C.c_int), ("block", C.c_int),
                ("blocks_per_sm", C.c_int), ("record_histories", C.c_int),
                ("bank_factor", C.c_double), ("max_iterations", C.c_int), ("pool", C.c_int),
                ("graphs", C.c_int)]


class Counters(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("histories", "collisions", "crossings", "leaks", "lost",
                                         "capped", "generations", "kernel_launches",
                                         "event_iterations", "world_bytes", "time_cut")]


# one fission site as exchanged between ranks (mcgb_site)
SITE_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("t", "<f8"), ("cell", "<i4"),
                       ("ix", "<i4"), ("iy", "<i4"), ("ucell", "<i4"), ("mat", "<i4"),
                       ("child", "<i4"), ("parent", "<i8")])
assert SITE_DTYPE.itemsize == 64


class Tune(C.Structure):
    _fields_ = [("block", C.c_int), ("blocks_per_sm", C.c_int), ("pool", C.c_int),
                ("ms", C.c_double)]


# the files that define the device code of the transport kernels
_KERNEL_SOURCES = ["kernels.h", "world.h", "fpint.cuh", "transport.cuh", "steps.cuh", "pool.cuh",
                   "kernels_pool.cu", "kernels_pool_mg.cu", "kernels_pool_mg_time.cu",
                   "kernels_pool_ce.cu", "kernels_pool_ce_time.cu", "kernels_transport.cu"]


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the transport kernels' device
    sources: profiler counters taken on a build are valid while it matches."""
    import hashlib
    h = hashlib.sha256()
    for name in _KERNEL_SOURCES:
        with open(os.path.join(_HERE, "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def library_path():
    return _LIBPATH


def build(force=False):
    """Compile the CUDA library for sm_103a (nvcc) and return its path."""
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded libmcgb.so (built on first use when nvcc is available)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIBPATH):
                build()
            if not os.path.exists(_LIBPATH):
                raise McgbError(-3, f"CUDA library missing: {_LIBPATH} (run build())")
            L = C.CDLL(_LIBPATH)
            P, i32, i64, u64, d = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
            sz = C.c_size_t
            L.mcgb_last_error.restype = C.c_char_p
            sigs = {
                "mcgb_create": [P, P], "mcgb_destroy": [P], "mcgb_set_stream": [P, P],
                "mcgb_set_mode": [P, i32],
                "mcgb_add_surface": [P, i32, P, i32, P],
                "mcgb_add_cell": [P, i32, i32, P, P, i32, i32, P],
                "mcgb_add_lattice": [P, d, d, d, i32, i32, P, P],
                "mcgb_set_groups": [P, i32],
                "mcgb_add_material_mg": [P, P, P, P, P, P],
                "mcgb_update_material_mg": [P, i32, P, P, P, P],
                "mcgb_add_nuclide_ce": [P, d, i32, P, P, P, P, d, P],
                "mcgb_add_material_ce": [P, i32, P, P, P],
                "mcgb_set_source": [P, i32, P, i32, i32, P, i32, i32, P],
                "mcgb_add_tally": [P, i32, i32, P, P],
                "mcgb_set_max_collisions": [P, i32],
                "mcgb_set_time": [P, d, d], "mcgb_set_inverse_speeds": [P, i32, P],
                "mcgb_set_free_gas": [P, d, d],
                "mcgb_shard_begin": [P, i64, i64, i64, i32, i32, u64],
                "mcgb_shard_cycle": [P, i32, P], "mcgb_shard_export": [P, P, sz, P, sz, P],
                "mcgb_shard_import": [P, i32, P, P, i64], "mcgb_shard_finish": [P],
                "mcgb_domain_begin": [P, i64, i32, i32, u64, i32, P, i32, i32],
                "mcgb_domain_sources": [P, i32, P, i64], "mcgb_domain_sweep": [P, P],
                "mcgb_domain_outbox": [P, P, sz], "mcgb_domain_inbox": [P, P, i64],
                "mcgb_domain_export": [P, P, P, sz, P, sz, P, P],
                "mcgb_domain_import": [P, i32, P, P, P, i64], "mcgb_domain_finish": [P],
                "mcgb_domain_records": [P, P, P, P, P, P, P],
                "mcgb_set_tally_time_bins": [P, i32, i32, P],
                "mcgb_run_eigenvalue": [P, i64, i32, i32, u64],
                "mcgb_run_fixed_source": [P, i64, i32, u64],
                "mcgb_eigen_begin": [P, i64, i32, i32, u64], "mcgb_eigen_cycles": [P, i32],
                "mcgb_eigen_finish": [P], "mcgb_get_cycle_times": [P, i32, P, P],
                "mcgb_eigen_checkpoint": [P, P, sz, P], "mcgb_eigen_restore": [P, P, sz],
                "mcgb_get_event_timing": [P, P, P, P, P],
                "mcgb_get_k": [P, P], "mcgb_get_cycle_k": [P, i32, P, P, P],
                "mcgb_tally_size": [P, i32, P, P, P], "mcgb_get_tally": [P, i32, P, P, sz, P],
                "mcgb_get_counters": [P, P],
                "mcgb_get_histories": [P, sz, P, P, P, P, P, P, P],
                "mcgb_get_bank": [P, sz, P, P, P, P, P],
                "mcgb_forward_fixed": [P, i64, u64, i32, P],
                "mcgb_backward_fixed": [P, P, P, P, P],
                "mcgb_update_material_mg_dev": [P, i32, i32, P, P, P],
                "mcgb_forward_fixed_dev": [P, i64, u64, i32, P],
                "mcgb_backward_fixed_dev": [P, P, P, P, P],
                "mcgb_batch_create": [P, P], "mcgb_batch_destroy": [P],
                "mcgb_batch_add_problem": [P, P, i64, i32, u64, P],
                "mcgb_batch_autotune": [P, i32, P], "mcgb_batch_run": [P, P],
                "mcgb_batch_tally": [P, i32, i32, P, P, sz, P], "mcgb_batch_counters": [P, P],
                "mcgb_rng_states": [P, u64, u64, i64, i32, P],
                "mcgb_log": [P, i64, P, P], "mcgb_probe": [P, i64, P, P, P, P, P],
                "mcgb_fp64_throughput": [P, i64, P, P],
                "mcgb_fpint_ops": [P, i64, P, P, P],
                "mcgb_ce_lookup": [P, i32, i64, P, P],
                "mcgb_bank_offsets_noalloc": [P, i64, P, P, P],
            }
            for name, args in sigs.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = i32
            _lib = L
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _chk(r):
    if r != 0:
        raise McgbError(r, lib().mcgb_last_error().decode())
    return r


def bank_offsets_noalloc(n_fis_ptr, n, first_ptr, total_ptr, stream=0):
    """mcgb_bank_offsets_noalloc on device pointers (ints); allocates nothing."""
    _chk(lib().mcgb_bank_offsets_noalloc(C.c_void_p(n_fis_ptr), n, C.c_void_p(first_ptr),
                                         C.c_void_p(total_ptr), C.c_void_p(stream)))


class Context:
    """One transport problem on one GPU (mcgb_ctx)."""

    def __init__(self, device=0, mode=MODE_EVENT, block=0, blocks_per_sm=0,
                 record_histories=False, bank_factor=0.0, max_iterations=0, pool=0, graphs=0):
        L = lib()
        self.L = L
        self.opts = Opts(device, mode, block, blocks_per_sm, int(record_histories),
                         bank_factor, max_iterations, pool, graphs)
        h = C.c_void_p()
        _chk(L.mcgb_create(C.byref(h), C.byref(self.opts)))
        self.h = h
        self.problem = None
        self.G = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.mcgb_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    # ---- C calls (argument marshalling only)
    def set_stream(self, stream):
        _chk(self.L.mcgb_set_stream(self.h, C.c_void_p(stream)))

    def set_mode(self, mode):
        _chk(self.L.mcgb_set_mode(self.h, mode))

    def add_surface(self, type_, coef, bc):
        i = C.c_int()
        c = _f64(list(coef) + [0.0] * (4 - len(coef)))
        _chk(self.L.mcgb_add_surface(self.h, type_, _p(c), bc, C.byref(i)))
        return i.value

    def add_cell(self, universe, surfs, senses, fill_kind, fill):
        i = C.c_int()
        s, x = _i32(surfs), _i32(senses)
        _chk(self.L.mcgb_add_cell(self.h, universe, len(s), _p(s), _p(x), fill_kind, fill,
                                  C.byref(i)))
        return i.value

    def add_lattice(self, x0, y0, pitch, nx, ny, universes):
        i = C.c_int()
        u = _i32(universes)
        _chk(self.L.mcgb_add_lattice(self.h, x0, y0, pitch, nx, ny, _p(u), C.byref(i)))
        return i.value

    def set_groups(self, G):
        _chk(self.L.mcgb_set_groups(self.h, G))
        self.G = G

    def add_material_mg(self, sigma_t, sigma_s, nu_sigma_f, chi):
        i = C.c_int()
        a = [_f64(sigma_t), _f64(sigma_s), _f64(nu_sigma_f), _f64(chi)]
        _chk(self.L.mcgb_add_material_mg(self.h, *[_p(x) for x in a], C.byref(i)))
        return i.value

    def update_material_mg(self, mid, sigma_t, sigma_s, nu_sigma_f, chi=None):
        a = [_f64(sigma_t), _f64(sigma_s), _f64(nu_sigma_f)]
        ch = None if chi is None else _f64(chi)
        _chk(self.L.mcgb_update_material_mg(self.h, mid, *[_p(x) for x in a], _p(ch)))

    def add_nuclide_ce(self, A, E, sig_s, sig_c, sig_f, nu):
        i = C.c_int()
        a = [_f64(E), _f64(sig_s), _f64(sig_c), _f64(sig_f)]
        _chk(self.L.mcgb_add_nuclide_ce(self.h, A, len(a[0]), *[_p(x) for x in a], nu,
                                        C.byref(i)))
        return i.value

    def add_material_ce(self, nuclides, density):
        i = C.c_int()
        n, d = _i32(nuclides), _f64(density)
        _chk(self.L.mcgb_add_material_ce(self.h, len(n), _p(n), _p(d), C.byref(i)))
        return i.value

    def set_source(self, kind, params, accept, energy_kind, energy, dir_kind, beam=None):
        p, e = _f64(params), _f64(energy)
        b = _f64(beam if beam is not None else [0.0, 0.0, 1.0])
        _chk(self.L.mcgb_set_source(self.h, kind, _p(p), accept, energy_kind, _p(e), len(e),
                                    dir_kind, _p(b)))

    def add_tally(self, filter_, edges=None):
        i = C.c_int()
        e = _f64(edges if edges is not None else [0.0])
        n = 0 if edges is None else len(e)
        _chk(self.L.mcgb_add_tally(self.h, filter_, n, _p(e), C.byref(i)))
        return i.value

    def set_max_collisions(self, m):
        _chk(self.L.mcgb_set_max_collisions(self.h, m))

    # sharded power iteration (see paper_2501_05440_gb300.sharded)
    def shard_begin(self, N, j0, n, inactive, active, seed):
        _chk(self.L.mcgb_shard_begin(self.h, int(N), int(j0), int(n), int(inactive), int(active),
                                     int(seed)))

    def shard_cycle(self, cycle):
        """Transport this rank's histories of `cycle`; returns the sites it banked."""
        m = C.c_int64()
        _chk(self.L.mcgb_shard_cycle(self.h, int(cycle), C.byref(m)))
        return m.value

    def shard_sums_size(self):
        n = C.c_size_t()
        _chk(self.L.mcgb_shard_export(self.h, None, 0, None, 0, C.byref(n)))
        return n.value

    def shard_export(self, bank, bank_cap, sums, sums_cap):
        """bank, sums: device addresses (ints) of 64-byte site records and doubles"""
        n = C.c_size_t()
        _chk(self.L.mcgb_shard_export(self.h, C.c_void_p(bank), int(bank_cap), C.c_void_p(sums),
                                      int(sums_cap), C.byref(n)))

    def shard_import(self, cycle, sums, bank, M):
        _chk(self.L.mcgb_shard_import(self.h, int(cycle), C.c_void_p(sums), C.c_void_p(bank),
                                      int(M)))

    def shard_finish(self):
        _chk(self.L.mcgb_shard_finish(self.h))

    # spatial domain decomposition: array arguments are device addresses (ints)
    def domain_begin(self, N, inactive, active, seed, axis, cuts, rank):
        c = _f64(cuts)
        _chk(self.L.mcgb_domain_begin(self.h, int(N), int(inactive), int(active), int(seed),
                                      int(axis), _p(c), len(c) - 1, int(rank)))

    def domain_sources(self, cycle, bank=None, M=0):
        _chk(self.L.mcgb_domain_sources(self.h, int(cycle), C.c_void_p(bank), int(M)))

    def domain_sweep(self):
        """Transport the slab's particles; returns how many leave it."""
        n = C.c_int64()
        _chk(self.L.mcgb_domain_sweep(self.h, C.byref(n)))
        return n.value

    def domain_outbox(self, out, cap):
        _chk(self.L.mcgb_domain_outbox(self.h, C.c_void_p(out), int(cap)))

    def domain_inbox(self, recs, n):
        _chk(self.L.mcgb_domain_inbox(self.h, C.c_void_p(recs), int(n)))

    def domain_export_sizes(self):
        m, ns = C.c_size_t(), C.c_size_t()
        _chk(self.L.mcgb_domain_export(self.h, None, None, 0, None, 0, C.byref(m), C.byref(ns)))
        return m.value, ns.value

    def domain_export(self, nfis, sites, sites_cap, sums, sums_cap):
        m, ns = C.c_size_t(), C.c_size_t()
        _chk(self.L.mcgb_domain_export(self.h, C.c_void_p(nfis), C.c_void_p(sites), int(sites_cap),
                                       C.c_void_p(sums), int(sums_cap), C.byref(m), C.byref(ns)))
        return m.value, ns.value

    def domain_import(self, cycle, sums, nfis, sites, M):
        _chk(self.L.mcgb_domain_import(self.h, int(cycle), C.c_void_p(sums), C.c_void_p(nfis),
                                       C.c_void_p(sites), int(M)))

    def domain_finish(self):
        _chk(self.L.mcgb_domain_finish(self.h))

    def domain_records(self, n_coll, n_cross, n_fis, fate, g_end, rng_end):
        _chk(self.L.mcgb_domain_records(self.h, *[C.c_void_p(a) for a in
                                                  (n_coll, n_cross, n_fis, fate, g_end, rng_end)]))

    def set_free_gas(self, kT, cut=0.0):
        _chk(self.L.mcgb_set_free_gas(self.h, float(kT), float(cut)))

    def set_time(self, t0, t_cut):
        _chk(self.L.mcgb_set_time(self.h, float(t0), float(t_cut)))

    def set_inverse_speeds(self, inv_v):
        a = _f64(inv_v)
        _chk(self.L.mcgb_set_inverse_speeds(self.h, len(a), _p(a)))

    def set_tally_time_bins(self, t, edges):
        a = _f64(edges)
        _chk(self.L.mcgb_set_tally_time_bins(self.h, t, len(a), _p(a)))

    def run_eigenvalue(self, n, inactive, active, seed):
        _chk(self.L.mcgb_run_eigenvalue(self.h, n, inactive, active, seed))

    def eigen_begin(self, n, inactive, active, seed):
        _chk(self.L.mcgb_eigen_begin(self.h, n, inactive, active, seed))

    def eigen_cycles(self, n_cycles):
        _chk(self.L.mcgb_eigen_cycles(self.h, n_cycles))

    def eigen_finish(self):
        _chk(self.L.mcgb_eigen_finish(self.h))

    def eigen_checkpoint(self):
        """The state of the power iteration between two cycles, as bytes."""
        need = C.c_size_t()
        _chk(self.L.mcgb_eigen_checkpoint(self.h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        _chk(self.L.mcgb_eigen_checkpoint(self.h, buf, need.value, C.byref(need)))
        return buf.raw

    def eigen_restore(self, blob):
        """Begin the power iteration again from eigen_checkpoint()'s bytes."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _chk(self.L.mcgb_eigen_restore(self.h, buf, len(blob)))

    def get_cycle_times(self, n):
        a, b = np.zeros(n), np.zeros(n)
        _chk(self.L.mcgb_get_cycle_times(self.h, n, _p(a), _p(b)))
        return a, b

    def get_event_timing(self):
        """Event mode: summed device time of each generation's first flight
        launch (the whole generation in one k_advance), the particles and
        launches it covers, and the algorithmic state bytes per particle."""
        ms, n, k, b = C.c_double(), C.c_int64(), C.c_int64(), C.c_double()
        _chk(self.L.mcgb_get_event_timing(self.h, C.byref(ms), C.byref(n), C.byref(k), C.byref(b)))
        return {"advance_ms": ms.value, "particles": n.value, "launches": k.value,
                "bytes_per_particle": b.value}

    def run_fixed_source(self, n, batches, seed):
        _chk(self.L.mcgb_run_fixed_source(self.h, n, batches, seed))

    def get_k(self):
        out = np.zeros(6)
        _chk(self.L.mcgb_get_k(self.h, _p(out)))
        return {"k": out[0], "k_sd": out[1], "k_col": out[2], "k_col_sd": out[3],
                "k_analog": out[4], "k_analog_sd": out[5]}

    def get_cycle_k(self, n):
        a, b, m = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.int64)
        _chk(self.L.mcgb_get_cycle_k(self.h, n, _p(a), _p(b), _p(m)))
        return a, b, m

    def tally_size(self, t=0):
        """(bins, energy bins or groups, time bins); 1 time bin without time bins."""
        nb, ne, nt = C.c_int(), C.c_int(), C.c_int()
        _chk(self.L.mcgb_tally_size(self.h, t, C.byref(nb), C.byref(ne), C.byref(nt)))
        return nb.value, ne.value, nt.value

    def get_tally(self, t=0):
        """Means and sds [bin, group or energy bin] (+ a time-bin axis when the
        tally has time bins)."""
        nb, ne, nt = self.tally_size(t)
        mean, sd = np.zeros(nb * ne * nt), np.zeros(nb * ne * nt)
        need = C.c_size_t()
        _chk(self.L.mcgb_get_tally(self.h, t, _p(mean), _p(sd), nb * ne * nt, C.byref(need)))
        shape = (nb, ne, nt) if t in getattr(self, "_timed_tallies", ()) else (nb, ne)
        return mean.reshape(shape), sd.reshape(shape)

    def get_counters(self):
        c = Counters()
        _chk(self.L.mcgb_get_counters(self.h, C.byref(c)))
        return {k: getattr(c, k) for k, _ in Counters._fields_}

    def get_histories(self):
        need = C.c_size_t()
        self.L.mcgb_get_histories(self.h, 0, None, None, None, None, None, None, C.byref(need))
        n = need.value
        nc, nx, nf, fate, g = (np.zeros(n, dtype=np.int32) for _ in range(5))
        rng = np.zeros(n, dtype=np.uint64)
        _chk(self.L.mcgb_get_histories(self.h, n, _p(nc), _p(nx), _p(rng), _p(nf), _p(fate),
                                       _p(g), C.byref(need)))
        return {"n_coll": nc, "n_cross": nx, "rng_end": rng, "n_fis": nf, "fate": fate, "g_end": g}

    def get_bank(self):
        need = C.c_size_t()
        self.L.mcgb_get_bank(self.h, 0, None, None, None, None, C.byref(need))
        n = need.value
        xyz = np.zeros((n, 3))
        par = np.zeros(n, dtype=np.int64)
        ch, mat = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
        _chk(self.L.mcgb_get_bank(self.h, n, _p(xyz), _p(par), _p(ch), _p(mat), C.byref(need)))
        return {"xyz": xyz, "parent": par, "child": ch, "mat": mat}

    def forward_fixed(self, n, seed, det_cell):
        out = np.zeros(self.G)
        _chk(self.L.mcgb_forward_fixed(self.h, n, seed, det_cell, _p(out)))
        return out

    def backward_fixed(self, weights, nmat):
        G = self.G
        w = _f64(weights)
        a, b, c = np.zeros(nmat * G), np.zeros(nmat * G * G), np.zeros(nmat * G)
        _chk(self.L.mcgb_backward_fixed(self.h, _p(w), _p(a), _p(b), _p(c)))
        return {"sigma_t": a.reshape(nmat, G), "sigma_s": b.reshape(nmat, G, G),
                "nu_sigma_f": c.reshape(nmat, G)}

    # device-pointer variants: arguments are device addresses (ints) on this
    # context's device, e.g. torch.Tensor.data_ptr() of contiguous float64 tensors
    def update_material_mg_dev(self, first, n_mat, sigma_t, sigma_s, nu_sigma_f):
        _chk(self.L.mcgb_update_material_mg_dev(self.h, int(first), int(n_mat), C.c_void_p(sigma_t),
                                                C.c_void_p(sigma_s), C.c_void_p(nu_sigma_f)))

    def forward_fixed_dev(self, n, seed, det_cell, tally):
        _chk(self.L.mcgb_forward_fixed_dev(self.h, int(n), int(seed), int(det_cell),
                                           C.c_void_p(tally)))

    def backward_fixed_dev(self, weights, d_sigma_t, d_sigma_s, d_nu_sigma_f):
        _chk(self.L.mcgb_backward_fixed_dev(self.h, C.c_void_p(weights), C.c_void_p(d_sigma_t),
                                            C.c_void_p(d_sigma_s), C.c_void_p(d_nu_sigma_f)))

    def rng_states(self, seed, first_id, n_streams, n_draws):
        out = np.zeros(n_streams * n_draws, dtype=np.uint64)
        _chk(self.L.mcgb_rng_states(self.h, seed, first_id, n_streams, n_draws, _p(out)))
        return out.reshape(n_streams, n_draws)

    def log(self, xi):
        x = _f64(xi)
        out = np.zeros_like(x)
        _chk(self.L.mcgb_log(self.h, len(x), _p(x), _p(out)))
        return out

    def fpint_ops(self, a, b):
        """The transport's float64 sqrt(a), a / b and 1 / b (integer-pipe,
        correctly rounded), as an (n, 3) array."""
        x, y = _f64(a).ravel(), _f64(b).ravel()
        if x.shape != y.shape:
            raise ValueError("a and b differ in length")
        out = np.zeros((len(x), 3))
        _chk(self.L.mcgb_fpint_ops(self.h, len(x), _p(x), _p(y), _p(out)))
        return out

    def fp64_throughput(self, iters=20000):
        """Measured FP64 thread-instructions per second of this device, and
        the timed launch in ms."""
        ops, ms = C.c_double(), C.c_double()
        _chk(self.L.mcgb_fp64_throughput(self.h, int(iters), C.byref(ops), C.byref(ms)))
        return ops.value, ms.value

    def probe(self, pos, direction):
        p, d = _f64(pos).reshape(-1, 3), _f64(direction).reshape(-1, 3)
        n = len(p)
        path = np.zeros((n, 5), dtype=np.int32)
        dist = np.zeros(n)
        kind = np.zeros(n, dtype=np.int32)
        _chk(self.L.mcgb_probe(self.h, n, _p(p), _p(d), _p(path), _p(dist), _p(kind)))
        return path, dist, kind

    def ce_lookup(self, mat, E):
        e = _f64(E)
        out = np.zeros((len(e), 4))
        _chk(self.L.mcgb_ce_lookup(self.h, mat, len(e), _p(e), _p(out)))
        return out

    # ---- convenience
    def run(self, **over):
        """Run the loaded problem with its own run settings (overridable)."""
        r = dict(self.problem["run"], **over)
        if r["mode"] == "eigen":
            self.run_eigenvalue(r["n"], r["inactive"], r["active"], r["seed"])
        else:
            self.run_fixed_source(r["n"], r["batches"], r["seed"])
        return self


def load_problem(ctx: Context, pb: dict) -> Context:
    """Define a problem description (see the workloads package) through the C calls."""
    for s in pb["surfaces"]:
        ctx.add_surface(SURF[s["type"]], s["coef"], BC[s["bc"]])
    for c in pb["cells"]:
        ctx.add_cell(c["universe"], c["surfs"], c["senses"], FILL[c["fill_kind"]], c["fill"])
    for L in pb["lattices"]:
        ctx.add_lattice(L["x0"], L["y0"], L["pitch"], L["nx"], L["ny"], L["universes"])
    if pb["G"] > 0:
        ctx.set_groups(pb["G"])
        for m in pb["materials"]:
            ctx.add_material_mg(m["sigma_t"], np.asarray(m["sigma_s"]).ravel(), m["nu_sigma_f"],
                                m["chi"])
    else:
        for u in pb["nuclides"]:
            ctx.add_nuclide_ce(u["A"], u["E"], u["sig_s"], u["sig_c"], u["sig_f"], u["nu"])
        for m in pb["materials"]:
            ctx.add_material_ce(m["nuclides"], m["density"])
    src = pb["source"]
    kind = 0 if src["kind"] == "box" else 1
    params = src["box"] if kind == 0 else src["point"]
    accept = 1 if src.get("accept") == "fissile" else 0
    ek = ENERGY[src["energy"]]
    energy = src["pdf"] if ek == 1 else ([src.get("E", 0.0)] if ek == 2 else [0.0])
    dk = 1 if src["direction"] == "beam" else 0
    ctx.set_source(kind, params, accept, ek, energy, dk, src.get("beam"))
    ctx._timed_tallies = set()
    for i, t in enumerate(pb["tallies"]):
        ctx.add_tally(FILTER[t["filter"]], t.get("edges"))
        if "time_edges" in t:
            ctx.set_tally_time_bins(i, t["time_edges"])
            ctx._timed_tallies.add(i)
    if "free_gas" in pb:
        ctx.set_free_gas(pb["free_gas"]["kT"], pb["free_gas"].get("cut", 0.0))
    if "time" in pb:
        ctx.set_time(pb["time"].get("t0", 0.0), pb["time"]["t_cut"])
        if pb["G"] > 0:
            ctx.set_inverse_speeds(pb["time"]["inv_v"])
    ctx.set_max_collisions(int(pb["run"].get("max_collisions", 0)))
    ctx.problem = pb
    return ctx


class Batch:
    """Many independent fixed-source problems run together (mcgb_batch)."""

    def __init__(self, device=0, mode=MODE_PERSISTENT, block=0, blocks_per_sm=0, pool=0):
        L = lib()
        self.L = L
        self.opts = Opts(device, mode, block, blocks_per_sm, 0, 0.0, 0, pool, 0)
        h = C.c_void_p()
        _chk(L.mcgb_batch_create(C.byref(h), C.byref(self.opts)))
        self.h = h
        self.ntallies = []

    def close(self):
        if getattr(self, "h", None):
            self.L.mcgb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def add_problem(self, ctx: Context, n, batches, seed):
        i = C.c_int()
        _chk(self.L.mcgb_batch_add_problem(self.h, ctx.h, n, batches, seed, C.byref(i)))
        self.ntallies.append(ctx)
        return i.value

    def autotune(self, budget_ms=2000):
        t = Tune()
        _chk(self.L.mcgb_batch_autotune(self.h, budget_ms, C.byref(t)))
        return {"block": t.block, "blocks_per_sm": t.blocks_per_sm, "pool": t.pool, "ms": t.ms}

    def run(self, tune=None):
        t = None if tune is None else Tune(tune["block"], tune["blocks_per_sm"],
                                          tune.get("pool", 0), 0.0)
        _chk(self.L.mcgb_batch_run(self.h, None if t is None else C.byref(t)))

    def tally(self, problem, t=0):
        ctx = self.ntallies[problem]
        nb, ne, nt = ctx.tally_size(t)
        mean, sd = np.zeros(nb * ne * nt), np.zeros(nb * ne * nt)
        need = C.c_size_t()
        _chk(self.L.mcgb_batch_tally(self.h, problem, t, _p(mean), _p(sd), nb * ne * nt,
                                     C.byref(need)))
        shape = (nb, ne, nt) if t in getattr(ctx, "_timed_tallies", ()) else (nb, ne)
        return mean.reshape(shape), sd.reshape(shape)

    def counters(self):
        c = Counters()
        _chk(self.L.mcgb_batch_counters(self.h, C.byref(c)))
        return {k: getattr(c, k) for k, _ in Counters._fields_}
