"""Helpers for GPU tests: run a workload on the CUDA library and on the oracle."""
import numpy as np

import workloads as W
from oracle import Oracle


def gpu_run(pb, mode=0, record=True, pool=0, graphs=0, **over):
    import paper_2501_05440_gb300 as m
    c = m.Context(mode=mode, record_histories=record, pool=pool, graphs=graphs)
    m.load_problem(c, pb)
    c.run(**over)
    return c


def oracle_run(pb, threads=0, strict=True, **over):
    """The oracle on the same problem; strict (the CUDA library's rounding
    conventions) for bit-for-bit comparisons, plain for tolerance ones."""
    return Oracle(pb, strict=strict).run(threads=threads, **over)


def assert_same_histories(hg, ho):
    for k in ["n_coll", "n_cross", "rng_end", "n_fis", "fate", "g_end"]:
        a, b = np.asarray(hg[k]), np.asarray(ho[k])
        assert a.shape == b.shape, k
        bad = np.nonzero(a != b)[0]
        assert len(bad) == 0, (k, len(bad), bad[:10], a[bad[:5]], b[bad[:5]])


def rel_close(a, b, rtol, atol=0.0):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.all(np.abs(a - b) <= rtol * np.abs(b) + atol)
