"""Sharded k-eigenvalue power iteration: every cycle's N histories are split
into contiguous source-index ranges, one per rank (Sec. 1: MC/DC runs on many
nodes through MPI; here the ranks are torch.distributed processes).

Per cycle each rank transports its slice on its own device (mcgb_shard_cycle),
then `exchange` -- the one place ranks communicate -- sums the k estimators and
tally sums over ranks and gathers every rank's (parent, child)-ordered bank;
concatenated in rank order those banks are the global bank, because the ranks'
parent ranges are contiguous and increasing.  Every rank then resamples its
own sources from the global bank with the cycle's draw, exactly as a single
device does (site of source j: floor((j + xi) M / N), clamped to M - 1).  With
one rank the exchange is the identity and the run equals mcgb_run_eigenvalue's
up to the order of floating-point sums.
"""

import numpy as np

from . import SITE_DTYPE


def shard_range(N, rank, world):
    """Source indices [j0, j1) of `rank` among `world` ranks."""
    return N * rank // world, N * (rank + 1) // world


def resample_indices(j0, j1, xi, M, N):
    """Global bank positions of sources j0..j1-1 (systematic resampling)."""
    j = np.arange(j0, j1, dtype=np.float64)
    t = (j + xi) * float(M) / float(N)
    idx = t.astype(np.int64)
    return np.minimum(idx, M - 1)


def exchange(group, ksum, tsum, bank):
    """The per-cycle exchange of a sharded power iteration.

    Returns (k sums over ranks, tally sums over ranks, global ordered bank).
    `group` is a torch.distributed module (or process group handle exposing
    all_reduce / all_gather_object) or None for a single rank."""
    if group is None:
        return np.asarray(ksum, float), np.asarray(tsum, float), bank
    import torch
    k = torch.tensor(np.concatenate([ksum, tsum]), dtype=torch.float64)
    group.all_reduce(k)
    k = k.numpy()
    banks = [None] * group.get_world_size()
    group.all_gather_object(banks, bank.tobytes())
    glob = np.concatenate([np.frombuffer(b, dtype=SITE_DTYPE) for b in banks])
    return k[:2], k[2:], glob


def run_sharded_eigen(ctx, N, inactive, active, seed, group=None):
    """Power iteration of the problem loaded in `ctx`, this process being one
    rank of `group` (None: a single rank).  Returns per-cycle k (track length,
    collision), bank sizes, k mean/sd over active cycles, tally means/sds per
    source particle (flat, layout of mcgb_get_tally) and the last global bank."""
    rank = group.get_rank() if group is not None else 0
    world = group.get_world_size() if group is not None else 1
    j0, j1 = shard_range(N, rank, world)
    ctx.shard_begin(N, j0, j1 - j0, seed)
    ncyc = inactive + active
    k_tl, k_c, bank_m = np.zeros(ncyc), np.zeros(ncyc), np.zeros(ncyc, dtype=np.int64)
    s = s2 = None
    ks = np.zeros(2)
    ks2 = np.zeros(2)
    sources = None
    glob = None
    for cyc in range(ncyc):
        ksum, _ = ctx.shard_cycle(cyc, sources)
        ksum_g, tsum_g, glob = exchange(group, ksum, ctx.shard_tally(), ctx.shard_bank())
        M = len(glob)
        if M == 0:
            raise RuntimeError(f"fission bank empty after cycle {cyc}")
        k_tl[cyc], k_c[cyc], bank_m[cyc] = ksum_g[0] / N, ksum_g[1] / N, M
        if cyc >= inactive:
            v = tsum_g / N
            s = v.copy() if s is None else s + v
            s2 = v * v if s2 is None else s2 + v * v
            kv = np.array([k_tl[cyc], k_c[cyc]])
            ks += kv
            ks2 += kv * kv
        sources = glob[resample_indices(j0, j1, ctx.cycle_xi(cyc), M, N)]

    def mean_sd(a, a2, n):
        mean = a / n
        var = (a2 - n * mean * mean) / (n - 1) if n > 1 else np.zeros_like(mean)
        return mean, np.sqrt(np.maximum(var, 0.0) / n) if n > 1 else np.zeros_like(mean)

    kmean, ksd = mean_sd(ks, ks2, active)
    tmean, tsd = (mean_sd(s, s2, active) if s is not None else (np.zeros(0), np.zeros(0)))
    return {"k_tl": k_tl, "k_col": k_c, "bank_m": bank_m, "k": kmean[0], "k_sd": ksd[0],
            "k_col_mean": kmean[1], "tally_mean": tmean, "tally_sd": tsd, "bank": glob,
            "rank": rank, "world": world, "j0": j0, "j1": j1}
