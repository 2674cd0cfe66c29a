"""Sharded k-eigenvalue power iteration: every cycle's N histories are split
into contiguous source-index ranges, one per rank (Sec. 1: MC/DC runs on many
nodes through MPI; here the ranks are torch.distributed processes, one GPU
each).

All of the method runs inside the library (mcgb_shard_*): transport of the
rank's slice, the ordered bank, the statistics, the resampling.  This module
only moves bytes between ranks, once per cycle (`exchange`): an all-reduce of
the ranks' [k_tl, k_c, tally] sums and an all-gather of their ordered banks as
64-byte site records.  Concatenated in rank order those banks are the global
(parent, child)-ordered bank, because the ranks' parent ranges are contiguous
and increasing.  On NCCL the buffers stay on the GPU
(all_gather_into_tensor, all_reduce on device tensors); on gloo (CPU ranks,
or ranks sharing one GPU) they are staged through host memory.  With one rank
the exchange is the identity and the run equals mcgb_run_eigenvalue's up to
the order of floating-point sums.
"""

SITE_BYTES = 64


def shard_range(N, rank, world):
    """Source indices [j0, j1) of `rank` among `world` ranks."""
    return N * rank // world, N * (rank + 1) // world


def exchange(group, sums, bank):
    """The per-cycle exchange: `sums` (float64 tensor) summed over ranks and
    `bank` (uint8 tensor [m, 64], this rank's ordered sites) gathered from all
    ranks in rank order.  Returns (global sums, global bank) on the inputs'
    device.  `group` is torch.distributed (or None for one rank)."""
    if group is None:
        return sums, bank
    import torch
    world = group.get_world_size()
    home = sums.device
    dev = home if group.get_backend() == "nccl" else torch.device("cpu")
    s = sums.to(dev)
    group.all_reduce(s)
    m = torch.tensor([bank.shape[0]], dtype=torch.int64, device=dev)
    ms = torch.empty(world, dtype=torch.int64, device=dev)
    group.all_gather_into_tensor(ms, m)
    sizes = ms.tolist()
    mx = max(max(sizes), 1)
    padded = torch.zeros((mx, SITE_BYTES), dtype=torch.uint8, device=dev)
    padded[: bank.shape[0]] = bank.to(dev)
    out = torch.empty((world * mx, SITE_BYTES), dtype=torch.uint8, device=dev)
    group.all_gather_into_tensor(out, padded)
    glob = torch.cat([out[r * mx: r * mx + sizes[r]] for r in range(world)])
    return s.to(home), glob.to(home)


def run_sharded_eigen(ctx, N, inactive, active, seed, group=None):
    """Power iteration of the problem loaded in `ctx` (a Context on this
    rank's GPU), this process being one rank of `group` (None: a single rank).
    Afterwards ctx.get_k(), ctx.get_cycle_k() and ctx.get_tally() hold the
    whole run's results on every rank; returns the last global bank (site
    records as a numpy structured array) and the rank's slice."""
    import numpy as np
    import torch

    from . import SITE_DTYPE
    rank = group.get_rank() if group is not None else 0
    world = group.get_world_size() if group is not None else 1
    j0, j1 = shard_range(N, rank, world)
    dev = torch.device("cuda", ctx.opts.device)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)   # the library and the copies below in one order
    ctx.shard_begin(N, j0, j1 - j0, inactive, active, seed)
    nsums = ctx.shard_sums_size()
    glob = None
    for cyc in range(inactive + active):
        m = ctx.shard_cycle(cyc)
        bank = torch.empty((max(m, 1), SITE_BYTES), dtype=torch.uint8, device=dev)
        sums = torch.empty(nsums, dtype=torch.float64, device=dev)
        ctx.shard_export(bank.data_ptr(), bank.shape[0], sums.data_ptr(), nsums)
        gsums, glob = exchange(group, sums, bank[:m])
        ctx.shard_import(cyc, gsums.contiguous().data_ptr(), glob.contiguous().data_ptr(),
                         glob.shape[0])
    ctx.shard_finish()
    last = np.frombuffer(glob.cpu().numpy().tobytes(), dtype=SITE_DTYPE)
    return {"bank": last, "rank": rank, "world": world, "j0": j0, "j1": j1}
