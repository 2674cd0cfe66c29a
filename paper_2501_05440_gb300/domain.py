"""Spatial domain decomposition of a k-eigenvalue power iteration: each rank
owns a slab of space along one axis and transports only the particles in it
(Sec. 1: MC/DC runs domain decomposed over MPI; here the ranks are
torch.distributed processes, one GPU each).

The library does the method (mcgb_domain_*): sources of the slab, transport
until a particle dies or reaches the slab's boundary -- where it stops with
the rest of its sampled collision distance, so that the next rank continues
the same flight without a new draw -- the statistics, the global bank order
and the resampling.  This module only moves bytes between ranks:

* after every sweep, the particles leaving each slab (128-byte records,
  addressed to the neighbouring rank) are gathered from all ranks; each rank
  keeps those addressed to it; sweeps repeat until no rank has one leaving;
* at the end of a cycle, the [k, tally] sums and the per-history site counts
  are summed over ranks and the sites every rank banked are gathered.

On NCCL the buffers stay on the GPU; on gloo (CPU ranks, or ranks sharing one
GPU) they are staged through host memory.  `run_domains_one_process` drives
several contexts, one per slab, from one process on one device -- the same
exchange without a process group.
"""

FLIGHT_BYTES = 128
SITE_BYTES = 64


def gather_rows(group, rows):
    """All ranks' rows (uint8 tensor [n, B], n may differ by rank), in rank
    order, on the input's device."""
    if group is None:
        return rows
    import torch
    world = group.get_world_size()
    home = rows.device
    dev = home if group.get_backend() == "nccl" else torch.device("cpu")
    m = torch.tensor([rows.shape[0]], dtype=torch.int64, device=dev)
    ms = torch.empty(world, dtype=torch.int64, device=dev)
    group.all_gather_into_tensor(ms, m)
    sizes = ms.tolist()
    mx = max(max(sizes), 1)
    padded = torch.zeros((mx, rows.shape[1]), dtype=torch.uint8, device=dev)
    padded[: rows.shape[0]] = rows.to(dev)
    out = torch.empty((world * mx, rows.shape[1]), dtype=torch.uint8, device=dev)
    group.all_gather_into_tensor(out, padded)
    return torch.cat([out[r * mx: r * mx + sizes[r]] for r in range(world)]).to(home)


def sum_over(group, t):
    """t summed over ranks (in place on a copy), on t's device."""
    if group is None:
        return t
    import torch
    dev = t.device if group.get_backend() == "nccl" else torch.device("cpu")
    s = t.to(dev).clone()
    group.all_reduce(s)
    return s.to(t.device)


def _cycle_end(ctx, N, dev):
    import torch
    m, ns = ctx.domain_export_sizes()
    nfis = torch.empty(N, dtype=torch.int32, device=dev)
    sites = torch.empty((max(m, 1), SITE_BYTES), dtype=torch.uint8, device=dev)
    sums = torch.empty(ns, dtype=torch.float64, device=dev)
    ctx.domain_export(nfis.data_ptr(), sites.data_ptr(), sites.shape[0], sums.data_ptr(), ns)
    return nfis, sites[:m], sums


def run_domain_eigen(ctx, N, inactive, active, seed, cuts, axis=0, group=None, max_sweeps=100000):
    """Power iteration of the problem loaded in `ctx` (a Context on this rank's
    GPU), this process owning slab `rank` of `cuts` (len = ranks + 1, -inf and
    +inf at the ends) along `axis`.  Afterwards ctx.get_k(), ctx.get_cycle_k()
    and ctx.get_tally() hold the whole run's results on every rank; returns
    the number of sweeps of every cycle."""
    import torch
    rank = group.get_rank() if group is not None else 0
    world = group.get_world_size() if group is not None else 1
    if len(cuts) != world + 1:
        raise ValueError("one slab per rank: len(cuts) must be ranks + 1")
    dev = torch.device("cuda", ctx.opts.device)
    ctx.set_stream(torch.cuda.current_stream(dev).cuda_stream)
    ctx.domain_begin(N, inactive, active, seed, axis, cuts, rank)
    sweeps = []
    for cyc in range(inactive + active):
        ctx.domain_sources(cyc)
        for k in range(max_sweeps):
            n_out = ctx.domain_sweep()
            out = torch.empty((max(n_out, 1), FLIGHT_BYTES), dtype=torch.uint8, device=dev)
            ctx.domain_outbox(out.data_ptr(), n_out)
            moving = gather_rows(group, out[:n_out])
            if moving.shape[0] == 0:
                break
            moving = moving.contiguous()
            ctx.domain_inbox(moving.data_ptr(), moving.shape[0])
        else:
            raise RuntimeError(f"cycle {cyc}: particles still moving after {max_sweeps} sweeps")
        sweeps.append(k + 1)
        nfis, sites, sums = _cycle_end(ctx, N, dev)
        nfis = sum_over(group, nfis).contiguous()
        sums = sum_over(group, sums).contiguous()
        sites = gather_rows(group, sites).contiguous()
        ctx.domain_import(cyc, sums.data_ptr(), nfis.data_ptr(), sites.data_ptr(), sites.shape[0])
    ctx.domain_finish()
    return sweeps


def run_domains_one_process(ctxs, N, inactive, active, seed, cuts, axis=0, max_sweeps=100000):
    """The same run with one context per slab driven from one process on one
    device (the contexts' kernels run one after the other and never wait on
    each other).  Every context ends with the whole run's results."""
    import torch
    if len(cuts) != len(ctxs) + 1:
        raise ValueError("one context per slab: len(cuts) must be contexts + 1")
    dev = torch.device("cuda", ctxs[0].opts.device)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for r, c in enumerate(ctxs):
        c.set_stream(stream)
        c.domain_begin(N, inactive, active, seed, axis, cuts, r)
    sweeps = []
    for cyc in range(inactive + active):
        for c in ctxs:
            c.domain_sources(cyc)
        for k in range(max_sweeps):
            outs = []
            for c in ctxs:
                n_out = c.domain_sweep()
                out = torch.empty((max(n_out, 1), FLIGHT_BYTES), dtype=torch.uint8, device=dev)
                c.domain_outbox(out.data_ptr(), n_out)
                outs.append(out[:n_out])
            moving = torch.cat(outs).contiguous()
            if moving.shape[0] == 0:
                break
            for c in ctxs:
                c.domain_inbox(moving.data_ptr(), moving.shape[0])
        else:
            raise RuntimeError(f"cycle {cyc}: particles still moving after {max_sweeps} sweeps")
        sweeps.append(k + 1)
        parts = [_cycle_end(c, N, dev) for c in ctxs]
        nfis = sum(p[0].to(torch.int64) for p in parts).to(torch.int32).contiguous()
        sums = sum(p[2] for p in parts).contiguous()
        sites = torch.cat([p[1] for p in parts]).contiguous()
        for c in ctxs:
            c.domain_import(cyc, sums.data_ptr(), nfis.data_ptr(), sites.data_ptr(), sites.shape[0])
    for c in ctxs:
        c.domain_finish()
    return sweeps
