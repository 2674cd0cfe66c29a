#!/usr/bin/env python
"""Benchmark of event-based Monte Carlo transport on GB300.

Headline: histories/s of k-eigenvalue power iteration on the C5G7-shaped
multigroup lattice (51x51 pins, 7 groups, 1e6 particles per cycle), one step =
one cycle (source from the resampled bank, transport of every history, bank
ordering, resampling, tallies), persistent event-loop form.  Beside it, in the
same JSON line: the plain one-kernel-per-event form and the monolithic
one-kernel-per-segment form (the paper's own GPU design) on the same workload, the
64-problem batched run against 64 separate plain runs, derivatives per second
through the replay-backward kernel, the paper's time-dependent
continuous-energy pin-cell benchmark (1e7 source histories), the FP64 roofline of the transport
kernel, the CPU oracle timed on this host's cores, and GPU clocks sampled
during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mcgb|reference]

Under torchrun (N > 1) every rank runs an independent replica (its own seed);
the histories of all ranks are added and divided by the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "histories/s on 1 GB300, batched vs plain event launch; % HBM roofline; grad/s"
WORKLOAD = "mg-c5g7-like-lattice-51x51-7g-keff"
# --workload: the headline problem (the lattice) or the continuous-energy pin
WORKLOADS = {"lattice": WORKLOAD, "ce-pin": "ce-pin-cell-4nuclides-keff"}
N_PER_CYCLE = 1_000_000
# Algorithmic particle-state bytes an event moves in the event-based form:
# advance reads position/direction/energy/RNG/cell path and writes position,
# RNG, event tag; collide or cross read and write direction, group, RNG and
# cell path (fields counted once per kernel that touches them).
STATE_BYTES_PER_EVENT = 120.0


def _hbm_peak():
    """The measured copy bandwidth of the GB300s (GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6777.0


HBM_PEAK_GBS = _hbm_peak()
# Counters from ncu captures of the transport kernels on the headline workload
# (one k_pool launch = one 1e6-history cycle; the first k_advance launch of an
# event-mode cycle).  They hold for the kernel sources they were taken on,
# NCU_SOURCES = paper_2501_05440_gb300.kernel_source_hash() of that build, and
# are reported as null once the sources differ.
#   fp64_inst_per_event: sm__thread_inst_executed_pipe_fp64_pred_on.sum of the
#   cycle's births kernel and transport kernel / events
#   dram_bytes_per_launch: dram__bytes_read.sum + dram__bytes_write.sum
#   l2_hit_rate: lts__t_sector_hit_rate; warp_exec_efficiency: active lanes per
#   issued instruction / 32; fp64_pipe_busy: FP64 pipe cycles / elapsed cycles
NCU_SOURCES = "8ef6620ef4fd8a01"
# k_source + k_pool of one cycle (2.233e7 events); DRAM bytes and rates of k_pool
NCU_K_POOL = {"fp64_inst_per_event": (818444896 + 13809408) / 2.233e7,
              "dram_bytes_per_launch": 129905408 + 72902144, "l2_hit_rate": 0.6307,
              "warp_exec_efficiency": 20.37 / 32, "fp64_pipe_busy": 0.4202,
              "births_kernel_dram_bytes": 59611392 + 101180416}
NCU_K_ADVANCE = {"dram_bytes_per_launch": 124712704 + 23436032, "l2_hit_rate": 0.4754,
                 "fp64_pipe_busy": 0.6500, "dram_throughput": 0.2374,
                 "fp64_inst_per_particle": 29000000 / 1e6}


def ncu_counters(m):
    """The recorded counters when they were taken on these kernel sources, else
    None (stale)."""
    if NCU_SOURCES is None or NCU_SOURCES != m.kernel_source_hash():
        return None, None
    return dict(NCU_K_POOL), dict(NCU_K_ADVANCE)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mcgb", choices=["mcgb", "reference"])
    ap.add_argument("--n", type=int, default=N_PER_CYCLE, help="particles per cycle")
    ap.add_argument("--quick", action="store_true", help="headline leg only")
    ap.add_argument("--pool", type=int, default=0,
                    help="persistent kernel variant (particles per warp/block in shared memory)")
    ap.add_argument("--graphs", type=int, default=0, help="0: cycles as CUDA graphs, -1: launches")
    ap.add_argument("--mode", default="persistent", choices=["persistent", "event", "segment"],
                    help="launch form of the headline leg (profiling the other forms)")
    ap.add_argument("--workload", default="lattice", choices=sorted(WORKLOADS),
                    help="problem of the headline leg: the lattice (the benchmark's) or, for "
                         "profiling, the continuous-energy pin cell")
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate(pg, ms, units):
    """Whole-job rate: units of every rank over the slowest rank's time (ms)."""
    ms_max = max_over_ranks(pg, ms)
    total = sum_over_ranks(pg, float(units))
    return ms_max, total, total / (ms_max / 1e3)


def replica_problem(W, n, rank, workload="lattice"):
    """The headline problem; replica `rank` draws from its own master seed."""
    pb = W.ce_pin_cell(seed=1, n=n) if workload == "ce-pin" else W.c5g7_like_lattice(seed=1, n=n)
    return W.with_run(pb, seed=int(pb["run"]["seed"]) + 1000003 * rank)


def sum_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def headline(m, W, torch, args, rank, pg):
    """Persistent form: K timed cycles after W warm-up cycles."""
    pb = replica_problem(W, args.n, rank, args.workload)
    mode = {"persistent": m.MODE_PERSISTENT, "event": m.MODE_EVENT,
            "segment": m.MODE_SEGMENT}[args.mode]
    c = m.Context(device=int(os.environ.get("LOCAL_RANK", "0")), mode=mode,
                  pool=args.pool, graphs=args.graphs)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    m.load_problem(c, pb)
    n = args.n
    c.eigen_begin(n, args.warmup, args.steps, pb["run"]["seed"])
    c.eigen_cycles(args.warmup)
    torch.cuda.synchronize()
    barrier(pg)
    launches0 = c.get_counters()["kernel_launches"]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    c.eigen_cycles(args.steps)
    e1.record()
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = c.get_counters()["kernel_launches"] - launches0
    c.eigen_finish()
    cnt = c.get_counters()
    ncyc = args.warmup + args.steps
    tms, cms = c.get_cycle_times(ncyc)
    k = c.get_k()
    events = (cnt["collisions"] + cnt["crossings"]) / ncyc    # per cycle (the cycles are alike)
    probe_clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    probe_clocks.start()
    fp64_ops, fp64_ms = c.fp64_throughput(iters=100_000)
    clk["fp64_probe"] = probe_clocks.stop()
    return {"ms": ms, "n": n, "launches": launches, "clocks": clk, "k": k,
            "fp64_ops_per_s": fp64_ops, "fp64_probe_ms": fp64_ms,
            "transport_ms": sum(tms[args.warmup:]) / args.steps,
            "cycle_ms": sum(cms[args.warmup:]) / args.steps, "events_per_cycle": events,
            "counters": cnt}


def plain_leg(m, W, torch, args, steps, mode=None):
    """Host-driven launch forms: one kernel per event type (MODE_EVENT) or the
    monolithic one-kernel-per-segment design of the paper's Sec. 2 (MODE_SEGMENT)."""
    mode = m.MODE_EVENT if mode is None else mode
    pb = W.c5g7_like_lattice(seed=1, n=args.n)
    c = m.Context(mode=mode)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    m.load_problem(c, pb)
    c.eigen_begin(args.n, 1, steps, 1)
    c.eigen_cycles(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    c.eigen_cycles(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c.eigen_finish()
    cnt = c.get_counters()
    events = (cnt["collisions"] + cnt["crossings"]) / (steps + 1)   # per cycle
    out = {"value": args.n * steps / (ms / 1e3), "unit": "histories/s",
           "mode": "segment" if mode == m.MODE_SEGMENT else "event",
           "ms_per_step": ms / steps, "steps": steps, "events_per_cycle": events,
           "event_iterations_per_cycle": cnt["event_iterations"] / (steps + 1)}
    # HBM roofline of the whole cycle: the algorithmic state bytes of every
    # event of the cycle over the cycle's time (all its launches)
    gbs_cycle = STATE_BYTES_PER_EVENT * events / (ms / steps / 1e3) / 1e9
    out["hbm_roofline_cycle"] = {"achieved": gbs_cycle, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                 "frac": gbs_cycle / HBM_PEAK_GBS,
                                 "basis": f"{STATE_BYTES_PER_EVENT:.0f} B/event x {events:.4g} "
                                          "events per cycle / cycle time (of measured copy bandwidth)"}
    if mode == m.MODE_EVENT:
        # HBM roofline of the flight kernel: each cycle's first k_advance launch
        # (the whole cycle's particles, identity list), timed with CUDA events
        # on the launching stream inside the library
        et = c.get_event_timing()
        _, adv = ncu_counters(m)
        if et["launches"] > 0 and et["advance_ms"] > 0:
            gbs = et["bytes_per_particle"] * et["particles"] / (et["advance_ms"] / 1e3) / 1e9
            out["roofline"] = {"bound": "hbm", "kernel": "k_advance (first flight of a cycle)",
                               "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                               "frac": gbs / HBM_PEAK_GBS,
                               "per_unit": f"{et['bytes_per_particle']:.0f} B/particle x "
                                           f"{et['particles'] / et['launches']:.4g} particles/launch",
                               "ms_per_launch": et["advance_ms"] / et["launches"],
                               "traffic": adv["dram_bytes_per_launch"] if adv else None,
                               "ncu": adv,
                               "peak_kind": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    return out


def e2e_leg(m, W, args, steps):
    """Through the public API with host buffers: define, upload, run, read back."""
    pb = W.c5g7_like_lattice(seed=1, n=args.n)
    t0 = time.perf_counter()
    c = m.Context(mode=m.MODE_PERSISTENT)
    m.load_problem(c, pb)
    c.run_eigenvalue(args.n, 0, steps, 1)
    k = c.get_k()
    mean, sd = c.get_tally(0)
    t1 = time.perf_counter()
    cnt = c.get_counters()
    d2h = mean.nbytes + sd.nbytes + 48 + 12 * steps
    return {"value": args.n * steps / (t1 - t0), "unit": "histories/s",
            "h2d_bytes_per_step": cnt["world_bytes"] / steps, "d2h_bytes_per_step": d2h / steps,
            "steps": steps, "k": k["k"]}


def batched_leg(m, W, torch):
    """64 fixed-source box problems: one batched persistent run vs 64 plain runs."""
    probs = W.batch_boxes()
    hist = sum(p["run"]["n"] for p in probs)
    ctxs = []
    for p in probs:
        c = m.Context(mode=m.MODE_EVENT)
        m.load_problem(c, p)
        ctxs.append(c)
    b = m.Batch(mode=m.MODE_PERSISTENT)
    for c, p in zip(ctxs, probs):
        b.add_problem(c, p["run"]["n"], p["run"]["batches"], p["run"]["seed"])
    tune = b.autotune(budget_ms=4000)
    b.run(tune)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(tune)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    for c, p in zip(ctxs, probs):     # warm-up of the separate runs
        c.run()
        break
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in ctxs:
        c.run()
    torch.cuda.synchronize()
    t_sep = time.perf_counter() - t0
    return {"histories": hist, "batched_persistent_s": t_batch, "separate_plain_s": t_sep,
            "batched_histories_per_s": hist / t_batch, "separate_histories_per_s": hist / t_sep,
            "speedup": t_sep / t_batch, "tune": tune}


def grad_leg(m, W, torch, n, reps=3):
    """Derivatives through the public torch API: DetectorTally on CUDA tensors
    (device-pointer calls, no host copies of any array), forward then backward
    of sum(tally), 1e7 histories of the slab; after one untimed pass at the
    same size, the median of `reps` host-timed passes."""
    import numpy as np

    from paper_2501_05440_gb300.autograd import detector_tally
    pb = W.diff_slab(n=n)
    dev = torch.device("cuda", torch.cuda.current_device())
    eng = m.load_problem(m.Context(device=dev.index, mode=m.MODE_PERSISTENT), pb)
    det = pb["detector_cell"]

    def xs():
        return [torch.tensor(np.array([mat[k] for mat in pb["materials"]]), device=dev,
                             requires_grad=True) for k in ("sigma_t", "sigma_s", "nu_sigma_f")]

    st, ss, nf = xs()     # warm-up at the full size (the engine's buffers allocated)
    detector_tally(pb, st, ss, nf, n, 1, det, engine=eng).sum().backward()
    fwd, bwd = [], []
    for _ in range(reps):
        st, ss, nf = xs()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y = detector_tally(pb, st, ss, nf, n, 1, det, engine=eng)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        y.sum().backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        fwd.append(t1 - t0)
        bwd.append(t2 - t1)
    tf, tb = sorted(fwd)[reps // 2], sorted(bwd)[reps // 2]
    return {"histories": n, "forward_s": tf, "backward_s": tb, "timing": f"median of {reps}",
            "grad_histories_per_s": n / tb, "forward_histories_per_s": n / tf,
            "detector_tally": float(y.detach().sum().item()),
            "api": "paper_2501_05440_gb300.autograd.DetectorTally on CUDA tensors",
            "grad_norm_sigma_t": float(st.grad.norm().item())}


def ce_leg(m, W, torch, steps=3):
    """Continuous-energy pin cell, 1e6 particles per cycle, persistent form."""
    pb = W.ce_pin_cell(seed=1, n=N_PER_CYCLE)
    c = m.Context(mode=m.MODE_PERSISTENT)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    m.load_problem(c, pb)
    c.eigen_begin(N_PER_CYCLE, 1, steps, 1)
    c.eigen_cycles(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    c.eigen_cycles(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c.eigen_finish()
    cnt = c.get_counters()
    ev = (cnt["collisions"] + cnt["crossings"]) / (steps + 1)
    return {"workload": "ce-pin-cell-4nuclides-keff", "value": N_PER_CYCLE * steps / (ms / 1e3),
            "unit": "histories/s", "ms_per_step": ms / steps, "events_per_s": ev * steps / (ms / 1e3),
            "k": c.get_k()["k"]}


def ce_time_leg(m, W, torch, n=10_000_000, sample=60_000):
    """The paper's continuous-energy benchmark shape (Sec. 4): infinite pin cell,
    uniform 14 MeV source, time-dependent fixed source with free-gas scattering,
    1e7 source histories; the CPU oracle on a `sample` of source histories."""
    pb = W.ce_time_pin(n=n)
    c = m.Context(mode=m.MODE_PERSISTENT, bank_factor=8.0)
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    m.load_problem(c, pb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    c.run()
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    cnt = c.get_counters()
    out = {"workload": "ce-pin-cell-4nuclides-time-14mev-free-gas", "source_histories": n,
           "s": s, "source_histories_per_s": n / s,
           "histories_incl_secondaries": cnt["histories"],
           "events_per_s": (cnt["collisions"] + cnt["crossings"]) / s,
           "generations": cnt["generations"], "time_cut": cnt["time_cut"]}
    import oracle
    cores = os.cpu_count() or 1
    o = oracle.Oracle(W.with_run(pb, n=sample))
    t0 = time.perf_counter()
    o.run(threads=cores)
    cpu_s = time.perf_counter() - t0
    out["cpu_oracle"] = {"source_histories_per_s": sample / cpu_s, "cores": cores,
                         "sample": f"{sample} source histories of the same problem"}
    from paper_2501_05440_gb300.report import core_equivalency
    out["core_equivalency"] = core_equivalency(cores, n / (sample / cpu_s), 1, s)
    return out


def _cpu_model():
    """The host CPU's model name (lscpu or /proc/cpuinfo), or the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(W, n=1_000_000, cycles=5, n1=50_000):
    """The oracle on this host's cores: `cycles` power-iteration cycles of the
    headline workload (all cores), and one cycle of n1 particles on one core."""
    import oracle
    cores = os.cpu_count() or 1
    pb = W.c5g7_like_lattice(seed=1, n=n, inactive=1, active=cycles - 1)
    o = oracle.Oracle(pb)
    t0 = time.perf_counter()
    o.run(threads=cores)
    dt = time.perf_counter() - t0
    o1 = oracle.Oracle(W.c5g7_like_lattice(seed=1, n=n1, inactive=0, active=1))
    t1 = time.perf_counter()
    o1.run(threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": n * cycles / dt, "unit": "histories/s", "cores": cores, "kind": "oracle",
            "sample": f"{cycles} power-iteration cycles of {WORKLOAD} at {n} particles, "
                      f"{dt:.2f} s wall on {cores} threads",
            "single_core": n1 / dt1, "single_core_sample": f"1 cycle of {n1} particles",
            "cpu_model": _cpu_model()}


def run_mcgb(args):
    import torch

    import paper_2501_05440_gb300 as m
    import workloads as W

    rank, world, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    m.build()
    h = headline(m, W, torch, args, rank, pg)
    ms_max, hist_total, value = aggregate(pg, h["ms"], h["n"] * args.steps)
    out = {
        "metric": METRIC, "value": value, "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "particles_per_cycle": h["n"],
                   "step": "one power-iteration cycle",
                   "mode": args.mode, "pool": args.pool, "graphs": args.graphs == 0, "l2": "inputs larger than L2 (particle state and fission "
                   "banks ~0.5 GB per GPU)", "parallelism": f"replicas x{world}"},
        "events_per_s": h["events_per_cycle"] * world / (ms_max / 1e3 / args.steps),
        "k": h["k"]["k"], "k_sd": h["k"]["k_sd"],
        "gpu_launches": h["launches"], "clocks": h["clocks"],
    }
    # roofline of the transport kernels (the generation's births, then the
    # persistent event loop: one launch of each per cycle, timed together with
    # CUDA events on their stream inside the library): bound by the FP64 pipe,
    # against the FP64 throughput measured in this run; the HBM fraction of the
    # event-based state traffic beside it
    ev = h["events_per_cycle"]
    t_kernel = max(h["transport_ms"], 1e-9) / 1e3
    pool, _ = ncu_counters(m) if args.workload == "lattice" else (None, None)
    ipe = pool["fp64_inst_per_event"] if pool else None
    peak = h["fp64_ops_per_s"] / 1e9
    ach = ipe * ev / t_kernel / 1e9 if ipe else None
    out["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak,
                       "unit": "G FP64 thread-instr/s", "frac": ach / peak if ach else None,
                       "traffic": pool["dram_bytes_per_launch"] if pool else None, "ncu": pool,
                       "kernel": "k_source + k_pool (the generation's births, then the persistent event loop)",
                       "per_unit": f"{ipe} FP64 instr/event (ncu) x {ev:.4g} events/launch",
                       "kernel_ms": h["transport_ms"],
                       "peak_kind": "measured in this run: mcgb_fp64_throughput (independent FMA "
                                    f"chains, {h['fp64_probe_ms']:.1f} ms launch)",
                       "kernel_sources": m.kernel_source_hash(), "ncu_sources": NCU_SOURCES}
    hbm = STATE_BYTES_PER_EVENT * ev / t_kernel / 1e9
    out["hbm_roofline"] = {"achieved": hbm, "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": hbm / HBM_PEAK_GBS,
                           "basis": f"{STATE_BYTES_PER_EVENT:.0f} B algorithmic state per event "
                                    "(of measured copy bandwidth)"}
    out["transport_ms_per_cycle"] = h["transport_ms"]
    if rank == 0 and not args.quick:
        out["plain_event"] = plain_leg(m, W, torch, args, max(2, args.steps // 4))
        out["monolithic_segment"] = plain_leg(m, W, torch, args, max(2, args.steps // 4),
                                              m.MODE_SEGMENT)
        out["e2e"] = e2e_leg(m, W, args, max(2, args.steps // 2))
        out["batched"] = batched_leg(m, W, torch)
        out["grad"] = grad_leg(m, W, torch, 10_000_000)
        out["ce_pin"] = ce_leg(m, W, torch)
        out["ce_time"] = ce_time_leg(m, W, torch)
        out["cpu_baseline"] = cpu_baseline(W)
        from paper_2501_05440_gb300.report import core_equivalency
        cb = out["cpu_baseline"]
        # Eq. 1 with run times of equal work (inverse rates): CPU cores per GPU
        out["core_equivalency"] = core_equivalency(cb["cores"], 1.0 / cb["value"], world,
                                                   1.0 / value)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_reference(args):
    """The CPU oracle on this host's cores, same workload and metric, bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workloads as W
    n = 50_000
    cores = os.cpu_count() or 1
    pb = W.c5g7_like_lattice(seed=1, n=n, inactive=args.warmup, active=args.steps)
    o = oracle.Oracle(pb)
    t0 = time.perf_counter()
    o.run(threads=cores)
    dt = time.perf_counter() - t0
    ncyc = args.warmup + args.steps
    value = n * ncyc / dt
    sample = (f"{WORKLOAD} at {n} particles per cycle (the GPU arm runs {N_PER_CYCLE}), "
              f"{ncyc} cycles on {cores} threads")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "histories/s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3 / ncyc, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "particles_per_cycle": N_PER_CYCLE,
                      "step": "one power-iteration cycle",
                      "sampled_particles_per_cycle": n},
           "cpu_baseline": {"value": value, "unit": "histories/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def launch_ranks(args):
    """--gpus N > 1 outside torchrun: start N ranks on this node (one process per
    GPU, rendezvous on 127.0.0.1) and return their exit status.  Refuses when
    the node has fewer GPUs than asked for."""
    import socket
    try:
        import torch
        have = torch.cuda.device_count()
    except Exception:
        have = 0
    if args.impl == "mcgb" and have < args.gpus:
        print(f"bench.py: --gpus {args.gpus} asked for, {have} CUDA device(s) visible; "
              "refusing to run fewer ranks", file=sys.stderr)
        return 2
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={args.gpus}", "--master-addr", "127.0.0.1",
           f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


if __name__ == "__main__":
    a = parse()
    world = os.environ.get("WORLD_SIZE")
    if world is None and a.gpus > 1:
        sys.exit(launch_ranks(a))
    if world is not None and int(world) != a.gpus:
        print(f"bench.py: --gpus {a.gpus} but WORLD_SIZE={world}; refusing", file=sys.stderr)
        sys.exit(2)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_mcgb(a)
