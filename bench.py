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
N_PER_CYCLE = 1_000_000
# FP64-pipe peak of one GB300: 152 SMs x 2 FP64 results per clock per SM x 2.07 GHz
# (the nominal 1.25 TFLOP/s counts an FMA as 2); a measured FP64 instruction
# throughput probe gave 504 G/s at the clocks it ran at.
FP64_PEAK_GOPS = 152 * 2 * 2.07
# FP64 thread-instructions per event of the persistent transport kernel on this
# workload: ncu sm__thread_inst_executed_pipe_fp64_pred_on.sum of one k_pool launch
# divided by the events of that cycle (1.455e9 / 2.246e7), profiles/k_pool_c5g7_lattice.md.
FP64_INST_PER_EVENT = 64.8
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
# DRAM bytes (read + write) of the first k_advance launch of a cycle (1e6
# particles) from an ncu capture, or None when the kernel has changed since.
ADVANCE_TRAFFIC_PER_LAUNCH = 124725504 + 25844480
# DRAM bytes (read + write) of one k_pool launch from the same ncu capture, or None
# when the kernel has changed since the counters were taken.
TRAFFIC_PER_LAUNCH = 79513600 + 90772992
# Other counters of the same two captures (profiles/k_pool_c5g7_lattice.md,
# profiles/event_mode_c5g7_lattice.md): L2 sector hit rate, active lanes per
# issued instruction / 32, FP64 pipe busy fraction of the elapsed time.
NCU_K_POOL = {"l2_hit_rate": 0.8478, "warp_exec_efficiency": 20.34 / 32, "fp64_pipe_busy": 0.4798,
              "source": "profiles/k_pool_c5g7_lattice.md"}
NCU_K_ADVANCE = {"l2_hit_rate": 0.4982, "fp64_pipe_busy": 0.7524, "dram_throughput": 0.1546,
                 "source": "profiles/event_mode_c5g7_lattice.md"}


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


def replica_problem(W, n, rank):
    """The headline problem; replica `rank` draws from its own master seed."""
    pb = W.c5g7_like_lattice(seed=1, n=n)
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
    pb = replica_problem(W, args.n, rank)
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
    return {"ms": ms, "n": n, "launches": launches, "clocks": clk, "k": k,
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
    out = {"value": args.n * steps / (ms / 1e3), "unit": "histories/s",
           "mode": "segment" if mode == m.MODE_SEGMENT else "event",
           "ms_per_step": ms / steps, "steps": steps,
           "event_iterations_per_cycle": cnt["event_iterations"] / (steps + 1)}
    if mode == m.MODE_EVENT:
        # HBM roofline of the flight kernel: each cycle's first k_advance launch
        # (the whole cycle's particles, identity list), timed with CUDA events
        # on the launching stream inside the library
        et = c.get_event_timing()
        if et["launches"] > 0 and et["advance_ms"] > 0:
            gbs = et["bytes_per_particle"] * et["particles"] / (et["advance_ms"] / 1e3) / 1e9
            out["roofline"] = {"bound": "hbm", "kernel": "k_advance (first flight of a cycle)",
                               "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                               "frac": gbs / HBM_PEAK_GBS,
                               "per_unit": f"{et['bytes_per_particle']:.0f} B/particle x "
                                           f"{et['particles'] / et['launches']:.4g} particles/launch",
                               "ms_per_launch": et["advance_ms"] / et["launches"],
                               "traffic": ADVANCE_TRAFFIC_PER_LAUNCH, "ncu": NCU_K_ADVANCE,
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


def grad_leg(m, W, torch, n):
    pb = W.diff_slab(n=n)
    c = m.Context(mode=m.MODE_PERSISTENT)
    m.load_problem(c, pb)
    det = pb["detector_cell"]
    c.forward_fixed(min(n, 10000), 1, det)
    c.backward_fixed([1.0] * pb["G"], len(pb["materials"]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tal = c.forward_fixed(n, 1, det)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    c.backward_fixed([1.0] * pb["G"], len(pb["materials"]))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"histories": n, "forward_s": t1 - t0, "backward_s": t2 - t1,
            "grad_histories_per_s": n / (t2 - t1), "forward_histories_per_s": n / (t1 - t0),
            "detector_tally": float(tal.sum())}


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
        "config": {"workload": WORKLOAD, "particles_per_cycle": h["n"], "step": "one power-iteration cycle",
                   "mode": args.mode, "pool": args.pool, "graphs": args.graphs == 0, "l2": "inputs larger than L2 (particle state and fission "
                   "banks ~0.5 GB per GPU)", "parallelism": f"replicas x{world}"},
        "events_per_s": h["events_per_cycle"] * world / (ms_max / 1e3 / args.steps),
        "k": h["k"]["k"], "k_sd": h["k"]["k_sd"],
        "gpu_launches": h["launches"], "clocks": h["clocks"],
    }
    # roofline of the transport kernel (the persistent event loop, one launch per cycle):
    # bound by the FP64 pipe; the HBM fraction of the event-based state traffic beside it
    ev = h["events_per_cycle"]
    t_kernel = max(h["transport_ms"], 1e-9) / 1e3
    ach = FP64_INST_PER_EVENT * ev / t_kernel / 1e9
    out["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GOPS,
                       "unit": "G FP64 thread-instr/s", "frac": ach / FP64_PEAK_GOPS,
                       "traffic": TRAFFIC_PER_LAUNCH, "ncu": NCU_K_POOL,
                       "kernel": "k_pool (persistent event loop)",
                       "per_unit": f"{FP64_INST_PER_EVENT} FP64 instr/event x {ev:.4g} events/launch",
                       "peak_kind": "derived: 152 SMs x 2 FP64/clk x 2.07 GHz (recipe's 1.25 TFLOP/s)"}
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


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_mcgb(a)
