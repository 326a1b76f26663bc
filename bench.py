#!/usr/bin/env python3
"""Throughput of the photon-packet life cycle on GB300.

One step = one skirt_trace call over the whole workload: the exponential-disk
galaxy on a 256^3 grid, 1e8 packets at one optical wavelength, three
512x512 instruments (inclinations 0/60/90 deg), traced in the mixed form
(FP32 traversal and phase-function sampling, FP64 optical-depth sums and
tallies) by one persistent launch replayed from a CUDA graph.  Inputs are
resident in HBM when the timed region starts; L2 is flushed (256 MB write)
before every timed step.

The schedule (block size, refill chunk, resident blocks, step_min) is picked
by the library's autotuner on a 2% sample before the timed region; the
default schedule is timed beside it.  Reported next to the headline: the
plain FP64 form on 1e7 packets of the same workload, the end-to-end time
through the C ABI with pinned host buffers, the rooflines of the trace
kernel (HBM bytes, FP64 reductions, the binding one as "roofline"), the CPU
FP64 oracle timed on a sample, on one core and on every host core, and the
batched form ("batched": the clumpy torus with 200 wavelengths of uneven
packet counts, 7.5e8 packets, one persistent graph launch) with its own
rooflines and the plain FP64 form through the same persistent schedule.

`--impl reference` times the oracle (the slow, plain CPU program the
parity tests compare against) on every host core instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon packets×wavelengths/s on 1 GB300 (FP32+batched vs plain FP64, at 1e-4 rel)"
UNIT = "packets*lambda/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=float, default=1e8)
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--fp64-packets", type=float, default=1e7)
    ap.add_argument("--cpu-packets", type=int, default=None,
                    help="oracle sample per core (default 60000; 2000 on the octree, whose oracle lists "
                         "every finest-lattice plane)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="trace with the default schedule instead of the autotuned one")
    ap.add_argument("--tune-fraction", type=float, default=0.02, help="autotuner sample (fraction of the packets)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form (200-wavelength torus) record")
    ap.add_argument("--batched-steps", type=int, default=1)
    ap.add_argument("--batched-fp64-fraction", type=float, default=0.005,
                    help="plain FP64 sample of the batched form (fraction of its packets)")
    ap.add_argument("--epochs", type=int, default=200, help="learned workload: training epochs")
    ap.add_argument("--batch", type=int, default=2048, help="learned workload: training batch")
    ap.add_argument("--lr", type=float, default=2e-3, help="learned workload: Adam step size")
    ap.add_argument("--cells", type=int, default=2_000_000, help="exact workload: cells")
    ap.add_argument("--workload", default="disk",
                    choices=["disk", "disk40", "torus", "octree", "learned", "selfabs", "exact"],
                    help="disk: 1 wavelength, --packets packets (default); disk40: 40 wavelengths, "
                         "--packets per wavelength; torus: clumpy torus, 200 wavelengths, uneven counts "
                         "(--packets scales them, 1e8 = the full 7.5e8-packet run); octree: the disk galaxy "
                         "on an 8.25M-leaf octree, 1 wavelength, --packets packets; exact: the exact dust "
                         "emission solve of --cells synthetic cells with 200 absorbed wavelengths")
    a = ap.parse_args()
    if a.cpu_packets is None:
        a.cpu_packets = 2000 if a.workload == "octree" else 60000
    return a


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(args):
    from paper_1705_04702_gb300 import workloads as W
    if args.workload == "disk40":
        return W.disk_problem(int(args.packets), n=args.grid, nlambda=40, npx=512)
    if args.workload == "torus":
        return W.torus_problem(n=args.grid, nlambda=200, npx=512, packet_scale=args.packets / 1e8)
    if args.workload == "octree":
        return W.octree_problem(W.disk_octree(), int(args.packets), npx=512)
    return W.disk_problem(int(args.packets), n=args.grid, nlambda=1, npx=512)


def workload_name(args, prob):
    if args.workload == "disk40":
        return (f"exponential-disk galaxy, {args.grid}^3 Cartesian grid, 40 wavelengths 0.1-5 um, "
                f"{int(args.packets):.0e} packets per wavelength, 3 instruments 512x512 (i=0/60/90)")
    if args.workload == "torus":
        return (f"clumpy two-phase dust torus, {args.grid}^3 Cartesian grid, 200 wavelengths 0.09-10 um, "
                f"{prob.total_packets:.3e} packets (1e5-2e7 per wavelength, log-uniform), "
                f"3 instruments 512x512 (i=0/60/90)")
    if args.workload == "octree":
        lv = prob.grid.leaves[:, 0]
        return (f"exponential-disk galaxy on an octree dust grid over [-24,24]^3: {prob.grid.ncell} leaves "
                f"(levels {lv.min()}-{lv.max()}, at most {prob.grid.max_level}), 1 wavelength (0.55 um), "
                f"{int(args.packets):.0e} packets, 3 instruments 512x512 (i=0/60/90)")
    return (f"exponential-disk galaxy, {args.grid}^3 Cartesian grid, 1 wavelength (0.55 um), "
            f"{int(args.packets):.0e} packets, 3 instruments 512x512 (i=0/60/90)")


def config_of(args, prob, extra=None):
    c = {
        "workload": workload_name(args, prob),
        "grid": f"octree, {prob.grid.ncell} leaves" if args.workload == "octree" else args.grid,
        "nlambda": prob.wl.n,
        "packets_per_step": prob.total_packets,
        "instruments": len(prob.instruments),
        "npx": 512,
        "l2": "flushed by a 256 MB write before every timed step",
    }
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ oracle on CPU
def packet_lambdas(npk, lo, hi):
    """Packet-wavelengths in packet range [lo, hi) of every wavelength."""
    return int(np.clip(np.minimum(npk.astype(np.int64), hi) - lo, 0, None).sum())


def _oracle_serve(spec, tasks, done):
    """Worker process: builds the workload once, then traces the packet
    ranges it is sent with the unmodified oracle and reports the
    packet-wavelengths it traced."""
    import oracle
    prob = workload(argparse.Namespace(**spec))
    done.put(0)
    while True:
        r = tasks.get()
        if r is None:
            break
        oracle.trace(prob, r[0], r[1])
        done.put(packet_lambdas(prob.npk, r[0], r[1]))


class OraclePool:
    """The oracle on every host core: one spawned process per core (started
    before any GPU work), each tracing its own packet range of a step."""

    def __init__(self, args, cores=None):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.cores = cores or os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        spec = {"workload": args.workload, "packets": args.packets, "grid": args.grid}
        self.tasks = [ctx.Queue() for _ in range(self.cores)]
        self.done = ctx.Queue()
        self.procs = [ctx.Process(target=_oracle_serve, args=(spec, q, self.done), daemon=True) for q in self.tasks]
        for p in self.procs:
            p.start()
        for _ in self.procs:
            self.done.get()

    def step(self, lo, per_core):
        """Packets [lo + i per_core, lo + (i + 1) per_core) on core i; returns
        (packet-wavelengths traced, wall seconds)."""
        t0 = time.perf_counter()
        for i, q in enumerate(self.tasks):
            q.put((lo + i * per_core, lo + (i + 1) * per_core))
        n = sum(self.done.get() for _ in self.tasks)
        return n, time.perf_counter() - t0

    def close(self):
        for q in self.tasks:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)


# ------------------------------------------------------------------ reference
def run_reference(args):
    """The CPU FP64 oracle on every host core, a bounded sample per step (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = workload(args)
    pool = OraclePool(args)
    per_core = max(1, min(args.cpu_packets // 3, int(args.packets) // max(pool.cores * (args.warmup + args.steps), 1)))
    lo = 0
    for _ in range(args.warmup):
        pool.step(lo, per_core)
        lo += pool.cores * per_core
    n_tot, dt = 0, 0.0
    for _ in range(args.steps):
        n, t = pool.step(lo, per_core)
        n_tot += n
        dt += t
        lo += pool.cores * per_core
    pool.close()
    value = n_tot / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_of(args, prob, {"sample_per_step": pool.cores * per_core}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"{pool.cores} processes x {per_core} packets of every wavelength per step "
                                   f"(disjoint packet ranges) of the workload, single-threaded FP64 oracle each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ replicas
def replica_seed(rank):
    """Every rank traces its own packets: the Philox key differs per rank."""
    return 1 + rank


def job_time(elapsed, dist=None, device=None):
    """Wall time of the whole job: the slowest rank's timed region."""
    if dist is None:
        return elapsed
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, steps, elapsed):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * world * steps / elapsed


# ------------------------------------------------------------------ learned
def run_learned_report(args):
    """The learned form on the clumpy torus (256^3, 200 wavelengths, then a
    1e8-packet re-emission trace): stage times, surrogate error and
    speedups, as one JSON line (not the headline metric)."""
    import torch
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300.learned import run_learned
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rep = run_learned(n=args.grid, nlambda=200, packet_scale=args.packets / 1e8, n_train=1_000_000,
                      n_test=100_000, epochs=args.epochs, batch=args.batch, lr=args.lr,
                      reemit_per_lambda=1_000_000)
    rep = {k: v for k, v in rep.items() if not k.startswith("_")}
    print(json.dumps({"report": "learned form", "workload": f"clumpy torus {args.grid}^3, 200 wavelengths",
                      **rep}), flush=True)


def run_exact_report(args):
    """The exact FP64 dust-emission solve (equilibrium temperatures of three
    grain populations, 100 emission wavelengths) on --cells synthetic cells
    absorbing on 200 wavelengths 0.09-10 um: device time per call, as one
    JSON line (not the headline metric)."""
    import torch
    from paper_1705_04702_gb300 import build
    from paper_1705_04702_gb300 import workloads as W
    build.build()
    from paper_1705_04702_gb300 import skirt as S
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lam = np.geomspace(0.09, 10.0, 200)
    a, m = W.absorbed_spectra(args.cells, lam, seed=3)
    a_d = torch.as_tensor(a, dtype=torch.float64, device="cuda")
    m_d = torch.as_tensor(m, dtype=torch.float32, device="cuda")
    del a
    em = torch.empty((args.cells, S.NEMIT), dtype=torch.float64, device="cuda")
    ms = []
    for _ in range(args.warmup + args.steps):
        st = S.skirt_dust_emission(a_d, args.cells, lam.size, lam, m_d, S.EMIT_EXACT, None, em)
        ms.append(st["ms_exact"])
    ms = ms[args.warmup:]
    print(json.dumps({"report": "exact dust emission", "cells": args.cells, "n_in": int(lam.size),
                      "ms_per_call": float(np.mean(ms)), "cells_per_s": args.cells / (np.mean(ms) / 1e3)}),
          flush=True)


def run_selfabs_report(args):
    """Dust self-absorption cycles on the clumpy torus (256^3, 200 stellar
    wavelengths, then 1e6 dust packets per emission wavelength per cycle):
    cycle count and per-stage times, as one JSON line (not the headline
    metric)."""
    import torch
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt as S
    from paper_1705_04702_gb300 import workloads as W
    from paper_1705_04702_gb300.selfabsorb import self_absorption
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    prob = W.torus_problem(n=args.grid, nlambda=200, npx=512, packet_scale=args.packets / 1e8)
    grid = S.Grid(prob.grid)
    ncell, NL = grid.ncell, prob.wl.n
    absorbed = torch.zeros((ncell, NL), dtype=torch.float64, device="cuda")
    opts = S.skirt_trace_opts_default()
    opts.use_graph = 1
    opts.peel = 0
    tables = S.Tables(prob.wl)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, led, _ = S.skirt_trace(grid.h, S.make_source(prob.source), tables.c, prob.npk, prob.seed, [], opts, absorbed,
                              None, None)
    torch.cuda.synchronize()
    t_star = time.perf_counter() - t0
    mass = torch.empty(ncell, dtype=torch.float32, device="cuda")
    S.skirt_dust_mass(grid.h, mass)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = self_absorption(grid, absorbed, prob.wl.lam, mass, 1_000_000, prob.seed, tol=1e-2, max_cycles=10)
    torch.cuda.synchronize()
    t_cycles = time.perf_counter() - t0
    grid.close()
    hist = [{"emitted": h["emitted"], "absorbed": h["absorbed"], "kernel_ms": h["ledger"]["kernel_ms"]}
            for h in out["history"]]
    print(json.dumps({"report": "dust self-absorption cycles",
                      "workload": f"clumpy torus {args.grid}^3, 200 stellar wavelengths "
                                  f"({prob.total_packets:.3e} packets, no peel-off), 100 dust wavelengths, "
                                  f"1e6 dust packets per wavelength per cycle",
                      "t_stellar_trace": t_star, "stellar_absorbed": led["absorbed"], "cycles": out["cycles"],
                      "converged": out["converged"], "t_cycles": t_cycles, "t_per_cycle": t_cycles / out["cycles"],
                      "history": hist}), flush=True)


# ----------------------------------------------------------------------- ours
# Warp instructions per packet of trace_mixed_kernel on the 256^3 disk, from
# the committed ncu capture of the kernel as it stands
# (profiles/trace_mixed_kernel_disk256_3e6_full.md); None when the kernel has
# changed since.
ISSUE_INST_PER_PACKET = 23468.0
# DRAM bytes (read + write) per packet of the trace kernel from one ncu
# capture of a 3e6-packet launch of the kernel as it stands (profiles/),
# scaled by the packets of the launch; None when the kernel has changed since.
TRAFFIC_PER_PACKET = {"disk": 30254.0, "octree": 102039.0}


def trace_rooflines(led, packets, k_ms, ninstr, red_rate, peak, peak_kind, kernel, crossing_bytes, traffic_pp,
                    clock_mhz=None, sm_count=None):
    """Rooflines of one trace launch: algorithmic bytes
    (the crossing's read, a 16-byte read-modify-write per deposit and per
    peel-off tally) against the measured copy bandwidth; FP64 reductions (one
    per deposit and per tally) against the random red.f64 rate measured in the
    same run; the bound is the one that binds (the larger fraction)."""
    steps = led["deposit_steps"] + led["locate_steps"] + led["peel_steps"]
    tallies = (packets + led["scatterings"]) * ninstr
    byts = crossing_bytes * steps + 16 * led["deposit_steps"] + 16 * tallies
    t = k_ms / 1e3
    hbm = {"bound": "hbm", "achieved": byts / t / 1e9, "peak": peak, "unit": "GB/s",
           "frac": byts / t / 1e9 / peak, "traffic": traffic_pp * packets if traffic_pp else None,
           "peak_source": peak_kind, "kernel": kernel, "kernel_ms": k_ms, "algorithmic_bytes_per_launch": byts,
           "per_packet": {"deposit_steps": led["deposit_steps"] / packets, "locate_steps": led["locate_steps"] / packets,
                          "peel_steps": led["peel_steps"] / packets, "scatterings": led["scatterings"] / packets}}
    reds = led["deposit_steps"] + tallies
    atom = {"bound": "atomics", "achieved": reds / t, "peak": red_rate, "unit": "red.f64/s",
            "frac": reds / t / red_rate, "traffic": hbm["traffic"], "kernel": kernel, "kernel_ms": k_ms,
            "atomics_per_packet": reds / packets,
            "peak_source": "measured in this run: random red.global.add.f64 into a table of the absorbed table's size"}
    if atom["frac"] > 1.0:
        # the deposits of a traversal share sectors (consecutive cells along x;
        # wavelength-major tables), which the random-address microbenchmark
        # does not: its rate is then no bound for this kernel
        atom["note"] = "not a bound for this access stream (fraction > 1: deposits share sectors)"
        binding = dict(hbm)
    else:
        binding = dict(atom if atom["frac"] >= hbm["frac"] else hbm)
    binding["min_of"] = {"hbm_frac": hbm["frac"], "atomics_frac": atom["frac"]}
    out = {"roofline": binding, "roofline_hbm": hbm, "roofline_atomic": atom}
    if ISSUE_INST_PER_PACKET and clock_mhz and sm_count:
        cap = sm_count * 4 * clock_mhz * 1e6 / ISSUE_INST_PER_PACKET
        out["roofline_issue"] = {"bound": "issue", "achieved": packets / t, "peak": cap, "unit": "packets/s",
                                 "frac": packets / t / cap, "warp_inst_per_packet": ISSUE_INST_PER_PACKET,
                                 "note": "4 warp instructions per SM per cycle at the median SM clock of the run"}
    return out


def run_steps(S, grid, src, tables, prob, seed, ins, opts, outs, steps, warmup, flush, stream, barrier, clocks=None):
    """warmup untimed then `steps` timed trace calls (L2 flushed before
    each; the clock sampler, if given, runs over the timed calls); returns
    (elapsed seconds, per-launch kernel ms, last ledger)."""
    import torch
    absorbed, images, sed = outs

    def step():
        return S.skirt_trace(grid.h, src, tables.c, prob.npk, seed, ins, opts, absorbed, images, sed,
                             stream=stream.cuda_stream)

    for _ in range(warmup):
        flush.zero_()
        step()
    barrier()
    if clocks is not None:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = []
    led = None
    ev0.record(stream)
    for _ in range(steps):
        flush.zero_()
        _, led, _ = step()
        kernel_ms.append(led["kernel_ms"])
    ev1.record(stream)
    barrier()
    return ev0.elapsed_time(ev1) / 1e3, kernel_ms, led


def plain_fp64(S, grid, src, tables, prob, seed, ins, outs, fraction, schedule, stream, barrier):
    """The plain FP64 form on a sample of the workload (every wavelength's
    packets scaled by fraction): one warm-up call, then one timed call."""
    absorbed, images, sed = outs
    p64 = prob.with_packets(np.maximum(np.round(prob.npk.astype(np.float64) * fraction), prob.npk > 0)
                            .astype(np.uint64))
    o64 = S.skirt_trace_opts_default()
    o64.precision = S.PREC_FP64
    o64.schedule = schedule
    small = prob.with_packets(np.minimum(p64.npk, 1000))
    S.skirt_trace(grid.h, src, tables.c, small.npk, seed, ins, o64, absorbed, images, sed, stream=stream.cuda_stream)
    barrier()
    t0 = time.perf_counter()
    _, l64, _ = S.skirt_trace(grid.h, src, tables.c, p64.npk, seed, ins, o64, absorbed, images, sed,
                              stream=stream.cuda_stream)
    barrier()
    dt = time.perf_counter() - t0
    return {"value": p64.total_packets / dt, "unit": UNIT, "packets": p64.total_packets, "kernel_ms": l64["kernel_ms"],
            "precision": "fp64",
            "schedule": "persistent (one launch for all wavelengths)" if schedule == S.SCHED_PERSISTENT
            else "one launch per wavelength"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "learned":
        run_learned_report(args)
        return
    if args.workload == "selfabs":
        run_selfabs_report(args)
        return
    if args.workload == "exact":
        run_exact_report(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # the CPU baseline runs before any GPU work (rank 0, single GPU only)
    cpu = None
    prob = workload(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        per = max(1, args.cpu_packets // prob.wl.n)  # packets per wavelength per core
        n1 = packet_lambdas(prob.npk, 0, per)
        t0 = time.perf_counter()
        oracle.trace(prob, 0, per)
        dt1 = time.perf_counter() - t0
        pool = OraclePool(args)
        n, dt = pool.step(per, per)
        pool.close()
        cpu = {"value": n / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
               "sample": f"{pool.cores} processes, each tracing its own {per} packets of every wavelength "
                         f"({n} packet-wavelengths in all) with the single-threaded FP64 oracle, {dt:.1f} s wall",
               "one_core": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"packets 0..{per - 1} of every wavelength ({n1} packet-wavelengths), "
                                      f"{dt1:.1f} s"}}

    import torch
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt as S

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    seed = replica_seed(rank)  # independent replicas: every rank traces its own packets
    prob.seed = seed
    grid = S.Grid(prob.grid)
    n = prob.wl.n
    npix = sum(i.npx * i.npx for i in prob.instruments) * n
    absorbed = torch.zeros((grid.ncell, n), dtype=torch.float64, device="cuda")
    images = torch.zeros(npix, dtype=torch.float64, device="cuda")
    sed = torch.zeros((len(prob.instruments), n), dtype=torch.float64, device="cuda")
    outs = (absorbed, images, sed)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    tables = S.Tables(prob.wl)
    ins = S.make_instruments(prob.instruments)
    src = S.make_source(prob.source)
    opts = S.skirt_trace_opts_default()
    opts.precision = S.PREC_MIXED
    opts.schedule = S.SCHED_PERSISTENT
    opts.use_graph = 1
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    tune = {"block": opts.block, "chunk": opts.chunk, "blocks_per_sm": opts.blocks_per_sm,
            "step_min": opts.step_min, "autotuned": False}
    default_opts = None
    if not args.no_autotune:
        default_opts = S.skirt_trace_opts()
        ctypes_copy(default_opts, opts)
        rep = S.skirt_autotune(grid.h, src, tables.c, prob.npk, seed, ins, opts, args.tune_fraction, absorbed,
                               images, sed, stream=stream.cuda_stream, repeats=2)
        ch = rep["points"][rep["chosen"]]
        tune = {"block": opts.block, "chunk": opts.chunk, "blocks_per_sm": opts.blocks_per_sm,
                "step_min": opts.step_min, "autotuned": True, "candidates": rep["n"],
                "sample_packets": rep["sample_packets"], "repeats": rep["repeats"],
                "confirm_packets": rep["confirm_packets"],
                "sample_ms_chosen": ch["ms"], "sample_ms_default": rep["points"][0]["ms"],
                "confirm_ms_chosen": ch["ms_confirm"], "confirm_ms_default": rep["points"][0]["ms_confirm"],
                "chosen_is_default": rep["chosen"] == 0}

    clocks = ClockSampler(local)
    elapsed, kernel_ms, led = run_steps(S, grid, src, tables, prob, seed, ins, opts, outs, args.steps, args.warmup,
                                        flush, stream, barrier, clocks)
    clk = clocks.stop()
    elapsed = job_time(elapsed, dist, "cuda")
    packets = prob.total_packets
    value = job_throughput(packets, world, args.steps, elapsed)
    if default_opts is not None:
        # the default schedule on the same workload, for comparison with the tuned one
        k = min(args.steps, 3)
        e_def, _, _ = run_steps(S, grid, src, tables, prob, seed, ins, default_opts, outs, k, 1, flush, stream,
                                barrier)
        tune["default_value"] = job_throughput(packets, world, k, job_time(e_def, dist, "cuda"))
        tune["default_steps"] = k

    # ---- rooflines of the trace kernel
    octree = args.workload == "octree"
    peak, peak_kind = peaks()
    red_rate, _ = S.skirt_microbench(3, grid.ncell * n)
    k_ms = float(np.mean(kernel_ms))
    key = "octree" if octree else ("disk" if args.workload == "disk" and args.grid == 256 else None)
    roofs = trace_rooflines(led, packets, k_ms, len(prob.instruments), red_rate, peak, peak_kind,
                            "trace_mixed_kernel<true> (octree)" if octree else "trace_mixed_kernel",
                            12 if octree else 4, TRAFFIC_PER_PACKET.get(key) if key else None,
                            clk["sm_mhz"] if clk else None, sm_count if key == "disk" else None)

    # ---- the same at 32-byte sector granularity (context): one sector per
    # crossing's read, and a read plus a write-back sector per FP64 reduction
    tallies = (packets + led["scatterings"]) * len(prob.instruments)
    sector_bytes = 32 * (led["deposit_steps"] + led["locate_steps"] + led["peel_steps"]) + 64 * (
        led["deposit_steps"] + tallies)
    roof_sector = {"bound": "hbm", "achieved": sector_bytes / (k_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                   "frac": sector_bytes / (k_ms / 1e3) / 1e9 / peak, "bytes_per_launch": sector_bytes,
                   "note": "context: 32-byte sector per crossing read, read + write-back sector per reduction; "
                           "L2 reuse lets this exceed the DRAM bytes actually moved"}

    # ---- plain FP64 form on a sample
    fp64 = None
    if args.fp64_packets > 0:
        fp64 = plain_fp64(S, grid, src, tables, prob, seed, ins, outs,
                          min(1.0, args.fp64_packets / max(prob.total_packets, 1)),
                          S.SCHED_PER_LAMBDA if n == 1 else S.SCHED_PERSISTENT, stream, barrier)

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_kr = torch.from_numpy(np.ascontiguousarray(prob.grid.kr, dtype=np.float32).ravel()).pin_memory()
        h_abs = torch.zeros((grid.ncell, n), dtype=torch.float64).pin_memory()
        h_img = torch.zeros(npix, dtype=torch.float64).pin_memory()
        h_sed = torch.zeros((len(prob.instruments), n), dtype=torch.float64).pin_memory()
        ksteps = min(args.steps, 3)

        def e2e_step():
            g2 = S.Grid(prob.grid, kr=h_kr)
            S.skirt_trace(g2.h, src, tables.c, prob.npk, seed, ins, opts, h_abs, h_img, h_sed,
                          stream=stream.cuda_stream)
            g2.close()

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            e2e_step()
        barrier()
        dte = (time.perf_counter() - t0) / ksteps
        h2d = h_kr.numel() * 4
        d2h = (h_abs.numel() + h_img.numel() + h_sed.numel()) * 8
        if octree:
            # grid creation uploads the node array (32 B per node, 1 + 8 (nleaf - 1) / 7 nodes), the
            # leaf table (16 B) and the leaf-to-node map (4 B), and reads kr back once (4 B per leaf)
            nl = prob.grid.ncell
            h2d += 32 * (1 + 8 * (nl - 1) // 7) + 20 * nl
            d2h += 4 * nl
        e2e = {"value": packets * world / dte, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ksteps}
    grid.close()
    del absorbed, images, sed, outs

    # ---- the batched form: the clumpy torus, 200 wavelengths with uneven
    # packet counts, in one persistent graph launch
    batched = None
    if args.workload == "disk" and not args.no_batched:
        batched = run_batched(S, args, seed, opts, flush, stream, barrier, peak, peak_kind, dist, world)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": config_of(args, prob, {"precision": "mixed", "schedule": "persistent + CUDA graph",
                                             "replicas": world, "tuning": tune}),
            **roofs,
            "roofline_sector": roof_sector,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * (1 + len(prob.instruments) + (1 if n > 1 else 0)),
            "clocks": clk,
            "plain_fp64": fp64,
            "speedup_vs_plain_fp64": (value / world / fp64["value"]) if fp64 else None,
            "batched": batched,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def ctypes_copy(dst, src):
    import ctypes
    ctypes.memmove(ctypes.addressof(dst), ctypes.addressof(src), ctypes.sizeof(src))


def run_batched(S, args, seed, opts, flush, stream, barrier, peak, peak_kind, dist, world):
    """The batched form (clumpy torus 256^3, 200 wavelengths, 1e5-2e7 packets
    each, 7.5e8 in all): one warm-up and args.batched_steps timed graph
    launches with the tuned schedule, its rooflines, and the plain FP64 form
    through the same persistent schedule on a sample."""
    import torch
    prob = W_torus(args)
    prob.seed = seed
    grid = S.Grid(prob.grid)
    n = prob.wl.n
    npix = sum(i.npx * i.npx for i in prob.instruments) * n
    outs = (torch.zeros((grid.ncell, n), dtype=torch.float64, device="cuda"),
            torch.zeros(npix, dtype=torch.float64, device="cuda"),
            torch.zeros((len(prob.instruments), n), dtype=torch.float64, device="cuda"))
    tables = S.Tables(prob.wl)
    ins = S.make_instruments(prob.instruments)
    src = S.make_source(prob.source)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    el, kms, led = run_steps(S, grid, src, tables, prob, seed, ins, opts, outs, args.batched_steps, 1, flush, stream,
                             barrier, clocks)
    clk = clocks.stop()
    el = job_time(el, dist, "cuda")
    packets = prob.total_packets
    value = job_throughput(packets, world, args.batched_steps, el)
    red_rate, _ = S.skirt_microbench(3, grid.ncell * n)
    roofs = trace_rooflines(led, packets, float(np.mean(kms)), len(prob.instruments), red_rate, peak, peak_kind,
                            "trace_mixed_kernel", 4, None)
    closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
    fp64 = plain_fp64(S, grid, src, tables, prob, seed, ins, outs, args.batched_fp64_fraction, S.SCHED_PERSISTENT,
                      stream, barrier)
    grid.close()
    del outs
    torch.cuda.empty_cache()
    return {"workload": workload_name(argparse.Namespace(**{**vars(args), "workload": "torus", "packets": 1e8}),
                                      prob),
            "value": value, "unit": UNIT, "steps": args.batched_steps, "warmup": 1,
            "ms_per_step": 1e3 * el / args.batched_steps, "packets_per_step": packets,
            "schedule": "persistent + CUDA graph, the headline's tuned schedule", **roofs,
            "ledger_closure": closure, "clocks": clk, "plain_fp64": fp64,
            "speedup_vs_plain_fp64": value / world / fp64["value"]}


def W_torus(args):
    from paper_1705_04702_gb300 import workloads as W
    return W.torus_problem(n=args.grid, nlambda=200, npx=512)


if __name__ == "__main__":
    main()
