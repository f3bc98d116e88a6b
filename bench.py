#!/usr/bin/env python
"""Throughput benchmark of batched seed extension on GB300.

One step = one xt_extend_batch call over the whole batch: classify and
bucket every pair, order the buckets, and run the persistent extension
kernels; inputs already resident in HBM (c3_mixed: 1.5 GB of inputs, far
larger than the 129 MB L2, so no flush is needed between steps).

Prints one JSON line: GCUPS (useful in-band cells per second, cells counted
by the oracle's definition and returned by the kernels), extensions/s, the
plain one-pair-per-block kernel on the same batch, the end-to-end figure
through the host-buffer API (H2D of inputs and D2H of results inside the
timed region), the roofline of the extension kernels against the integer
ALU pipe's and the issue rate measured on this GPU by instruction probes,
SM clocks sampled during the timed region, and the CPU oracle timed on the
host cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3_mixed]
  python bench.py --impl reference ...   # the CPU oracle on the same workload
N > 1 runs under torchrun: each rank extends its own shard of the workload
(weak scaling; pairs are independent, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import gc
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "seed-extension GCUPS & extensions/s (bit-exact), batched vs plain; p50/p99 latency"
# Fallback only (no measured rate): 152 SMs, 2070 MHz maximum SM clock.
SMS, MAX_MHZ = 152, 2070.0
# Algorithmic instructions of one cell update (one 32-bit cell, or two cells
# in the packed 16-bit form), with the fused DPX forms native on sm_103a:
# on the integer ALU pipe S (byte permute), the anchored diagonal's add-min,
# E and F (add-max with relu each), H (3-way max) and the row key's max: 6;
# on the multiply-add pipe the anchoring multiplier D * 2^k, the row key
# H * 64 + step (H * 65536 + j in 32-bit) and H - alpha (a packed add issues
# there, per the pipe counters of the instruction probes): 3.
ALU_OPS_PER_UPDATE, MAD_OPS_PER_UPDATE = 6, 3
OPS_PER_UPDATE = ALU_OPS_PER_UPDATE + MAD_OPS_PER_UPDATE
# BWA-MEM-compatible cell, 32-bit: S, M (add, select), E and F (M minus the
# opening penalty, then add-max each), H (3-way max), the row key's max: 9 on
# the ALU pipe, and the key's multiply-add on the other: 10
BWA_ALU_OPS_PER_CELL, BWA_OPS_PER_CELL = 9, 10
# instruction probes whose rate is the integer ALU pipe's (the kinds the
# cell update issues there; ncu pipe counters put the packed add on the
# multiply-add pipe instead)
ALU_PROBES = ("max3.s16x2", "addmax.relu.s16x2", "prmt", "max3.s32")
LANE_MAX_QLEN = 510  # one-lane (packed-capable) buckets: qlen + 2 <= 2^9
WORKLOAD_TEXT = {
    "c1_tiny": "1,000 pairs, 100 bp queries, 116 bp targets, 2% sub / 0.2% indel",
    "c2_short": "1,000,000 pairs, qlen U[1,150], tlen = qlen + 200, 1% sub / 0.1% indel, 5% unrelated",
    "c3_mixed": "4,000,000 pairs, read lengths 100/150/250 at 40/40/20%, qlen U[1,read], "
                "tlen = qlen + 200, 1% sub / 0.1% indel, 5% unrelated",
    "c4_long": "250,000 pairs, qlen log-uniform [1000,10000], tlen = qlen + 1000, 8% errors",
    "c5_stream": "10,000,000 pairs, qlen lognormal median 120 sigma 1 clipped [1,2000]",
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["xt", "reference"], default="xt")
    ap.add_argument("--workload", default="c3_mixed")
    ap.add_argument("--pairs", type=int, default=0, help="override the pair count per GPU")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-ascii", action="store_true",
                    help="skip the same batch given as raw ASCII reads")
    ap.add_argument("--no-bwa", action="store_true",
                    help="skip the BWA-MEM-compatible extension leg")
    ap.add_argument("--no-x2", action="store_true",
                    help="skip the equal-length 5,000-pair calls of the paper's kernel comparison")
    ap.add_argument("--no-packed4", action="store_true",
                    help="skip the same batch given as 4-bit codes (device-resident and e2e)")
    ap.add_argument("--no-c4", action="store_true",
                    help="skip the 250,000 long pairs of c4_long (w = 500, z-drop 400)")
    ap.add_argument("--serve-pairs", type=int, default=10_000_000,
                    help="pairs of the c5 stream per offered-load level")
    ap.add_argument("--tune", choices=["auto", "off"], default="auto",
                    help="auto: autotune the workload's length buckets before warm-up")
    ap.add_argument("--streams", type=int, default=0,
                    help="streams the extension kernels of a call fork onto (0: library default)")
    ap.add_argument("--schedule", default="",
                    help="P,R: one forced schedule for every bucket (profiling a kernel on a "
                         "subset of a workload); default: the count-aware plan")
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--serve-batch-pairs", type=int, default=0,
                    help="pairs per batch at most (0: library default)")
    ap.add_argument("--serve-batch-mib", type=int, default=1024,
                    help="staged bytes per batch (the slot capacity), MiB")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0,
                    help="device memory budget of the whole server, GB")
    ap.add_argument("--serve-gather-threads", type=int, default=0, help="0: library default")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[device] if vis else str(device)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", self.index, "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            txt, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            txt, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in txt.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus > 1 and world == 1:
        sys.exit("bench.py: --gpus > 1 runs under torchrun (one rank per GPU)")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce(world, value, op):
    """All-reduce one number across ranks (on the GPU under NCCL, on the host
    under gloo): the timing max and the work sums of the weak-scaling line."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def shard_of(rank: int, world: int, n_per_gpu: int, wl):
    """Weak scaling: the job is the first world * n_per_gpu pairs of the
    workload's counter-based stream, split over the ranks by the library's
    LPT partitioner on estimated cells (xt_shard_lpt; every rank computes the
    same split from the pairs' lengths alone).  Returns this rank's stream
    indices (all of [0, n) on one GPU) and the estimated cells of every part."""
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth
    n_job = world * n_per_gpu
    if world == 1:
        return np.arange(n_per_gpu, dtype=np.int64), None
    q_len, t_len, _ = synth.shapes(wl, n=n_job)
    shard, part_cells = xt.xt_shard_lpt(q_len, t_len, wl.scoring.w, world)
    return np.nonzero(shard == rank)[0].astype(np.int64), part_cells


def batch_of(wl, idx, n_per_gpu):
    """This rank's pairs: the contiguous prefix on one GPU, else by index."""
    from paper_2301_09310_gb300 import synth
    if idx.size == n_per_gpu and (idx.size == 0 or int(idx[-1]) == idx.size - 1):
        return synth.generate(wl, n=n_per_gpu)
    return synth.generate_at(wl, idx)


def aggregate(world, units_local: float, seconds_local: float):
    """Whole-job throughput: units summed over ranks / the slowest rank's time."""
    total = reduce(world, units_local, _sum_op() if world > 1 else None)
    slowest = reduce(world, seconds_local, _max_op() if world > 1 else None)
    return total, slowest, total / slowest


def cell_updates(b, cells, sc):
    """Cell updates the extension DP needs for this batch: cells of pairs that
    the packed 16-bit class takes (score bound B = h0 + match*min(qlen,tlen)
    with (B+1)*2^k and B*64+63 within int16, query within the one-lane
    buckets) count half (two cells per update), the rest one each."""
    m = sc.match
    k = 0
    while (1 << k) < m + 1:
        k += 1
    bound = b.h0.astype(np.int64) + m * np.minimum(b.q_len, b.t_len).astype(np.int64)
    packed = ((bound + 1) << k <= 32767) & (bound * 64 + 63 <= 32767) & (b.q_len <= LANE_MAX_QLEN)
    c = cells.astype(np.float64)
    updates = 0.5 * c[packed].sum() + c[~packed].sum()
    return float(updates), float(c[packed].sum() / max(c.sum(), 1.0))


def measure_int_rates(local):
    """Throughput of each integer instruction kind of the cell update on this
    GPU (xt_int_rate probes, CUDA events), with the SM clock sampled while
    they run: thread-instructions per SM per clock for each kind."""
    import paper_2301_09310_gb300 as xt
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    raw = {}
    for op, name in xt.RATE_NAMES.items():
        s, units, ms = xt.xt_int_rate(local, op, 5)
        if s != xt.XT_OK:
            raise RuntimeError(f"xt_int_rate({name}): {xt.xt_status_str(s)}")
        raw[name] = (units, ms)
    clocks = sampler.stop()
    mhz = clocks["sm_mhz"] if clocks else MAX_MHZ
    sms = _sm_count(local)
    per_clk = {k: u / (ms / 1e3) / sms / (mhz * 1e6) for k, (u, ms) in raw.items()}
    return {"per_sm_per_clock": {k: round(v, 2) for k, v in per_clk.items()},
            "ms": {k: round(ms, 4) for k, (_, ms) in raw.items()},
            "sm_mhz": mhz, "sms": sms, "clocks": clocks,
            "alu_pipe": max(per_clk[k] for k in ALU_PROBES),
            "mad_pipe": per_clk["imad.u32"], "issue": per_clk["max3.s16x2 + add.s16x2 by chain"],
            "cell_update_cells": per_clk["packed cell update (cells)"]}


def _sm_count(local):
    import torch
    return torch.cuda.get_device_properties(local).multi_processor_count


def int_roofline(updates, kernel_ms, rates, mhz, alu_ops=ALU_OPS_PER_UPDATE,
                 all_ops=OPS_PER_UPDATE):
    """Roofline of integer DP kernels against the measured pipe rates at the
    SM clock the kernels ran at: the headline fraction is the algorithmic
    ALU-pipe instructions per second over the ALU pipe's measured rate (the
    pipe that binds the cell update's mix); the issue fraction counts every
    algorithmic instruction against the measured issue rate."""
    sec = kernel_ms / 1e3
    clk = mhz * 1e6 * rates["sms"]
    alu_peak = rates["alu_pipe"] * clk / 1e12
    issue_peak = rates["issue"] * clk / 1e12
    alu_ach = updates * alu_ops / sec / 1e12
    all_ach = updates * all_ops / sec / 1e12
    return {"bound": "alu", "unit": "Tops/s (int-ALU-pipe instructions)",
            "achieved": round(alu_ach, 3), "peak": round(alu_peak, 3),
            "frac": round(alu_ach / alu_peak, 4),
            "peak_basis": (f"measured: ALU-pipe probe {rates['alu_pipe']:.2f} thread-instr/SM/clk "
                           f"x {rates['sms']} SMs x {mhz:.0f} MHz (median SM clock of the timed "
                           "region), of measured"),
            "issue": {"achieved": round(all_ach, 3), "peak": round(issue_peak, 3),
                      "frac": round(all_ach / issue_peak, 4),
                      "basis": f"measured issue probe {rates['issue']:.2f} thread-instr/SM/clk "
                               "(ALU and multiply-add pipes, half the chains each), every algorithmic "
                               "instruction counted, of measured"},
            "cell_update_ceiling": {
                "updates_per_s": round(rates["cell_update_cells"] / 2 * clk, 1),
                "frac": round(updates / sec / (rates["cell_update_cells"] / 2 * clk), 4),
                "basis": "the packed cell update alone on registers (xt_int_rate "
                         "XT_RATE_CELL_P16, 16 cells per step, N-base select included): "
                         "the engine's own arithmetic with no memory, band or row work"}}


# the files that define the extension kernels' device code
KERNEL_SOURCES = ("xt_common.cuh", "xt_engine.cuh", "xt_lane.cuh", "xt_kernels.cuh",
                  "xt_kernels.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2301_09310_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per step of the extension kernels from the committed ncu
    summary, only while the kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_step")


# ------------------------------------------------------------ CPU oracle
def oracle_sample(wl, seconds: float, first: int = 0, single_core: bool = False):
    """Time the CPU oracle on a prefix of the workload sized (from a pilot) to
    about `seconds` of work on all host cores."""
    import oracle
    from paper_2301_09310_gb300 import synth
    sc = oracle.Scoring(*wl.scoring.as_tuple())
    cores = os.cpu_count() or 1
    pilot_n = min(wl.n_pairs, 4000 if wl.name != "c4_long" else 64)
    b = synth.generate(wl, n=pilot_n, first=first)
    t = time.perf_counter()
    oracle.extend_batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0, sc, cores)
    dt = max(time.perf_counter() - t, 1e-3)
    n = int(min(wl.n_pairs, max(pilot_n, pilot_n * seconds / dt)))
    b = synth.generate(wl, n=n, first=first)
    t = time.perf_counter()
    _, cells = oracle.extend_batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0,
                                   sc, cores)
    dt = time.perf_counter() - t
    res = {"value": round(float(cells.sum()) / dt / 1e9, 4), "unit": "GCUPS", "cores": cores,
           "kind": "oracle", "ext_per_s": round(n / dt, 1), "seconds": round(dt, 2),
           "sample": f"first {n} pairs of {wl.name} ({int(cells.sum())} useful cells)"}
    if single_core:
        # the same oracle on one core, on a sample of about a fifth of the time
        n1 = max(1, int(n / cores / 5))
        b1 = b.take(np.arange(n1))
        t = time.perf_counter()
        _, c1 = oracle.extend_batch(b1.q_seq, b1.q_off, b1.q_len, b1.t_seq, b1.t_off, b1.t_len,
                                    b1.h0, sc, 1)
        dt1 = time.perf_counter() - t
        res["single_core"] = {"value": round(float(c1.sum()) / dt1 / 1e9, 4), "unit": "GCUPS",
                              "cores": 1, "seconds": round(dt1, 2),
                              "sample": f"first {n1} pairs of {wl.name}"}
    return res


def run_reference(args):
    from paper_2301_09310_gb300 import synth
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    wl = synth.WORKLOADS[args.workload]
    if args.pairs:
        wl = synth.with_n(wl, args.pairs)
    import oracle
    sc = oracle.Scoring(*wl.scoring.as_tuple())
    cores = os.cpu_count() or 1
    budget = min(10.0, 150.0 / max(1, args.steps + args.warmup))  # whole run within a few minutes
    pilot = oracle_sample(wl, min(2.0, budget))
    n = int(min(wl.n_pairs, max(1000, pilot["ext_per_s"] * budget)))
    b = synth.generate(wl, n=n)
    for _ in range(args.warmup):
        oracle.extend_batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0, sc, cores)
    t = time.perf_counter()
    cells = None
    for _ in range(args.steps):
        _, cells = oracle.extend_batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len,
                                       b.h0, sc, cores)
    dt = (time.perf_counter() - t) / max(1, args.steps)
    value = float(cells.sum()) / dt / 1e9
    sample = f"first {n} pairs of {wl.name} per step ({int(cells.sum())} useful cells)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GCUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{wl.name}: {WORKLOAD_TEXT.get(wl.name, '')}",
                   "pairs_per_step": n, "scoring": wl.scoring.as_tuple()},
        "cpu_baseline": {"value": round(value, 4), "unit": "GCUPS", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ GPU
def run_xt(args):
    import torch
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2301_09310_gb300 import build as xbuild
    xbuild.build()
    wl = synth.WORKLOADS[args.workload]
    n_per_gpu = args.pairs or wl.n_pairs
    idx, part_cells = shard_of(rank, world, n_per_gpu, wl)
    b = batch_of(wl, idx, n_per_gpu)
    n = b.n
    dev = torch.device("cuda", local)
    T = lambda a: torch.from_numpy(a).to(dev)  # noqa: E731
    d = [T(b.q_seq), T(b.q_off), T(b.q_len), T(b.t_seq), T(b.t_off), T(b.t_len), T(b.h0)]
    out = torch.empty((n, 7), dtype=torch.int32, device=dev)
    cells = torch.empty(n, dtype=torch.int64, device=dev)
    ctx = xt.Context(local)
    if args.streams:
        ctx.set_streams(args.streams)
    if args.schedule:
        ctx.set_schedule(*(int(x) for x in args.schedule.split(",")))
    stream = torch.cuda.current_stream(dev)
    tuning = None
    j_max = max(5, int(np.ceil(np.log2(int(b.q_len.max()) + 2))))
    if args.tune == "auto" and not args.schedule:
        # tune the workload's buckets, then keep the tuned table only if it
        # beats the built-in rule on the workload itself (the tuner's trials
        # are synthetic and one bucket at a time)
        t0 = time.perf_counter()
        ctx.autotune(wl.scoring, j_max=j_max)
        tune_s = time.perf_counter() - t0
        sched = {f"j{j}": "P{}R{}".format(*ctx.bucket_schedule(wl.scoring.w, j))
                 for j in range(5, j_max + 1)}
        builtin = xt.Context(local)
        if args.streams:
            builtin.set_streams(args.streams)

        def step_ms(c, reps=3):
            for _ in range(2):
                c.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                c.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
            z.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(z) / reps

        tuned_ms, builtin_ms = step_ms(ctx), step_ms(builtin)
        kept = "tuned table"
        if builtin_ms < tuned_ms:
            ctx.close()
            ctx, kept = builtin, "built-in rule"
        else:
            builtin.close()
        tuning = {"seconds": round(tune_s, 2), "schedule": sched, "kept": kept,
                  "step_ms_tuned": round(tuned_ms, 3), "step_ms_builtin": round(builtin_ms, 3)}

    def step(plain=False):
        ctx.extend(*d, wl.scoring, plain=plain, out=out, cells=cells, stream=stream)

    rates = measure_int_rates(local)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    cells_step = int(cells.sum().item())
    updates_step, packed_frac = cell_updates(b, cells.cpu().numpy(), wl.scoring)
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)  # a clock sample before the timed region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.stats()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.stats()["launches"]
    # the extension kernels' own time, from CUDA events the library records
    # around them on this stream (a short separate pass: timed calls launch
    # directly instead of replaying the captured graph)
    ctx.set_timing(True)
    ctx.stats()
    for _ in range(min(args.steps, 5)):
        step()
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.set_timing(False)
    total_cells, s_max, cells_per_s = aggregate(world, cells_step, ms / 1e3)
    ms_max = s_max * 1e3
    total_pairs = reduce(world, n, _sum_op() if world > 1 else None)
    value = cells_per_s / 1e9
    dp_ms = st["dp_ms"] / max(1, st["timed_calls"])
    run_mhz = clocks["sm_mhz"] if clocks else MAX_MHZ
    roof = int_roofline(updates_step, dp_ms, rates, run_mhz)
    traffic = profiled_traffic(wl.name)
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # packed 16-bit lanes where the score bound allows, 32-bit otherwise
        "dtype": ("int16x2" if packed_frac >= 1.0 else
                  "int32" if packed_frac <= 0.0 else "int16x2+int32"),
        "data": "synthetic",
        "config": {"workload": f"{wl.name}: {WORKLOAD_TEXT.get(wl.name, '')}",
                   "pairs_per_gpu": n, "scoring": wl.scoring.as_tuple(),
                   "useful_cells_per_gpu": cells_step,
                   "l2": f"inputs {b.nbytes() / 1e9:.2f} GB per GPU > 129 MB L2, no flush",
                   "parallelism": (f"dp{world}: the first {world} x {n_per_gpu} pairs split by "
                                   "LPT on estimated cells (xt_shard_lpt), no collective"
                                   if world > 1 else "dp1")},
        "ext_per_s": round(total_pairs / (ms_max / 1e3), 1),
        "gpu_launches": launches,
        "roofline": dict(roof, **{
            "traffic": traffic,
            "kernel": "extension DP launches of one step (k_lane packed/32-bit, k_queue)",
            "kernel_ms_per_step": round(dp_ms, 4),
            "cell_updates_per_step": updates_step,
            "ops_per_update": {"alu_pipe": ALU_OPS_PER_UPDATE, "mad_pipe": MAD_OPS_PER_UPDATE,
                               "note": "one update = one 32-bit cell or two packed 16-bit cells"},
            "packed_cell_fraction": round(packed_frac, 4),
            "cell_update_ceiling_gcups": round(rates["cell_update_cells"] * rates["sms"]
                                               * run_mhz * 1e6 / 1e9, 1),
            "measured_rates": rates}),
        "clocks": clocks,
        "tuning": tuning or "built-in schedule",
    }
    if not args.no_plain:
        step(plain=True)
        torch.cuda.synchronize()
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            step(plain=True)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / reps
        res["plain"] = {"value": round(cells_step / (pms / 1e3) / 1e9, 3), "unit": "GCUPS",
                        "ms_per_step": round(pms, 3),
                        "kernel": "k_plain: one pair per one-warp block, int32"}
        res["speedup_vs_plain"] = round(pms / ms, 3)
    if not args.no_ascii:
        res["ascii_reads"] = ascii_leg(b, wl, args, local, stream, cells_step)
    if not args.no_bwa:
        res["bwa_compatible"] = bwa_leg(b, wl, args, local, stream, rates, run_mhz)
    if not args.no_e2e:
        res["e2e"] = e2e_leg(ctx, b, wl, args, dev, stream, world)
    if not args.no_packed4 and world == 1:
        res["packed4"] = packed4_leg(b, wl, args, local, stream, cells_step)
    if not args.no_x2 and world == 1:
        res["paper_x2"] = x2_leg(local, stream)
    if not args.no_c4 and world == 1 and args.workload != "c4_long":
        res["c4_long"] = c4_leg(args, local, stream, rates, run_mhz)
    if not args.no_serve and world == 1:
        res["serving"] = serve_leg(args, local, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = oracle_sample(wl, args.cpu_seconds, first=0, single_core=True)
    ctx.close()
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ascii_leg(b, wl, args, local, stream, cells_step):
    """The same batch as raw reads (ASCII letters, mixed case, N as 'N'): each
    call first packs both sequence buffers into base codes on the GPU."""
    import torch
    import paper_2301_09310_gb300 as xt

    dev = torch.device("cuda", local)
    letters = np.frombuffer(b"ACGTN", np.uint8)
    d = [torch.from_numpy(a).to(dev) for a in
         (letters[np.minimum(b.q_seq, 4)], b.q_off, b.q_len, letters[np.minimum(b.t_seq, 4)],
          b.t_off, b.t_len, b.h0)]
    ctx = xt.Context(local)
    ctx.set_alphabet(xt.XT_ALPHABET_ASCII)
    out = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
    cells = torch.empty(b.n, dtype=torch.int64, device=dev)
    for _ in range(3):
        ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(reps):
        ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    same = int(cells.sum().item()) == cells_step
    ctx.close()
    return {"value": round(cells_step / (ms / 1e3) / 1e9, 3), "unit": "GCUPS",
            "ms_per_step": round(ms, 4), "same_cells_as_codes": same,
            "input": "ASCII letters; xt_ctx_set_alphabet(XT_ALPHABET_ASCII): an on-GPU packing "
                     "pass per call, then the same extension"}


def bwa_leg(b, wl, args, local, stream, rates, mhz):
    """The same batch under the BWA-MEM-compatible semantics
    (xt_extend_batch_bwa: gaps from the match value, band narrowing from the
    end bonus 5, row trimming; the workload's penalties for both gap kinds).
    Its useful cells differ from the default definition's (trimmed rows)."""
    import torch
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300.synth import BwaScoringParams

    dev = torch.device("cuda", local)
    d = [torch.from_numpy(a).to(dev) for a in
         (b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0)]
    sc = BwaScoringParams.from_scoring(wl.scoring)
    ctx = xt.Context(local)
    out = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
    cells = torch.empty(b.n, dtype=torch.int64, device=dev)
    for _ in range(3):
        ctx.extend_bwa(*d, sc, out=out, cells=cells, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(reps):
        ctx.extend_bwa(*d, sc, out=out, cells=cells, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    n_cells = int(cells.sum().item())
    ctx.close()
    return {"value": round(n_cells / (ms / 1e3) / 1e9, 3), "unit": "GCUPS",
            "ms_per_step": round(ms, 4), "useful_cells": n_cells,
            "ext_per_s": round(b.n / (ms / 1e3), 1),
            "roofline": dict(int_roofline(n_cells, ms, rates, mhz, BWA_ALU_OPS_PER_CELL,
                                          BWA_OPS_PER_CELL),
                             ops_per_cell={"alu_pipe": BWA_ALU_OPS_PER_CELL,
                                           "all": BWA_OPS_PER_CELL},
                             kernel="whole call (classify, order, k_bwa)"),
            "scoring": list(sc.as_tuple()),
            "kernel": "k_bwa: one pair per group of 2..256 lanes, a row's live columns at a time, int32"}


def packed4_leg(b, wl, args, local, stream, cells_step):
    """The same batch as 4-bit codes, two per byte (xt_ctx_set_alphabet
    XT_ALPHABET_PACKED4, the paper's 4-bit packing): device-resident calls
    (each unpacks both buffers on the GPU first), and the host-buffer call,
    which copies the packed bytes (half those of base codes) in chunks and
    unpacks each chunk on the GPU as it arrives."""
    import torch
    import paper_2301_09310_gb300 as xt

    dev = torch.device("cuda", local)
    q4, t4 = xt.pack4(b.q_seq), xt.pack4(b.t_seq)
    d = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
         (q4, b.q_off, b.q_len, t4, b.t_off, b.t_len, b.h0)]
    ctx = xt.Context(local)
    ctx.set_alphabet(xt.XT_ALPHABET_PACKED4)
    out = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
    cells = torch.empty(b.n, dtype=torch.int64, device=dev)
    for _ in range(3):
        ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(reps):
        ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    same = int(cells.sum().item()) == cells_step
    del d, out, cells

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    h = [pinned(a) for a in (q4, b.q_off, b.q_len, t4, b.t_off, b.t_len, b.h0)]
    hout = pinned(np.zeros((b.n, 7), np.int32))
    hcells = pinned(np.zeros(b.n, np.int64))
    for _ in range(max(2, min(args.warmup, 3))):  # untimed: the chunk plans' graphs are captured
        ctx.extend_host(*h, wl.scoring, out=hout, cells=hcells, stream=stream)
    ereps = max(1, min(args.steps, 5))
    t = time.perf_counter()
    for _ in range(ereps):
        ctx.extend_host(*h, wl.scoring, out=hout, cells=hcells, stream=stream)
    dt = (time.perf_counter() - t) / ereps
    ctx.close()
    return {"value": round(cells_step / (ms / 1e3) / 1e9, 3), "unit": "GCUPS",
            "ms_per_step": round(ms, 4), "same_cells_as_codes": same,
            "input": "4-bit codes, two per byte; unpacked on the GPU in each call",
            "e2e": {"value": round(int(hcells.sum()) / dt / 1e9, 3), "unit": "GCUPS",
                    "h2d_bytes_per_step": sum(int(a.nbytes) for a in h),
                    "d2h_bytes_per_step": int(hout.nbytes + hcells.nbytes),
                    "ms_per_step": round(dt * 1e3, 3),
                    "api": "xt_extend_batch_host with XT_ALPHABET_PACKED4 (pinned host buffers)"}}


def c4_leg(args, local, stream, rates, mhz):
    """c4_long at its stated size: 250,000 pairs, query lengths log-uniform in
    [1000, 10000], w = 500, z-drop 400, 32-bit scores (the score bound rules
    out the packed form), the whole batch in one call with the built-in
    count-aware plan; the plain kernel on the same batch beside it."""
    import torch
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth

    wl = synth.WORKLOADS["c4_long"]
    b = synth.generate(wl)
    dev = torch.device("cuda", local)
    d = [torch.from_numpy(a).to(dev) for a in
         (b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0)]
    out = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
    cells = torch.empty(b.n, dtype=torch.int64, device=dev)
    ctx = xt.Context(local)
    for _ in range(2):
        ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    torch.cuda.synchronize()
    n_cells = int(cells.sum().item())
    updates, packed_frac = cell_updates(b, cells.cpu().numpy(), wl.scoring)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.set_timing(True)
    ctx.stats()
    ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.set_timing(False)
    dp_ms = st["dp_ms"] / max(1, st["timed_calls"])
    e0.record(stream)
    ctx.extend(*d, wl.scoring, plain=True, out=out, cells=cells, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1)
    ctx.close()
    return {"value": round(n_cells / (ms / 1e3) / 1e9, 3), "unit": "GCUPS",
            "ms_per_step": round(ms, 3), "ext_per_s": round(b.n / (ms / 1e3), 1),
            "useful_cells": n_cells, "pairs": b.n, "scoring": wl.scoring.as_tuple(),
            "dtype": "int32" if packed_frac <= 0.0 else "int16x2+int32",
            "workload": f"c4_long: {WORKLOAD_TEXT['c4_long']}",
            "plain": {"value": round(n_cells / (pms / 1e3) / 1e9, 3), "unit": "GCUPS",
                      "ms_per_step": round(pms, 3)},
            "roofline": dict(int_roofline(updates, dp_ms, rates, mhz),
                             kernel_ms_per_step=round(dp_ms, 3))}


def e2e_leg(ctx, b, wl, args, dev, stream, world):
    """Same metric through xt_extend_batch_host: pinned host inputs copied in,
    results (and cells) copied out, inside the timed region of every step."""
    import torch

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    h = [pinned(a) for a in (b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0)]
    n = b.n
    out = pinned(np.zeros((n, 7), np.int32))
    cells = pinned(np.zeros(n, np.int64))
    # untimed warm-up: a call's CUDA graphs (one per chunk plan) are captured
    # on the second call with that plan
    for _ in range(max(2, min(args.warmup, 3))):
        ctx.extend_host(*h, wl.scoring, out=out, cells=cells, stream=stream)
    reps = max(1, min(args.steps, 5))
    barrier(world)
    t = time.perf_counter()
    for _ in range(reps):
        ctx.extend_host(*h, wl.scoring, out=out, cells=cells, stream=stream)
    dt = (time.perf_counter() - t) / reps
    dt = reduce(world, dt, _max_op())
    total_cells = reduce(world, int(cells.sum()), _sum_op())
    h2d = sum(int(a.nbytes) for a in h)
    d2h = int(out.nbytes + cells.nbytes)
    return {"value": round(total_cells / dt / 1e9, 3), "unit": "GCUPS",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": round(dt * 1e3, 3), "api": "xt_extend_batch_host (pinned host buffers)"}


# The paper's only absolute kernel times for this comparison: 64 bp, 5,000 pairs
# per call (Sec. V-B): SALoBa 0.51 ms on a GTX 1650 and 0.24 ms on an RTX 3090.
PAPER_X2_MS = {64: {"GTX1650": 0.51, "RTX3090": 0.24}}
X2_CANDIDATES = ((0, 0), (1, 8), (1, 16), (4, 8), (8, 8), (16, 8), (16, 4), (32, 8), (32, 4))


def x2_leg(local, stream):
    """Equal-length reads of the paper's kernel comparison (Sec. V-B): one
    call of 5,000 pairs per length, unbanded (w = L), z-drop off.  These calls
    are small and latency-bound, so each length times every schedule its
    bucket can take on the batch itself and keeps the fastest (all of them
    must give identical results); CUDA events around whole calls, averaged."""
    import torch
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth

    dev = torch.device("cuda", local)
    rows = []
    for L in synth.X2_LENGTHS:
        wl = synth.x2_workload(L)
        b = synth.generate(wl)
        d = [torch.from_numpy(a).to(dev) for a in
             (b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0)]
        out = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
        cells = torch.empty(b.n, dtype=torch.int64, device=dev)
        j = int(np.ceil(np.log2(L + 2)))
        reps = 20 if L <= 512 else 4
        best, first, agree = None, None, True
        for P, R in X2_CANDIDATES:
            ctx = xt.Context(local)
            try:
                if P:
                    ctx.set_bucket_schedule(wl.scoring.w, j, P, R)
            except xt.XtError:
                ctx.close()
                continue
            for _ in range(3):
                ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
            torch.cuda.synchronize()
            got = (out.cpu().numpy(), cells.cpu().numpy())
            if first is None:
                first = got
            elif not (np.array_equal(first[0], got[0]) and np.array_equal(first[1], got[1])):
                agree = False
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ctx.extend(*d, wl.scoring, out=out, cells=cells, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ctx.close()
            if best is None or ms < best[0]:
                best = (ms, P, R)
        useful = int(first[1].sum())
        row = {"L": L, "pairs": b.n, "ms_per_call": round(best[0], 4),
               "schedule": "built-in" if best[1] == 0 else f"P{best[1]}R{best[2]}",
               "gcups": round(useful / (best[0] / 1e3) / 1e9, 2),
               "table_gcups": round(b.n * L * L / (best[0] / 1e3) / 1e9, 2),
               "schedules_agree": agree}
        if L in PAPER_X2_MS:
            row["paper_ms"] = PAPER_X2_MS[L]
        rows.append(row)
    return {"workload": "5,000 pairs per call, qlen = tlen = L, wgsim-like 2% substitutions and "
                        "0.1% indels, w = L (whole table), z-drop off",
            "timing": "CUDA events around whole xt_extend_batch calls, inputs resident",
            "note": "paper times are other GPUs and full local (restarting) tables: context only",
            "lengths": rows}


def serve_leg(args, local, stream):
    """The c5 served stream through the serving loop (xt_serve_*): requests of
    U[1,4096] host pairs arriving as a Poisson process at 25/50/90% of the
    batched path's peak pairs/s on the same mix.  Latency of a request is from
    its scheduled arrival to its results in host memory (xt_serve_times
    stamps, CLOCK_MONOTONIC, the clock of time.monotonic_ns)."""
    import torch
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth

    wl = synth.WORKLOADS["c5_stream"]
    b = synth.generate(wl, n=args.serve_pairs)
    dev = torch.device("cuda", local)
    # schedules tuned for this mix, for large and for small calls; every slot
    # context of the server loads the table
    import tempfile
    table = os.path.join(tempfile.mkdtemp(prefix="xt_tune_"), "tuning.json")
    j_max = max(5, int(np.ceil(np.log2(int(b.q_len.max()) + 2))))
    ctx = xt.Context(local)
    t0 = time.perf_counter()
    ctx.autotune(wl.scoring, j_max=j_max, table_path=table)
    tune_s = time.perf_counter() - t0
    sched = {f"j{j}": "P{}R{}/P{}R{}".format(*ctx.bucket_schedule(wl.scoring.w, j, xt.XT_BATCH_LARGE),
                                            *ctx.bucket_schedule(wl.scoring.w, j, xt.XT_BATCH_SMALL))
             for j in range(5, j_max + 1)}
    # peak of the batched path on this mix: device-resident, one call per step
    d = [torch.from_numpy(a).to(dev) for a in
         (b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0)]
    out_d = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
    cells_d = torch.empty(b.n, dtype=torch.int64, device=dev)
    for _ in range(3):
        ctx.extend(*d, wl.scoring, out=out_d, cells=cells_d, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        ctx.extend(*d, wl.scoring, out=out_d, cells=cells_d, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    peak_ms = e0.elapsed_time(e1) / reps
    peak_pairs = b.n / (peak_ms / 1e3)
    ref_out, ref_cells = out_d.cpu().numpy(), cells_d.cpu().numpy()
    total_cells = int(ref_cells.sum())
    ctx.close()
    del d, out_d, cells_d
    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(2e-4)
    builtin = serve_levels(args, local, b, wl, peak_pairs, ref_out, ref_cells, total_cells, None)
    tuned = serve_levels(args, local, b, wl, peak_pairs, ref_out, ref_cells, total_cells, table)
    sys.setswitchinterval(old_switch)
    return {"workload": f"c5_stream: {args.serve_pairs:,} pairs, qlen lognormal median 120 "
                        "sigma 1 clipped [1,2000], tlen = qlen + 200; requests U[1,4096] "
                        "pairs, Poisson arrivals",
            "api": f"xt_serve_submit/xt_serve_wait (host buffers; {args.serve_slots} slots of "
                   f"{args.serve_batch_mib} MiB and "
                   f"{args.serve_batch_pairs or 'the default'} pairs at most, "
                   f"device budget {args.serve_budget_gb:g} GB, "
                   f"gather threads {args.serve_gather_threads or 'default'})",
            "latency": "scheduled arrival -> results in host memory",
            "schedules": "levels: built-in count-aware schedules (the server's default); "
                         "levels_with_tuning_table: the slots load the table tuned below",
            "tuning": {"seconds": round(tune_s, 2), "schedule_large/small": sched},
            "peak_batched_pairs_per_s": round(peak_pairs, 1),
            "peak_batched_gcups": round(total_cells / (peak_ms / 1e3) / 1e9, 3),
            "levels": builtin, "levels_with_tuning_table": tuned}


def serve_levels(args, local, b, wl, peak_pairs, ref_out, ref_cells, total_cells, table):
    """Run the request stream at 25/50/90% of peak_pairs through a server."""
    import ctypes
    import queue
    import threading

    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth

    lib = xt.load_library()
    sc = xt._scoring(wl.scoring)
    levels = []
    for frac in (0.25, 0.5, 0.9):
        rs = synth.request_stream(b, frac * peak_pairs, seed=5)
        nreq = int(rs.size.size)
        out = np.zeros((b.n, 7), np.int32)
        cells = np.zeros(b.n, np.int64)
        calls = []
        for r in range(nreq):
            q_seq, q_off, q_len, t_seq, t_off, t_len, h0 = rs.request(r)
            a = int(rs.start[r])
            calls.append((ctypes.c_void_p(q_seq.ctypes.data), q_seq.size,
                          ctypes.c_void_p(q_off.ctypes.data), ctypes.c_void_p(q_len.ctypes.data),
                          ctypes.c_void_p(t_seq.ctypes.data), t_seq.size,
                          ctypes.c_void_p(t_off.ctypes.data), ctypes.c_void_p(t_len.ctypes.data),
                          ctypes.c_void_p(h0.ctypes.data), int(rs.size[r]), ctypes.byref(sc),
                          ctypes.c_void_p(out.ctypes.data + 28 * a),
                          ctypes.c_void_p(cells.ctypes.data + 8 * a)))
        srv = xt.xt_serve_create(local, xt.xt_serve_config(
            args.serve_slots, args.serve_batch_pairs, args.serve_batch_mib << 20, 0,
            int(args.serve_budget_gb * 1e9),
            args.serve_gather_threads, table.encode() if table else None, 0))
        # untimed warm-up: the stream's first requests (whose results the timed
        # stream writes again), 2 ms apart so that each slot runs a batch before
        # the clock starts
        warm = []
        for r in range(min(args.serve_slots, nreq)):
            wtk = ctypes.c_uint64(0)
            ws = lib.xt_serve_submit(ctypes.c_void_p(srv), *calls[r], ctypes.byref(wtk))
            if ws != xt.XT_OK:
                raise RuntimeError(f"xt_serve_submit (warm-up): {xt.xt_status_str(ws)}")
            warm.append(wtk.value)
            time.sleep(0.002)
        for tk_w in warm:
            ws, _ = xt.xt_serve_wait(srv, tk_w, -1)
            if ws != xt.XT_OK:
                raise RuntimeError(f"xt_serve_wait (warm-up): {xt.xt_status_str(ws)}")
        tickets = queue.Queue()
        stamps = np.zeros((nreq, 4), np.int64)   # arrival, submit, launch, done
        bpairs = np.zeros(nreq, np.int64)
        status = []

        def waiter():
            for r in range(nreq):
                tk = tickets.get()
                s, tm = xt.xt_serve_wait(srv, tk, -1)
                if s != xt.XT_OK:
                    status.append(s)
                stamps[r, 1:] = (tm.submit_ns, tm.launch_ns, tm.done_ns)
                bpairs[r] = tm.batch_pairs

        th = threading.Thread(target=waiter)
        # no garbage-collection pauses in the load generator: a late submit
        # counts as latency (from the scheduled arrival)
        gc_on = gc.isenabled()
        gc.disable()
        th.start()
        t0 = time.monotonic_ns() + 5_000_000
        arrive = t0 + (rs.arrival_s * 1e9).astype(np.int64)
        stamps[:, 0] = arrive
        busy = 0
        tk = ctypes.c_uint64(0)
        submit = lib.xt_serve_submit
        for r in range(nreq):
            while True:
                left = int(arrive[r]) - time.monotonic_ns()
                if left <= 0:
                    break
                if left > 300_000:
                    time.sleep((left - 200_000) / 1e9)
            backoff = 50e-6
            while True:
                s = submit(ctypes.c_void_p(srv), *calls[r], ctypes.byref(tk))
                if s != xt.XT_EBUSY:
                    break
                busy += 1
                # the queue drains as batches form: leave the host cores to
                # the server's gather threads meanwhile
                time.sleep(backoff)
                backoff = min(2 * backoff, 1e-3)
            if s != xt.XT_OK:
                raise RuntimeError(f"xt_serve_submit: {xt.xt_status_str(s)}")
            tickets.put(tk.value)
        th.join()
        if gc_on:
            gc.enable()
        st = xt.xt_serve_get_stats(srv)
        xt.xt_serve_destroy(srv)
        if status:
            raise RuntimeError(f"served requests failed: {set(status)}")
        lat = (stamps[:, 3] - stamps[:, 0]) / 1e6
        span = (stamps[:, 3].max() - t0) / 1e9
        # steady state: the pairs whose results landed in the last three
        # quarters of the arrival window, per second of that window (a server
        # that keeps up completes pairs as fast as they arrive; the drain after
        # the last arrival, one batch latency, is left out)
        t_arr = int(arrive.max())
        w0 = t0 + (t_arr - t0) // 4
        done_in = (stamps[:, 3] >= w0) & (stamps[:, 3] <= t_arr)
        steady = float(rs.size[done_in].sum()) / ((t_arr - w0) / 1e9)
        half = stamps[:, 0] < t0 + (t_arr - t0) // 2
        levels.append({
            "offered_frac_of_peak": frac,
            "offered_pairs_per_s": round(frac * peak_pairs, 1),
            "achieved_pairs_per_s": round(b.n / span, 1),
            "steady_pairs_per_s": round(steady, 1),
            "arrival_ms": round((t_arr - t0) / 1e6, 3),
            "drain_ms": round((stamps[:, 3].max() - t_arr) / 1e6, 3),
            "p99_ms_first_half": round(float(np.percentile(lat[half], 99)), 3),
            "p99_ms_second_half": round(float(np.percentile(lat[~half], 99)), 3),
            "gcups": round(total_cells / span / 1e9, 3),
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "queue_p99_ms": round(float(np.percentile((stamps[:, 2] - stamps[:, 1]) / 1e6, 99)), 3),
            "submit_lag_p99_ms": round(float(np.percentile((stamps[:, 1] - stamps[:, 0]) / 1e6,
                                                           99)), 3),
            "mean_batch_pairs": round(float(np.mean(bpairs)), 1),
            "batches": st.batches,
            "gather_ms_per_batch": round(st.gather_ns / 1e6 / max(1, st.batches), 3),
            "device_ms_per_batch": round(st.device_ns / 1e6 / max(1, st.batches), 3),
            "requests": nreq, "busy_retries": busy,
            "equal_to_batched": bool(np.array_equal(out, ref_out)
                                     and np.array_equal(cells, ref_cells)),
        })
    return levels


def _max_op():
    import torch.distributed as dist
    return dist.ReduceOp.MAX


def _sum_op():
    import torch.distributed as dist
    return dist.ReduceOp.SUM


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_xt(args)


if __name__ == "__main__":
    main()
