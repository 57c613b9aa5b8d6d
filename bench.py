#!/usr/bin/env python3
"""Benchmark: spin updates/ns of the batched bit-sliced checkerboard sweep.

Workload (one GPU): 3D Edwards-Anderson +-J glass, L = 64 periodic, 256
disorder samples x 2 real replicas packed 64 samples per uint64 word, heat
bath at T = 1.0, energy and replica overlap measured every 10 sweeps.  One
step is a block of 100 sweeps with its 10 measurements; the default 100
steps are the workload's full 10^4 sweeps.  Inputs are synthetic and seeded
(couplings and initial spins drawn on the device from the counter-based
stream).

Printed JSON line (rank 0): value = spin updates/ns of the device-resident
run; e2e = the same through the C ABI with the state uploaded from pinned
host memory and the measurement series read back every step; plain = the
one-byte-per-spin kernel on the same workload, with its roofline; roofline =
the dominant sweep kernel against the integer-issue peak (lop3-class logic
and 64-bit products share one issue slot, measured by the integer probe);
cpu_baseline = the CPU oracle on a bounded sample of the same workload;
serving = the 2000-job serving mix at 0.8 x its calibrated capacity (p50 /
p99 job latency, aggregate updates/ns); other_workloads = the other
configurations and the paper's other models, each with its roofline.

``--impl reference`` times the CPU oracle instead (the only reference this
method has: the paper ships no code).
"""

from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin updates/ns (3D EA ±J, batched vs plain, bit-exact); p50/p99 job latency"
UNIT = "spin updates/ns"
L, S, R = 64, 256, 2
T = 1.0
SWEEPS_PER_STEP = 100
MEASURE_EVERY = 10
SEED = 0x0704357300000001
WORKLOAD = ("3D EA +-J, L=64 periodic, 256 samples x 2 replicas (64 samples per uint64), heat bath T=1.0, "
            "E and Q every 10 sweeps; step = 100 sweeps")
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the dominant
# kernel from one ncu capture of it on this workload, per (kernel variant,
# words per block), valid while the kernel source is unchanged (hash of the
# sources it is compiled from).
TRAFFIC_BYTES_PER_LAUNCH = {(24, 0): 41977600}
TRAFFIC_SOURCE_HASH = "0b06d535be286e49"
# Memory traffic of one colour launch of the q=4 Potts sweep (k_sweep_potts)
# on its L=32, 128 x 2 workload, from one ncu capture, valid while its
# sources are unchanged: global loads through L1 (spin words, couplings and
# the 16-byte table row of every update), L2 and DRAM bytes, L1 hit rate.
POTTS_TRAFFIC = {"l1_global_load_bytes": 179127744, "l2_bytes": 73770400, "dram_bytes": 21049344,
                 "l1_hit_rate_pct": 78.5}
POTTS_SOURCE_HASH = "ab9e8badae2a5729"
# DRAM traffic of one colour launch of the plain-layout sweep
# (k_sweep_i8_sliced) on the bench workload, from one ncu capture, valid
# while its sources are unchanged.
PLAIN_TRAFFIC = {"dram_read_bytes": 337867008, "dram_write_bytes": 94819584}
PLAIN_SOURCE_HASH = "69d32de33006c0d7"
# The kernel variant and launch shape the bench runs by default: the
# lane-queue kernel in its one-wave launch (the automatic choice for one
# temperature), fixed so that the profile above describes the timed kernel.
DEFAULT_VARIANT = (24, 0)


def kernel_source_hash(names=("common.cuh", "jit_sweep_lt.cuh", "jit.cu")) -> str:
    import hashlib

    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_0704_3573_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def config_dict(ws: int) -> dict:
    return {"workload": WORKLOAD, "L": L, "samples_per_gpu": S, "replicas": R, "T": T,
            "sweeps_per_step": SWEEPS_PER_STEP, "measure_every": MEASURE_EVERY,
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"dp{ws}: independent sample batches per GPU, no collective"}


def expected_plane_pairs(lanes: int = 64) -> float:
    """E[plane pairs a 64-lane word needs]: a lane is undecided after k planes
    with probability 2^-k exactly (uniform r), the word while any lane is."""
    return sum(1.0 - (1.0 - 4.0 ** (-m)) ** lanes for m in range(16))


def algorithmic_ops_per_word_hb3d(R_: int = 2) -> dict:
    """Least 32-bit integer operations one 3D heat-bath update of a 64-lane
    site word needs (64-bit logic counts as two 32-bit operations), counted
    on the resource they share: three-input logic (lop3) and 64-bit products
    (mad.wide) issue from one slot on GB300 -- the probe's independent
    lop3 / mad.wide chains run no faster together than either alone.
      per word: 6 unsatisfied-bond words (12) and the 6 -> 3 adder tree (16)
        of lop3; the flip as one lop3 per half (2);
      per plane pair (times the expected pairs a word needs): Philox4x32-10
        rounds 2..9, 8 x (2 mad.wide + 2 lop3) = 32; rounds 0 and 1 leave
        each counter word a site part XOR a part shared by every site of the
        block, 2 lop3 to combine them; the two planes, 3 lop3 per half each
        (12);
      once per word: plane 0 with every lane undecided takes 2 lop3 per half
        instead of 3 (-2);
      per site, shared by its R words: the site part of rounds 0 and 1
        (2 mad.wide + 1 lop3).
    Loads and stores (7 spin + 6/R coupling words, 1 store) issue elsewhere
    and are listed apart.  ALU-only count of the earlier definition (Philox
    rounds 0 and 1 not shared, 2-lop3 merges): the "alu_previous" entry."""
    e_p = expected_plane_pairs()
    lop3 = 12 + 16 + 2 + e_p * (16 + 2 + 12) - 2 + 1.0 / R_
    mad_wide = e_p * 16 + 2.0 / R_
    alu_previous = (12 + 16 + 4 + 2) + e_p * (2 * (2 + 4) + 21 + 2)
    lsu = 7 + 6.0 / R_ + 1
    return {"issue": lop3 + mad_wide, "lop3": lop3, "mad_wide": mad_wide, "lsu": lsu, "alu_previous": alu_previous}


# ---------------- distributed helpers ----------------

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------- clocks ----------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ianus_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------- CPU oracle ----------------

def oracle_rate(nthreads: int, sweeps: int, seed: int = SEED):
    """The oracle as it stands on nthreads samples (2 replicas each) of the
    workload; returns (updates/ns, wall seconds, updates)."""
    import oracle

    ids = list(range(nthreads))
    o = oracle.Oracle(dim=3, L=L, sample_ids=ids, n_replicas=R, seed=seed)
    t0 = time.perf_counter()
    o.sweep(oracle.HEATBATH, 1.0 / T, sweeps, measure_every=MEASURE_EVERY, nthreads=nthreads)
    dt = time.perf_counter() - t0
    upd = nthreads * R * L ** 3 * sweeps
    return upd / (dt * 1e9), dt, upd


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    nthr = max(1, min(cores, 16))
    ids = list(range(nthr))
    o = oracle.Oracle(dim=3, L=L, sample_ids=ids, n_replicas=R, seed=SEED)
    for _ in range(args.warmup):
        o.sweep(oracle.HEATBATH, 1.0 / T, 1, nthreads=nthr)
    # one step: MEASURE_EVERY sweeps ending in one E/Q measurement, as the workload measures
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.sweep(oracle.HEATBATH, 1.0 / T, MEASURE_EVERY, measure_every=MEASURE_EVERY, nthreads=nthr)
        times.append(time.perf_counter() - t0)
    upd_step = nthr * R * L ** 3 * MEASURE_EVERY
    total = sum(times)
    value = upd_step * args.steps / (total * 1e9)
    sample = (f"{nthr} samples x {R} replicas of the L=64 workload, {MEASURE_EVERY} sweeps + one E/Q "
              f"measurement per step (the workload's cadence); {cores} host cores")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i8", "data": "synthetic",
        "config": config_dict(ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "nproc": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------- GPU arm ----------------

def run_gpu(args, ws, rank, local):
    import torch

    import paper_0704_3573_gb300 as ianus

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    seed = SEED + 0x100000 * rank  # each rank: its own independent batch of samples
    beta = 1.0 / T
    upd_step = S * R * L ** 3 * SWEEPS_PER_STEP
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    lat = ianus.Lattice(dim=3, L=L, n_samples=S, n_replicas=R, seed=seed, layout="bits64",
                        series_capacity=4096, stream=stream)
    tuned = None
    if not args.tune:  # a fixed kernel variant and launch shape
        v, bw = (args.variant, args.block_words) if args.variant is not None else DEFAULT_VARIANT
        lat.set_variant(v)
        lat.set_block_words(bw)
        tuned = {"variant": v, "block_words": bw, "us_per_sweep": None, "source": "fixed"}
    else:  # kernel variant and launch shape by the autotuner (restores the state)
        from paper_0704_3573_gb300 import tune

        t = tune.tune(lat, ianus.HEATBATH, beta, sweeps=40, use_cache=False)
        tuned = {"variant": t["variant"], "block_words": t["block_words"], "us_per_sweep": t["us_per_sweep"]}
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            lat.sweep(ianus.HEATBATH, beta, SWEEPS_PER_STEP, MEASURE_EVERY)
    torch.cuda.synchronize()
    lat.series(clear=True)

    # ---- device-resident timed region ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)  # evict the 40 MiB working set from L2
            ev[k][0].record(stream)
            lat.sweep(ianus.HEATBATH, beta, SWEEPS_PER_STEP, MEASURE_EVERY)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    dev_s = max_over_ranks(dev_s, ws)
    value = ws * upd_step * args.steps / (dev_s * 1e9)
    lat.synchronize()
    n_rows = len(lat.series()[0])

    # ---- dominant kernel: colour half-sweeps alone, timed on the same stream ----
    nsw = 200
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.fill_(1)
        a0.record(stream)
        lat.sweep(ianus.HEATBATH, beta, nsw, 0)
        a1.record(stream)
    torch.cuda.synchronize()
    kern_s = a0.elapsed_time(a1) / 1e3 / (2 * nsw)
    words_per_launch = (S // 64) * R * L ** 3 // 2
    ops = algorithmic_ops_per_word_hb3d(R)
    achieved = ops["issue"] * words_per_launch / kern_s / 1e12  # T lop3 + mad.wide ops/s
    probe = probe_peak()
    peak = _issue_peak()
    peak_alu = _alu_peak()
    vkey = (tuned["variant"], tuned["block_words"]) if tuned else None
    traffic = TRAFFIC_BYTES_PER_LAUNCH.get(vkey) if kernel_source_hash() == TRAFFIC_SOURCE_HASH else None
    ach_prev = ops["alu_previous"] * words_per_launch / kern_s / 1e12
    roofline = {
        "bound": "alu", "kernel": "ianus_jit_sweep_lt (3D heat bath, R=2, lane-queue kernel, tables as lop3 "
                                  "immediates)",
        "achieved": achieved, "peak": peak, "unit": "T int32 ops/s (lop3 + mad.wide, one shared issue slot)",
        "frac": (achieved / peak) if peak else None, "traffic": traffic,
        "ops_per_word": ops, "words_per_launch": words_per_launch, "launch_us": kern_s * 1e6, "variant": tuned,
        "peak_source": ("probe: independent lop3.b32 and mad.wide.u32 chains side by side, ops/clk/SM x 152 SMs "
                        "x 2070 MHz (of measured)") if peak else None,
        "previous_definition": {"alu_ops_per_word": ops["alu_previous"], "achieved": ach_prev, "peak": peak_alu,
                                "frac": (ach_prev / peak_alu) if peak_alu else None,
                                "what": "ALU-pipe share only, against lop3 alone"},
        "probe": probe,
    }

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = run_e2e(ianus, lat, stream, args, ws)

    # ---- plain one-byte-per-spin kernel on the same workload ----
    plain = None
    if args.plain_steps > 0:
        del lat
        torch.cuda.empty_cache()
        pl = ianus.Lattice(dim=3, L=L, n_samples=S, n_replicas=R, seed=seed, layout="i8", stream=stream)
        with torch.cuda.stream(stream):
            pl.sweep(ianus.HEATBATH, beta, 2, 0)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nps = args.plain_steps * MEASURE_EVERY
        with torch.cuda.stream(stream):
            flush.fill_(2)
            p0.record(stream)
            pl.sweep(ianus.HEATBATH, beta, nps, MEASURE_EVERY)
            p1.record(stream)
        torch.cuda.synchronize()
        ps = p0.elapsed_time(p1) / 1e3
        pv = S * R * L ** 3 * nps / (ps * 1e9)
        # roofline of the plain form: the smaller of two bounds.  HBM: per
        # update the site's byte read and written and its share of the other
        # colour's bytes (3 B) and the 6 coupling bytes each configuration
        # streams (9 B, the couplings larger than L2).  Issue: the kernel
        # updates 64-lane words built in shared memory, so per update the
        # per-lane-plane word update of the bit-sliced form / 64 (e-words 12,
        # adder tree 16, "always" and undecided masks 16, per plane the
        # threshold multiplexers 6 + compare 4, per pair Philox 21 + merge 2,
        # 3.92 pairs; 20 mad.wide per Philox block) plus the layout's own
        # work: the sign packing (9 ops per 32 bytes and lane) and the 32 x 32
        # bit transposes (5 ops per stage, 5 stages) of the bytes read and
        # written, about 13.5 B per update
        hbm = MEASURED.get("hbm_gbs")
        b_upd = 9.0
        npp = expected_plane_pairs()
        ops_upd = (44 + npp * (2 * 10 + 23) + npp * 20) / 64 + 13.5 * (9 + 25) / 32
        pk = _issue_peak()
        bounds = {"hbm": hbm / b_upd if hbm else None, "alu": pk * 1e3 / ops_upd if pk else None}
        binding = min((v, k) for k, v in bounds.items() if v)[1] if any(bounds.values()) else None
        traffic = None
        if kernel_source_hash(("common.cuh", "sweep_planes.cuh", "k_plain.cu")) == PLAIN_SOURCE_HASH:
            upd_pass = S * R * L ** 3 // 2
            traffic = {"dram_bytes_per_update": (PLAIN_TRAFFIC["dram_read_bytes"] + PLAIN_TRAFFIC["dram_write_bytes"])
                       / upd_pass, **PLAIN_TRAFFIC,
                       "what": "ncu, one colour launch; below the 9 B algorithmic figure because one block sweeps "
                               "both replicas of a tile and reads their shared couplings once"}
        plain = {"value": pv, "unit": UNIT, "layout": "i8 (one byte per spin)", "sweeps": nps,
                 "kernel": "k_sweep_i8_sliced (tiles of the 64-sample group, both replicas, turned into 64-lane "
                           "words in shared memory by warp bit transposes, updated bit-sliced, written back as bytes)",
                 "speedup_bitsliced_over_plain": value / ws / pv,
                 "roofline": {"bound": binding, "bytes_per_update": b_upd, "ops_per_update": ops_upd,
                              "bound_updates_per_ns": bounds,
                              "frac": pv / bounds[binding] if binding else None,
                              "traffic": traffic,
                              "peaks": {"hbm_gbs": hbm, "issue_tops": pk}}}
        del pl

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        nproc = os.cpu_count() or 1
        nthr = max(1, min(nproc, 16))
        rate, dt, upd = oracle_rate(nthr, args.cpu_sweeps)
        cpu = {"value": rate, "unit": UNIT, "cores": nthr, "nproc": nproc, "kind": "oracle",
               "sample": f"samples 0..{nthr - 1} x {R} replicas, {args.cpu_sweeps} sweeps of the L=64 workload with "
                         f"E/Q every {MEASURE_EVERY} ({upd} updates, {dt:.1f} s wall)"}

    serving = run_serving(args) if (rank == 0 and args.serve_jobs > 0) else None
    others = run_other_configs(args) if (rank == 0 and not args.no_others) else None

    launches = args.steps * (2 * SWEEPS_PER_STEP + 2 * (SWEEPS_PER_STEP // MEASURE_EVERY))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": config_dict(ws),
        "wall_s": wall, "series_rows": n_rows, "gpu_launches": launches, "clocks": clk, "roofline": roofline,
        "e2e": e2e, "plain": plain, "cpu_baseline": cpu, "serving": serving, "other_workloads": others,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_other_configs(args):
    """Device throughput of the other workloads (parity-test cases, not the
    headline): L=16 single sample Metropolis T=1.1 with E/M every sweep
    (plain layout, shared-memory-resident); L=32 parallel tempering, 32
    temperatures in [0.7, 1.6], 64 samples x 2 replicas, Metropolis, swap every
    10 sweeps; q=4 Potts glass L=32, 128 samples x 2 replicas, heat bath
    T=0.8, E and Q every 10 sweeps."""
    import torch

    import paper_0704_3573_gb300 as ianus

    out = {}
    stream = torch.cuda.Stream()

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # L=16, one sample, 1000 sweeps, E and M every sweep
    lat = ianus.Lattice(dim=3, L=16, n_samples=1, seed=SEED - 1, layout="i8", series_capacity=1000, stream=stream)
    lat.sweep(ianus.METROPOLIS, 1 / 1.1, 10, 1)
    sec = timed(lambda: lat.sweep(ianus.METROPOLIS, 1 / 1.1, 1000, 1), 1)
    # latency floor of a sweep: two passes, each a cluster barrier round trip
    # (0.19 us, measured with a barrier probe on GB300) and one dependent
    # update of a site (about 410 cycles at 2070 MHz, read with clock64)
    floor_us = 2 * (0.19 + 410 / 2070.0)
    sweep_us = sec * 1e3
    # integer work per update (one lane of the plane stream, plain layout):
    # the local field 2 per bond (12), E[pairs] = 1 + 1/4 + 1/16 + ... = 4/3
    # Philox blocks of 16 lop3-class + 16 mad.wide (rounds 2..9) + 2 + 3 for
    # rounds 0..1, the compare 3 per plane (8/3 planes), flip and write-back 2
    rate16 = 16 ** 3 * 1000 / (sec * 1e9)
    alu_u, madw_u = 12 + (4 / 3) * (16 + 2 + 1) + 3 * 8 / 3 + 2, (4 / 3) * (16 + 2)
    ach = rate16 * (alu_u + madw_u) / 1e3
    pk = _issue_peak()
    sms_used = 16
    out["L16_single_sample_metropolis"] = {"updates_per_ns": rate16, "ms_per_1000_sweeps": sec * 1e3,
                                           "sweep_us": sweep_us,
                                           "mode": "plain int8, one lattice split over a 16-block cluster "
                                                   "(one z-plane per block, halos in shared memory), E/M every sweep",
                                           "bound": "latency (2 cluster barriers and 2 dependent passes per sweep)",
                                           "roofline": {"bound": "alu", "ops_per_update": alu_u + madw_u,
                                                        "achieved": ach,
                                                        "peak": pk * sms_used / SM_COUNT if pk else None,
                                                        "unit": "T int32 ops/s on the 16 SMs used",
                                                        "frac": ach / (pk * sms_used / SM_COUNT) if pk else None,
                                                        "one_sm_peak": pk / SM_COUNT if pk else None,
                                                        "frac_of_one_sm": ach / (pk / SM_COUNT) if pk else None},
                                           "latency_floor": {"achieved_us": sweep_us, "floor_us": floor_us,
                                                             "frac": floor_us / sweep_us,
                                                             "what": "2 cluster barrier round trips + 2 dependent "
                                                                     "site updates per sweep"}}
    if not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(dim=3, L=16, sample_ids=[0], seed=SEED - 1)
        t0 = time.perf_counter()
        o.sweep(oracle.METROPOLIS, 1 / 1.1, 100, measure_every=1)
        dt = time.perf_counter() - t0
        out["L16_single_sample_metropolis"]["cpu_baseline"] = {
            "value": 16 ** 3 * 100 / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "the single sample, 100 sweeps with E/M every sweep"}
    del lat
    # parallel tempering
    K = 32
    beta = [1.0 / (0.7 + 0.9 * k / 31) for k in range(K)]
    pt = ianus.Lattice(dim=3, L=32, n_samples=64, n_replicas=2, n_temps=K, seed=SEED + 1, layout="bits64", stream=stream)
    pt.sweep_pt(ianus.METROPOLIS, beta, 20, swap_every=10)
    reps = 20
    sec = timed(lambda: pt.sweep_pt(ianus.METROPOLIS, beta, 100, swap_every=10), reps)
    upd = 64 * 2 * K * 32 ** 3 * 100 * reps
    rate = upd / (sec * 1e9)
    # per-lane-plane kernel, 3D Metropolis: e-words 12, adder tree 16, the
    # "always" plane by a 6-multiplexer tree over the class bits (12) and the
    # need / undecided masks (4); per plane the threshold bit by 2
    # multiplexers (4) + compare (4); per pair one Philox block from rounds 2
    # on (rounds 0 and 1 split into a site key, once per word, and parts
    # shared by the block): 16 ALU + 2 to merge the parts + 2 to merge the
    # planes, and 16 mad.wide; the site key 1 ALU and 2 mad.wide per word,
    # shared by its 2 replicas; ~3.9 plane pairs per word
    alu_word = 44 + 3.9 * (2 * 8 + 20) + 1 / 2
    out["L32_pt_32temps"] = {
        "updates_per_ns": rate, "ms_per_100_sweeps": sec * 1e3 / reps,
        "mode": "bit-sliced, per-lane threshold planes, device PT swap every 10 sweeps",
        "roofline": issue_roof(alu_word, 3.9 * 16 + 2 / 2, 64, rate),
    }
    if not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(dim=3, L=32, sample_ids=[0, 37], n_replicas=2, n_temps=K, seed=SEED + 1)
        nthr = 2
        t0 = time.perf_counter()
        o.sweep(oracle.METROPOLIS, beta, 1, nthreads=nthr)
        dt = time.perf_counter() - t0
        out["L32_pt_32temps"]["cpu_baseline"] = {"value": 2 * 2 * K * 32 ** 3 / (dt * 1e9), "unit": UNIT, "cores": nthr,
                                                 "kind": "oracle", "sample": "samples 0, 37 (64 configurations each), 1 sweep"}
    del pt
    # Potts q=4
    po = ianus.Lattice(model="potts", dim=3, L=32, n_samples=128, n_replicas=2, seed=SEED + 2, stream=stream)
    po.sweep(ianus.HEATBATH, 1 / 0.8, 10, 10)
    reps = 10
    sec = timed(lambda: po.sweep(ianus.HEATBATH, 1 / 0.8, 100, 10), reps)
    upd = 128 * 2 * 32 ** 3 * 100 * reps
    rate = upd / (sec * 1e9)
    # per 4-sample word: Philox 21 ALU; per sample 6 neighbours x (state,
    # coupling, shift, add: 4) + 3 compares with "always" flags (6) + pack (3)
    alu_word = 21 + 4 * (24 + 6 + 3)
    upd_launch = 128 * 2 * 32 ** 3 // 2
    potts_traffic = None
    if kernel_source_hash(("common.cuh", "k_potts.cu")) == POTTS_SOURCE_HASH:
        potts_traffic = dict(POTTS_TRAFFIC)
        potts_traffic["table_lookup_bytes_algorithmic"] = 16 * upd_launch  # one 16-byte row per update
        potts_traffic["updates_per_launch"] = upd_launch
        potts_traffic["source"] = "ncu, one colour launch of k_sweep_potts on this workload"
    out["potts_L32_128x2"] = {
        "updates_per_ns": rate, "ms_per_100_sweeps": sec * 1e3 / reps,
        "mode": "4 samples per uint32 word, heat bath, E/Q every 10 sweeps",
        "roofline": issue_roof(alu_word, 20, 4, rate),
        "table_traffic_per_launch": potts_traffic,
    }
    if not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(model=oracle.MODEL_POTTS, dim=3, L=32, sample_ids=[0, 127], n_replicas=2, seed=SEED + 2)
        t0 = time.perf_counter()
        o.sweep(oracle.HEATBATH, 1 / 0.8, 2, nthreads=2)
        dt = time.perf_counter() - t0
        out["potts_L32_128x2"]["cpu_baseline"] = {"value": 2 * 2 * 32 ** 3 * 2 / (dt * 1e9), "unit": UNIT, "cores": 2,
                                                  "kind": "oracle", "sample": "samples 0, 127 x 2 replicas, 2 sweeps"}
    del po
    # random-field Ising model (Eq. 2, h_i = +-|h|), bit-sliced layout, heat bath
    hm, Tr = 1.5, 2.0
    rf = ianus.Lattice(dim=3, L=64, n_samples=256, n_replicas=1, seed=SEED + 4, layout="bits64", disorder="rfim",
                       field=hm, stream=stream)
    rf.sweep(ianus.HEATBATH, 1 / Tr, 10, 10)
    reps = 10
    sec = timed(lambda: rf.sweep(ianus.HEATBATH, 1 / Tr, 100, 10), reps)
    upd = 256 * 64 ** 3 * 100 * reps
    rate = upd / (sec * 1e9)
    # kernel specialised at run time for the field tables; per word: e-words
    # 12, adder tree 16, f 2, "always"/"need" tables (u, f) 12, write-back 3;
    # per plane: threshold bit 3 lop3 x 2 halves + compare 4; per pair Philox
    # 21 ALU + merge 2; 3.92 plane pairs per word on average
    alu_word = 45 + 3.92 * (2 * (6 + 4) + 23)
    out["rfim_L64_256_h1.5"] = {
        "updates_per_ns": rate, "ms_per_100_sweeps": sec * 1e3 / reps,
        "mode": "bit-sliced, field kernel specialised at run time ((u, f) tables as lop3 immediates), heat bath "
                "T=2.0, |h|=1.5, E/M/F every 10 sweeps",
        "roofline": issue_roof(alu_word, 3.92 * 20, 64, rate),
    }
    if not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(dim=3, L=64, sample_ids=[0, 255], seed=SEED + 4, disorder=oracle.DIS_RFIM, field=hm)
        t0 = time.perf_counter()
        o.sweep(oracle.HEATBATH, 1 / Tr, 2, nthreads=2)
        dt = time.perf_counter() - t0
        out["rfim_L64_256_h1.5"]["cpu_baseline"] = {"value": 2 * 64 ** 3 * 2 / (dt * 1e9), "unit": UNIT, "cores": 2,
                                                    "kind": "oracle", "sample": "samples 0, 255, 2 sweeps"}
    del rf
    # diluted antiferromagnet in a field, bit-sliced, Metropolis
    hd, occ, Td = 1.0, 0.7, 1.5
    da = ianus.Lattice(dim=3, L=64, n_samples=256, n_replicas=1, seed=SEED + 5, layout="bits64", disorder="daff",
                       field=hd, occupation=occ, stream=stream)
    da.sweep(ianus.METROPOLIS, 1 / Td, 10, 10)
    reps = 10
    sec = timed(lambda: da.sweep(ianus.METROPOLIS, 1 / Td, 100, 10), reps)
    upd = 256 * 64 ** 3 * 100 * reps
    rate = upd / (sec * 1e9)
    # kernel specialised at run time; per word: e-words 12, occupied
    # satisfied-bond words 12, occupation and bond count trees 32, the 4-bit
    # sum t 10, f 2, "always"/"need" tables 28, write-back 4; per plane:
    # threshold bit 7 lop3 x 2 halves + compare 4; per pair Philox 21 ALU +
    # merge 2; 3.92 plane pairs per word on average (occupied lanes)
    alu_word = 100 + 3.92 * (2 * (14 + 4) + 23)
    out["daff_L64_256_occ0.7_h1.0"] = {
        "updates_per_ns": rate, "ms_per_100_sweeps": sec * 1e3 / reps,
        "mode": "bit-sliced with occupation words, kernel specialised at run time ((t, f) tables, t = v + 2D as "
                "4 bit-planes), Metropolis T=1.5, |h|=1.0, occupation 0.7, E/M/F every 10 sweeps",
        "roofline": issue_roof(alu_word, 3.92 * 20, 64, rate),
    }
    if not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(dim=3, L=64, sample_ids=[0, 255], seed=SEED + 5, disorder=oracle.DIS_DAFF, field=hd,
                          occupation=occ)
        t0 = time.perf_counter()
        o.sweep(oracle.METROPOLIS, 1 / Td, 2, nthreads=2)
        dt = time.perf_counter() - t0
        out["daff_L64_256_occ0.7_h1.0"]["cpu_baseline"] = {
            "value": 2 * 64 ** 3 * 2 / (dt * 1e9), "unit": UNIT, "cores": 2, "kind": "oracle",
            "sample": "samples 0, 255, 2 sweeps"}
    del da
    # the headline update on a lattice 8x larger than the bench workload, L=128:
    # 320 MiB of spins and couplings, beyond the 129 MB L2, so every sweep
    # streams the state from HBM; unique bytes per site word per sweep: both
    # replicas' words read and written (32) and the three couplings (24), for
    # 128 updates
    big = ianus.Lattice(dim=3, L=128, n_samples=S, n_replicas=R, seed=SEED + 8, layout="bits64", stream=stream)
    big.set_variant(DEFAULT_VARIANT[0])
    big.set_block_words(DEFAULT_VARIANT[1])
    big.sweep(ianus.HEATBATH, 1.0 / T, 4, 0)
    reps = 3
    sec = timed(lambda: big.sweep(ianus.HEATBATH, 1.0 / T, 20, 0), reps)
    upd = S * R * 128 ** 3 * 20 * reps
    rate = upd / (sec * 1e9)
    bytes_upd = (32 + 24) / 128.0
    hbm = MEASURED.get("hbm_gbs")
    ops = algorithmic_ops_per_word_hb3d(R)
    out["L128_256x2_hb_out_of_l2"] = {
        "updates_per_ns": rate, "ms_per_sweep": sec * 1e3 / (20 * reps),
        "mode": "bit-sliced, lane-queue kernel (the bench variant), state 320 MiB > L2",
        "roofline": issue_roof(ops["lop3"], ops["mad_wide"], 64, rate),
        "hbm": {"bytes_per_update": bytes_upd, "achieved": rate * bytes_upd, "peak": hbm, "unit": "GB/s",
                "frac": (rate * bytes_upd / hbm) if hbm else None},
    }
    del big
    # the bench workload on the plain layout driven by Parisi-Rapuano wheels (Eq. 5)
    wh = ianus.Lattice(dim=3, L=L, n_samples=S, n_replicas=R, seed=SEED + 7, layout="i8", rng="wheel", stream=stream)
    wh.sweep(ianus.HEATBATH, 1.0 / T, 2, 0)
    reps = 3
    sec = timed(lambda: wh.sweep(ianus.HEATBATH, 1.0 / T, 10, 10), reps)
    upd = S * R * L ** 3 * 10 * reps
    rate = upd / (sec * 1e9)
    # unique bytes per update: spin read + write (2), 3 couplings, and per
    # row-colour wheel the 64-word ring read + L/2 words written for L/2 updates
    bytes_upd = 2.0 + 3.0 + (64 + L / 2) * 4 / (L / 2)
    hbm = MEASURED.get("hbm_gbs")
    out["wheel_L64_256x2_hb"] = {
        "updates_per_ns": rate, "ms_per_10_sweeps": sec * 1e3 / reps,
        "mode": "plain int8, one Parisi-Rapuano wheel per (configuration, row, colour), heat bath T=1.0",
        "roofline": {"bound": "hbm", "bytes_per_update": bytes_upd, "achieved": rate * bytes_upd, "peak": hbm,
                     "unit": "GB/s", "frac": (rate * bytes_upd / hbm) if hbm else None},
    }
    if not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(dim=3, L=L, sample_ids=[0, 255], n_replicas=R, seed=SEED + 7, rng=oracle.RNG_WHEEL)
        t0 = time.perf_counter()
        o.sweep(oracle.HEATBATH, 1.0 / T, 1, nthreads=2)
        dt = time.perf_counter() - t0
        out["wheel_L64_256x2_hb"]["cpu_baseline"] = {"value": 2 * R * L ** 3 / (dt * 1e9), "unit": UNIT, "cores": 2,
                                                     "kind": "oracle", "sample": "samples 0, 255 x 2 replicas, 1 sweep"}
    del wh
    # glassy Potts model with permutation couplings (Eq. 3), 3D and 4D, heat bath
    for dim, Lp, bp, key in ((3, 32, 2.4, "potts_perm_3d_L32_256x2"), (4, 16, 1.405, "potts_perm_4d_L16_256x2")):
        pp = ianus.Lattice(model="potts_perm", dim=dim, L=Lp, n_samples=256, n_replicas=2, seed=SEED + 6,
                           stream=stream)
        pp.sweep(ianus.HEATBATH, bp, 10, 10)
        reps = 5
        sec = timed(lambda: pp.sweep(ianus.HEATBATH, bp, 100, 10), reps)
        upd = 256 * 2 * Lp ** dim * 100 * reps
        rate = upd / (sec * 1e9)
        # per 4-sample word: Philox 21; per sample and bond ~7 (state and code
        # fields, target state, nibble increment), table index 4, selection 6,
        # pack 2
        alu_word = 21 + 4 * (2 * dim * 7 + 12)
        out[key] = {
            "updates_per_ns": rate, "ms_per_100_sweeps": sec * 1e3 / reps,
            "mode": f"4 samples per uint32 word, {dim}D, heat bath beta={bp}, E/Q every 10 sweeps",
            "roofline": issue_roof(alu_word, 20, 4, rate),
        }
        if not args.no_cpu_baseline:
            import oracle

            o = oracle.Oracle(model=oracle.MODEL_PERM, dim=dim, L=Lp, sample_ids=[0, 255], n_replicas=2,
                              seed=SEED + 6)
            t0 = time.perf_counter()
            o.sweep(oracle.HEATBATH, bp, 1, nthreads=2)
            dt = time.perf_counter() - t0
            out[key]["cpu_baseline"] = {"value": 2 * 2 * Lp ** dim / (dt * 1e9), "unit": UNIT, "cores": 2,
                                        "kind": "oracle", "sample": "samples 0, 255 x 2 replicas, 1 sweep"}
        del pp
    # resident sweeps of small bit-sliced lattices: 3D L=8 (the serving mix's
    # smallest side), one replica, heat bath T=1.0, no measurements; 152
    # groups of 64 samples (one resident block per SM) and a single group,
    # against the same lattices swept launch by launch (resident mode off)
    res_out = {}
    for groups, n in ((152, 1000), (1, 1000)):
        rl = ianus.Lattice(dim=3, L=8, n_samples=64 * groups, n_replicas=1, seed=SEED + 9, layout="bits64",
                           stream=stream)
        rates = {}
        for mode in (1, 0):
            rl.set_resident(mode)
            rl.sweep(ianus.HEATBATH, 1.0, 20)
            reps = 3
            sec = timed(lambda: rl.sweep(ianus.HEATBATH, 1.0, n), reps)
            rates["resident" if mode else "launch_per_colour"] = {
                "updates_per_ns": 64 * groups * 8 ** 3 * n * reps / (sec * 1e9), "us_per_sweep": sec * 1e6 / (n * reps)}
        res_out[f"{groups}x64"] = rates
        del rl
    # per-lane-plane update, 3D heat bath: e-words 12, adder tree 16, the
    # "always" plane (12) and the undecided mask (4); per plane the
    # threshold bit by a 7-way multiplexer tree (6) + compare (4); per pair
    # one Philox block from rounds 2 on (18 ALU, 16 mad.wide) + merge 2;
    # 3.92 plane pairs per word; the site key 1 ALU and 2 mad.wide per word
    alu_word = 44 + 3.92 * (2 * 10 + 20) + 1
    out["resident_L8_64xG_hb"] = {
        **res_out,
        "mode": "bit-sliced, k_resident_bits: one block per 64-sample group holds spins, couplings and threshold "
                "planes in shared memory for up to 4096 sweeps per launch; heat bath T=1.0, one replica",
        "roofline": issue_roof(alu_word, 3.92 * 16 + 2, 64, res_out["152x64"]["resident"]["updates_per_ns"]),
    }
    # device-side set-up: couplings and initial spins of the bench workload from the seed
    t0 = time.perf_counter()
    lat = ianus.Lattice(dim=3, L=L, n_samples=S, n_replicas=R, seed=SEED + 3, layout="bits64", stream=stream)
    torch.cuda.synchronize()
    out["init_L64_256x2"] = {"seconds": time.perf_counter() - t0,
                             "what": "ianus_lattice_create: buffer clear + couplings and spins from the seed (wall)"}
    del lat
    return out


def _measured_peaks() -> dict:
    """Measured copy bandwidth and GEMM peaks of this GPU model, if recorded."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


MEASURED = _measured_peaks()


def _alu_peak():
    p = probe_peak()
    return p["lop3_per_clk_sm"] * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12 if p else None


def issue_roof(alu_word: float, madw_word: float, lanes: int, rate: float) -> dict:
    """Roofline entry of an integer-bound sweep: algorithmic lop3-class ops
    (ALU pipe) and 64-bit products (mad.wide) per word of `lanes` updates,
    against the shared issue peak of the two."""
    peak = _issue_peak()
    per_upd = (alu_word + madw_word) / lanes
    ach = rate * per_upd / 1e3
    return {"bound": "alu", "ops_per_update": per_upd, "alu_ops_per_word": alu_word, "mad_wide_per_word": madw_word,
            "achieved": ach, "peak": peak, "unit": "T int32 ops/s (lop3 + mad.wide, one shared issue slot)",
            "frac": (ach / peak) if peak else None}


def _issue_peak():
    """lop3 and mad.wide share one issue slot: the rate of the two side by
    side is the peak for any mix of them."""
    p = probe_peak()
    return p["lop3_madwide_per_clk_sm"] * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12 if p else None


def run_serving(args):
    """The serving mix as configured (2000 jobs: 3D/2D EA jobs of 1..64
    samples, L from the listed sides, T in [0.5, 2], sweeps log-uniform in
    [10^3, 10^5] times --serve-scale, Metropolis or heat bath), Poisson
    arrivals at 0.8 x the capacity the lane-fusing server (FusedServer: jobs
    of equal (D, L) share the 64-bit lanes of pool lattices, large jobs on
    their own lattices) reaches on a saturated run of the whole mix; p50/p99
    latency and aggregate spin updates/ns.  Beside it, the server that gives
    every job its own lattice (Server), saturated on the first 100 jobs."""
    from paper_0704_3573_gb300 import serve

    jobs = serve.job_mix(args.serve_jobs, sweep_scale=args.serve_scale)
    fused = serve.FusedServer(mem_budget=16 << 30, groups_per_pool=4, n_streams=16, chunk_sweeps=50)
    calib = jobs  # capacity: the whole mix at t = 0
    _, sat = fused.run(calib, realtime=False)
    rate = 0.8 * len(calib) / sat["makespan_s"] if sat["makespan_s"] > 0 else math.inf
    arrivals = serve.poisson_arrivals(jobs, rate)
    _, st = fused.run(arrivals)
    st["server"] = "FusedServer (lane fusion of jobs of equal (D, L); jobs over 2^16 sites on their own lattices)"
    st["arrival_rate_per_s"] = rate
    st["offered_load"] = 0.8
    st["sweep_scale"] = args.serve_scale
    st["mix"] = ("3D L in {8..80} / 2D L in {64..1024}, 1-64 samples, T~U[0.5,2], sweeps log-U[1e3,1e5] x scale, "
                 "Metropolis / heat bath")
    st["saturated"] = {"jobs": len(calib), "makespan_s": sat["makespan_s"], "updates_per_ns": sat["updates_per_ns"],
                       "p50_latency_s": sat["p50_latency_s"], "p99_latency_s": sat["p99_latency_s"],
                       "what": "the whole mix at t = 0: the capacity the arrival rate is calibrated on"}
    plain = serve.Server(mem_budget=16 << 30, max_active=64, n_streams=16, chunk_sweeps=50)
    sub = jobs[: min(100, len(jobs))]
    _, sat_plain = plain.run(sub, realtime=False)
    st["unfused_saturated"] = {"jobs": len(sub), "makespan_s": sat_plain["makespan_s"],
                               "updates_per_ns": sat_plain["updates_per_ns"],
                               "what": "Server: every job on its own lattice, all jobs at t=0"}
    return st


_PROBE = []


def probe_peak():
    """Integer rates per clock per SM from libianus_probe.so (measured once
    per process)."""
    if _PROBE:
        return _PROBE[0]
    import paper_0704_3573_gb300.build as b

    out = None
    try:
        P = C.CDLL(b.PROBE_LIB)
        P.ianus_probe_int.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
        out = {}
        for kind, name in ((0, "lop3_per_clk_sm"), (1, "imad_wide_per_clk_sm"), (2, "philox_mix_per_clk_sm"),
                           (3, "philox_blocks_per_clk_sm"), (4, "lop3_madwide_per_clk_sm"),
                           (7, "lop3_imad_per_clk_sm"), (8, "imad_hi_per_clk_sm")):
            v = C.c_double()
            if P.ianus_probe_int(kind, 4, C.byref(v)) != 0:
                out = None
                break
            out[name] = v.value
    except OSError:
        out = None
    _PROBE.append(out)
    return out


def run_e2e(ianus, lat, stream, args, ws):
    """Per step: upload the state blob from pinned host memory (set_state),
    run the 100-sweep block, read the measurement series into pinned host
    arrays.  All through the C ABI."""
    import torch

    L_ = lat._lib
    n = C.c_size_t()
    L_.ianus_get_state(lat._h, None, 0, C.byref(n))
    blob = torch.empty(n.value, dtype=torch.uint8, pin_memory=True)
    assert L_.ianus_get_state(lat._h, C.c_void_p(blob.data_ptr()), n.value, C.byref(n)) == 0
    rows = SWEEPS_PER_STEP // MEASURE_EVERY
    SK, SKR = S, S * R
    sw = torch.empty(rows, dtype=torch.int64, pin_memory=True)
    E = torch.empty(rows * SKR, dtype=torch.int64, pin_memory=True)
    M = torch.empty(rows * SKR, dtype=torch.int64, pin_memory=True)
    Q = torch.empty(rows * SK, dtype=torch.int64, pin_memory=True)
    beta = (C.c_double * 1)(1.0 / T)
    nrow = C.c_size_t()
    steps = max(3, min(args.steps, args.e2e_steps))
    times = []
    for k in range(steps + 1):
        t0 = time.perf_counter()
        st = L_.ianus_set_state(lat._h, C.c_void_p(blob.data_ptr()), n.value)
        st |= L_.ianus_sweep(lat._h, ianus.HEATBATH, beta, SWEEPS_PER_STEP, MEASURE_EVERY)
        st |= L_.ianus_read_series(lat._h, C.c_void_p(sw.data_ptr()), C.c_void_p(E.data_ptr()),
                                   C.c_void_p(M.data_ptr()), C.c_void_p(Q.data_ptr()), rows, C.byref(nrow), 1)
        dt = time.perf_counter() - t0
        assert st == 0 and nrow.value == rows
        if k > 0:  # first iteration re-uploads tables after set_state
            times.append(dt)
    t = max_over_ranks(sum(times), ws)
    return {"value": ws * S * R * L ** 3 * SWEEPS_PER_STEP * len(times) / (t * 1e9), "unit": UNIT,
            "h2d_bytes_per_step": int(n.value), "d2h_bytes_per_step": int(rows * (8 + 8 * (2 * SKR + SK))),
            "steps": len(times), "what": "set_state (pinned H2D) + 100 sweeps + read_series (pinned D2H)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ianus", choices=["ianus", "reference"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-sweeps", type=int, default=MEASURE_EVERY)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--no-others", action="store_true")
    ap.add_argument("--tune", action="store_true", help="pick the kernel variant with the autotuner")
    ap.add_argument("--variant", type=int, default=None, help="kernel variant (default: the profiled one)")
    ap.add_argument("--block-words", type=int, default=0, help="launch shape with --variant (0 = heuristic)")
    ap.add_argument("--serve-scale", type=float, default=1.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        import __graft_entry__

        __graft_entry__.build()
        run_gpu(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
