"""Autotuner for the bit-sliced sweep: kernel variant and launch shape.

For a lattice and an (algorithm, beta) it times every candidate kernel
variant (the automatic choice, which sweeps small lattices resident in shared
memory; precompiled per-lane threshold planes; or one of the shapes of the
kernel specialised at run time: lockstep, per-warp queues, the lane-queue
kernel and its persistent form) and several launch shapes (colour words per
block) on a short block of sweeps, and keeps the fastest.  The state is snapshotted before and
restored after every trial, so tuning never changes the simulation: the
trajectory after tune() is the one the lattice would have followed anyway.
Choices are cached in a JSON file keyed by GPU name and lattice shape.
"""

from __future__ import annotations

import json
import os
import tempfile

VARIANTS = tuple(range(0, 28))
BLOCK_WORDS = (0, 256, 512, 1024, 2048)


def cache_path() -> str:
    return os.environ.get("IANUS_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "ianus_tune.json"))


def _key(lat, algo: int, gpu: str) -> str:
    return f"{gpu}|D{lat.dim}|L{lat.L}|S{lat.S}|R{lat.R}|K{lat.K}|layout{lat.cfg.layout}|algo{algo}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict):
    path = cache_path()
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(lat, algo, beta, sweeps: int = 20, variants=VARIANTS, block_words=BLOCK_WORDS, use_cache: bool = True):
    """Pick and apply the fastest (variant, block_words) for this lattice.
    Returns {"variant", "block_words", "us_per_sweep", "trials"}."""
    import torch

    gpu = torch.cuda.get_device_name(lat.device)
    key = _key(lat, algo, gpu)
    cache = _load() if use_cache else {}
    if key in cache:
        best = cache[key]
        lat.set_variant(best["variant"])
        lat.set_block_words(best["block_words"])
        return dict(best, cached=True)
    blob = lat.get_state()
    trials = []
    for v in variants:
        for bw in block_words:
            lat.set_state(blob)
            lat.set_variant(v)
            lat.set_block_words(bw)
            with torch.cuda.stream(lat.stream):
                lat.sweep(algo, beta, 2)  # builds tables / compiles the specialised kernel
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(lat.stream)
                lat.sweep(algo, beta, sweeps)
                e1.record(lat.stream)
            torch.cuda.synchronize()
            trials.append((e0.elapsed_time(e1) * 1e3 / sweeps, v, bw))
    lat.set_state(blob)
    us, v, bw = min(trials)
    lat.set_variant(v)
    lat.set_block_words(bw)
    best = {"variant": v, "block_words": bw, "us_per_sweep": us}
    if use_cache:
        cache = _load()
        cache[key] = best
        _save(cache)
    return dict(best, cached=False, trials=[{"us_per_sweep": t, "variant": a, "block_words": b} for t, a, b in trials])
