"""Autotuner for the bulk stream-collide pass of the 16/32-bit storages.

The variants (include/fsl.h, FSL_VARIANT_*) differ in cells per thread (two
or four), block shape (64 or 128 threads), register cap and the way stored
values reach the registers (direct loads with warp shuffles, TMA bulk copies
into a shared-memory ring, or 16-byte asynchronous copies by every thread
into a shared-memory ring).  All give identical results, so the choice
is purely a matter of speed, and the best one depends on the domain's extent
along x, its liquid fraction, the lattice and the storage type.  `tune`
times each candidate on the simulation's current state with the library's
own CUDA-event measurement (the bulk pass together with any list pre-pass
the variant needs) and keeps the fastest; `tune_batch` tunes one
representative per distinct (lattice, storage, shape) and applies the pick
to every simulation of that kind.  Picks can be kept in a JSON file so that a
later run skips the measurements.
"""
from __future__ import annotations

import json
import os

from . import fsl

CANDIDATES = ("pair", "pair_r128", "pair_r96", "pair_r80", "tma", "quad64", "warp_tma", "pair_pipe",
              "cpa", "cpa_deep", "cpa_r96", "seg", "seg_r128",
              "cell", "cell_r80", "tma_r96")
HALF_ONLY = ("quad64", "pair_pipe", "cpa_r96", "tma_r96")


def key_of(sim) -> str:
    nx, ny, nz = sim.shape
    return f"q{sim.q}/{sim.precision}/{nx}x{ny}x{nz}"


def _allowed(sim, v: str) -> bool:
    return not (v in HALF_ONLY and sim.precision == "fp32")


def tune(sim, reps: int = 5, candidates=CANDIDATES) -> dict:
    """Time every candidate variant on `sim` (initialised), switch it to the
    fastest and return {"variant": name, "ms": {name: time per pass}}.  The
    FP64 path has a single kernel and is left alone."""
    if sim.precision == "fp64":
        return dict(variant="default", ms={})
    ms = {}
    for v in candidates:
        if not _allowed(sim, v):
            continue
        sim.set_variant(v)
        ms[v] = sim.kernel_stats(reps=reps, kernel=fsl.KERNEL_BULK_PASS)["ms"]
    best = min(ms, key=ms.get)
    sim.set_variant(best)
    return dict(variant=best, ms=ms)


def tune_step(sim, candidates, steps: int = 20) -> dict:
    """Time whole steps (CUDA events on the simulation's stream, graph
    replay) with each candidate variant and keep the fastest: the interface
    pass runs beside the bulk pass and competes with it for the SMs, so the
    fastest bulk pass alone need not give the fastest step.  The state is
    checkpointed first and restored at the end, so the tuning steps leave no
    trace.  Returns
    {"variant": name, "ms_step": {name: ms per step}}."""
    import torch
    if sim.precision == "fp64":
        return dict(variant="default", ms_step={})
    ck = sim.save()
    ms = {}
    for v in candidates:
        if not _allowed(sim, v):
            continue
        sim.set_variant(v)
        sim.step(2)  # capture the step graph outside the timing
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms[v] = e0.elapsed_time(e1) / steps
    best = min(ms, key=ms.get)
    sim.set_variant(best)
    sim.load(ck)
    return dict(variant=best, ms_step=ms)


def tune_batch(sims, reps: int = 5, cache_path: str | None = None) -> dict:
    """Tune one representative per (lattice, storage, shape) and apply the
    pick to all simulations of that kind.  With `cache_path`, picks found in
    the file are applied without measuring and new picks are added to it."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    groups: dict[str, list] = {}
    for s in sims:
        groups.setdefault(key_of(s), []).append(s)
    picks = {}
    for key, members in groups.items():
        if key in cache and _allowed(members[0], cache[key]["variant"]):
            r = cache[key]
        else:
            r = tune(members[0], reps)
        for s in members:
            if r["variant"] != "default":
                s.set_variant(r["variant"])
        picks[key] = r
    if cache_path:
        cache.update(picks)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return picks
