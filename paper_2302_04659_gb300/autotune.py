"""Autotuner of the substep's launch shape.

The knobs are those of ``mpm_set_launch``: the most particles per chunk of a bin (one CTA iteration of
the fused G2P->P2G pass; smaller chunks cut bins with many particles into more pieces, balancing the
persistent CTAs), the resident CTAs per SM of the fused pass (more hide latency, fewer leave more L1 and
issue slots to each) and the CTAs per SM of the grid update. The best shape depends on the particle
count, the number and size of the grids and the materials, so it is measured, not modelled: a
coordinate descent over the three knobs, each candidate timed with CUDA events over a few substeps of
the handle's own scene after a warm-up (the first replay of a shape also captures its graph). Results
are cached per workload signature and device in a JSON file next to the built library.

The trials advance the handle's state; ``prepare`` (called before every trial) and ``restore`` (called
once at the end) let the caller reset colliders and particles.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import _native as mpm
from . import build as _build

CHUNKS = (256, 192, 128, 96, 64)
FUSED_CTAS = (7, 6, 5, 4, 3, 2)
GRID_CTAS = (1, 2, 4)
CACHE_PATH = os.path.join(os.path.dirname(_build.LIB_PATH), "autotune.json")


def signature(sim) -> str:
    """Workload signature: device, env count, particle count (to a factor of sqrt 2), grid sizes, kinds."""
    dev = torch.cuda.get_device_name(sim.device)
    N = max(sim.N, 1)
    bucket = round(2 * math.log2(N))
    ns = sorted(set(getattr(sim, "ns", [getattr(sim, "n", 0)])))
    kinds = sorted(set(getattr(sim, "kinds", [])))
    nenv = getattr(sim, "nenv", 1)
    return (f"{dev}|envs={nenv}|N~2^{bucket / 2:.1f}|n={','.join(map(str, ns))}|kinds={','.join(map(str, kinds))}"
            f"|chunks<={CHUNKS[0]}")


def _load_cache() -> dict:
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
    tmp = CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE_PATH)


def time_shape(sim, shape, substeps: int, reps: int, prepare=None, stream=None) -> float:
    """Mean milliseconds per substep of ``sim`` with launch shape (chunk, fused CTAs/SM, grid CTAs/SM)."""
    stream = stream or torch.cuda.current_stream(sim.device)
    sim.set_launch(*shape)
    if prepare:
        prepare()
    sim.substep(substeps, stream=stream)  # warm-up: captures this shape's graph
    best = float("inf")
    for _ in range(reps):
        if prepare:
            prepare()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.substep(substeps, stream=stream)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) / substeps)
    return best


def max_fused_for(sim, chunk: int, cap: int | None = None) -> int:
    """The most fused-pass CTAs per SM the handle accepts with this chunk size (the fused pass's CTA size,
    and so its occupancy limit, follows the chunk)."""
    for f in FUSED_CTAS:
        if cap is not None and f > cap:
            continue
        try:
            sim.set_launch(chunk, f, 0)
            return f
        except mpm.MpmError:
            continue
    return FUSED_CTAS[-1]


def tune(sim, substeps: int = 10, reps: int = 3, prepare=None, restore=None, use_cache: bool = True,
         max_fused: int | None = None):
    """Choose and apply the fastest launch shape for ``sim``'s current scene. Returns
    (shape, ms per substep, trials) where trials maps each timed shape to its ms per substep (empty when
    the shape came from the cache)."""
    key = signature(sim)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        shape = tuple(cache[key]["shape"])
        sim.set_launch(*shape)
        return shape, cache[key]["ms_per_substep"], {}
    start_shape = tuple(sim.get_launch())
    limits = {c: max_fused_for(sim, c, max_fused) for c in CHUNKS}
    trials = {}

    def trial(shape):
        if shape not in trials:
            trials[shape] = time_shape(sim, shape, substeps, reps, prepare)
        return trials[shape]

    c0, f0, g0 = start_shape
    best = (c0, min(f0, limits.get(c0, f0)), g0)
    for _ in range(2):  # coordinate descent, two rounds
        start = best
        c, f, g = best
        cands = [(c, fo, g) for fo in FUSED_CTAS if fo <= limits.get(c, fo)]
        best = min(cands, key=trial)
        c, f, g = best
        # a chunk of another CTA size takes that size's own most CTAs per SM when f exceeds it
        best = min([(co, min(f, limits[co]), g) for co in CHUNKS], key=trial)
        c, f, g = best
        best = min([(c, f, go) for go in GRID_CTAS], key=trial)
        if best == start:
            break
    sim.set_launch(*best)
    if restore:
        restore()
    if use_cache:
        cache = _load_cache()
        cache[key] = {"shape": list(best), "ms_per_substep": trials[best]}
        _store_cache(cache)
    return best, trials[best], {f"{c}/{f}/{g}": ms for (c, f, g), ms in trials.items()}
