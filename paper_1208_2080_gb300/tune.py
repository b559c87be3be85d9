"""Autotuner for the batched replica runner.

Chooses, for a given batch (its mix of lattice sizes), the labelling tile
height (32, 64 or 128 rows of 128 sites), the merge schedule (the boundary
unions in a kernel of their own, or done by the labeller itself: the tile
that finishes second unites across a shared edge) and whether a batch sweep
is replayed as a CUDA graph or launched directly, by timing a few sweeps of
each candidate with CUDA events.  Results are cached in a JSON file keyed by
the GPU name and the batch's size histogram.  Choices never change results:
every candidate is bit-identical (tests check that), only speed differs.
"""
import json
import os
import time

import numpy as np

from ._binding import Batch

CANDIDATES = [(th, g, m) for th in (128, 64, 32) for m in ("kernel", "fused") for g in (True, False)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "swgb", "tune.json")


def _key(L, gpu):
    vals, counts = np.unique(np.asarray(L, dtype=np.uint64), return_counts=True)
    return gpu + "|" + ",".join(f"{int(v)}x{int(c)}" for v, c in zip(vals, counts))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def time_batch(L, q, T, seed, tile_h, graph, merge="kernel", sweeps=4, warmup=2):
    """Mean device milliseconds per batch sweep for one candidate."""
    import torch
    with Batch(L, q, T, seed, tile_h=tile_h, graph=graph, merge=merge) as b:
        b.sweep(warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.sweep(sweeps)
        e1.record()
        torch.cuda.synchronize()
        b.sync()
        return e0.elapsed_time(e1) / sweeps


def tune_batch(L, q, T, seed, *, cache=DEFAULT_CACHE, sweeps=4, force=False, candidates=None):
    """Returns {"tile_h": .., "graph": .., "merge": .., "ms_per_sweep": .., "timings": [...]}
    for the batch, measuring (and caching) if needed."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(L, gpu)
    db = _load(cache)
    if not force and key in db:
        return db[key]
    timings = []
    for th, g, m in (candidates or CANDIDATES):
        t0 = time.time()
        ms = time_batch(L, q, T, seed, th, g, m, sweeps=sweeps)
        timings.append({"tile_h": th, "graph": g, "merge": m, "ms_per_sweep": ms, "wall_s": time.time() - t0})
    best = min(timings, key=lambda x: x["ms_per_sweep"])
    res = {"tile_h": best["tile_h"], "graph": best["graph"], "merge": best["merge"],
           "ms_per_sweep": best["ms_per_sweep"], "timings": timings}
    db[key] = res
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache + ".tmp", "w") as f:
            json.dump(db, f, indent=1)
        os.replace(cache + ".tmp", cache)
    except OSError:
        pass
    return res


def tuned_batch(L, q, T, seed, **kw):
    """A Batch built with the tuned tile height, merge schedule and launch mode."""
    cfg = tune_batch(L, q, T, seed)
    return Batch(L, q, T, seed, tile_h=cfg["tile_h"], graph=cfg["graph"],
                 merge=cfg.get("merge", "kernel"), **kw), cfg
