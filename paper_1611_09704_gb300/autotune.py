"""Autotuner of the batched search's launch shape (spd_tuning).

For a given batch (the DM ranges' shapes, storage type, width sets,
thresholds and sigma modes) every candidate launch shape -- persistent CTAs
per SM, width-group size (widths per pass between bounds) and tile length
(threads per CTA: a tile is 16 starts per thread less the halo's blocks) --
is timed on the device with CUDA events, and the fastest is kept.  Results are cached in a JSON file keyed by the device
and a hash of the batch description, so a serving process tunes once.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

CANDIDATES = [{"ctas_per_sm": c, "group_scale": g, "tile_threads": t}
              for t in (256, 128) for c in (0, 1) for g in (1, 2, 4)]


def batch_key(specs, device_name: str) -> str:
    """Stable key of a batch: device, storage type, shapes and search parameters."""
    desc = []
    for r in specs:
        x = r.x.data if hasattr(r.x, "n_samp") else r.x
        n_samp = r.x.n_samp if hasattr(r.x, "n_samp") else x.shape[1]
        desc.append([str(x.dtype), int(x.shape[0]), int(n_samp), [int(w) for w in r.widths],
                     float(r.threshold), int(r.sigma_mode), int(r.scope), int(r.nmax)])
    blob = json.dumps([device_name, desc], sort_keys=True).encode()
    return hashlib.sha1(blob).hexdigest()


def load_cache(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(path, cache):
    if not path:
        return
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(timings: dict) -> dict:
    """The candidate with the smallest median time (ties: first listed)."""
    best = min(timings, key=lambda k: (timings[k], list(timings).index(k)))
    return json.loads(best)


def autotune(specs, capacity, cache_path=None, reps=5, candidates=None, timer=None):
    """Return {"tuning": {...}, "timings_ms": {...}, "cached": bool}.

    timer(specs, capacity, tuning, reps) -> median milliseconds; the default
    times BatchedSearch runs with CUDA events on the current stream."""
    import torch
    candidates = candidates or CANDIDATES
    dev = (specs[0].x.data if hasattr(specs[0].x, "n_samp") else specs[0].x).device
    name = torch.cuda.get_device_name(dev) if dev.type == "cuda" else str(dev)
    key = batch_key(specs, name)
    cache = load_cache(cache_path)
    if key in cache:
        e = cache[key]
        return {"tuning": e["tuning"], "timings_ms": e["timings_ms"], "cached": True}
    timer = timer or _time_batched
    timings = {}
    for cand in candidates:
        timings[json.dumps(cand, sort_keys=True)] = timer(specs, capacity, cand, reps)
    best = choose(timings)
    cache[key] = {"tuning": best, "timings_ms": timings}
    save_cache(cache_path, cache)
    return {"tuning": best, "timings_ms": timings, "cached": False}


def _time_batched(specs, capacity, tuning, reps):
    import torch

    from .binding import BatchedSearch
    bs = BatchedSearch(specs, capacity, tuning=tuning, graph=False)
    bs.run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        bs.run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)
