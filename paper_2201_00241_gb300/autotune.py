"""Autotuner for the right-hand-side interleave width of batched launches.

The width (directions per CTA) trades lane occupancy and level-barrier
amortisation against the number of CTAs: narrow widths spread a batch over more
SMs, wide ones amortise each CTA's per-level latency over more directions.  The
best value depends on the grids and the batch, so it is measured: each candidate
runs the batch (after one warm-up) and the fastest CUDA-event time wins.
Results are cached per (grid shapes, widths of the items) in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import rh

DEFAULT_WIDTHS = (0, 2, 4, 8, 16, 32)


def _key(items) -> str:
    sig = [(g.n_bus, g.n_x, g.n_p, int(W.shape[1])) for g, W, _, _ in items]
    return hashlib.sha256(json.dumps(sig).encode()).hexdigest()[:24]


def tune_width(items, widths=DEFAULT_WIDTHS, reps: int = 3, cache_path: str | None = None) -> tuple[int, dict]:
    """Return (best width, {width: ms}) for rh_batch_hessvec on `items`."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    key = _key(items)
    if key in cache:
        return int(cache[key]["best"]), {int(k): v for k, v in cache[key]["ms"].items()}
    times = {}
    stream = torch.cuda.current_stream()
    for w in widths:
        rh.batch_hessvec(items, w)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            rh.batch_hessvec(items, w)
        e1.record(stream)
        torch.cuda.synchronize()
        times[w] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    if cache_path:
        cache[key] = {"best": best, "ms": {str(k): v for k, v in times.items()}}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, times
