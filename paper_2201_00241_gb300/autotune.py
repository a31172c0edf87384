"""Autotuner of batched reduced-Hessian-vector launches (Algorithm 2 over blocks of
N directions, section 5.3).

A batched launch (rh_batch_hessvec_cfg) has four choices that trade against one
another and depend on the grids and the batch:

* width: directions per CTA (the right-hand-side interleave width; 0 spreads each
  item over the CTA slots).  Narrow widths spread a batch over more SMs, wide ones
  amortise each CTA's per-level barrier over more directions.
* threads: the CTA shape, one of the compiled 128 x 6, 192 x 4, 256 x 3 and
  384 x 2 (threads x resident CTAs per SM).  Small CTAs give an SM more
  independent level chains, large ones more (bus, direction) items per barrier.
* split_lanes: the k-split cap of narrow levels (1: one lane per row; up to 32:
  a row's dot product over that many adjacent lanes).
* max_tail: the dense-tail bound of each grid's factors.  It is a property of a
  loaded grid, so tuning it loads each grid again with every candidate bound
  (Grid.clone: same record, same state) and tunes the launch knobs for each.

Every candidate runs the batch once to warm up, then `reps` times between CUDA
events; the fastest mean wins.  The batch's working set usually sits in L2 during
tuning, which ranks the candidates but is not a measurement of record.  Results
are cached per (device, grid structures and tails, directions per item, candidate
sets) in memory and, optionally, in a JSON file.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import torch

from . import rh

WIDTHS = (0, 2, 4, 8, 16, 32)
SHAPES = (128, 192, 256, 384)          # threads per CTA of the compiled shapes
CTAS_PER_SM = {128: 6, 192: 4, 256: 3, 384: 2}
SPLITS = (1, 4, 32)
TAILS = (64, 128, 256)

_memo: dict[str, dict] = {}


def _grid_sig(g) -> list:
    d = g.dims
    return [int(d.n_bus), int(d.n_branch), int(d.n_x), int(d.n_p), int(d.nnz_l), int(d.nnz_u), int(d.max_tail)]


def key(items, widths, shapes, splits, tails) -> str:
    dev = torch.cuda.get_device_name(items[0][0].device) if items else ""
    sig = {"dev": dev, "items": [_grid_sig(g) + [int(W.shape[1])] for g, W, _, _ in items],
           "widths": list(widths), "shapes": list(shapes), "splits": list(splits),
           "tails": None if tails is None else list(tails)}
    return hashlib.sha256(json.dumps(sig).encode()).hexdigest()[:24]


def launch(items, cfg: dict, stream=None):
    """rh_batch_hessvec_cfg with a tuned configuration (the grids must carry cfg's tail:
    see with_tail)."""
    rh.batch_hessvec(items, cfg["width"], stream=stream, threads=cfg["threads"], split_lanes=cfg["split_lanes"])


def with_tail(grids, max_tail: int):
    """The grids loaded with dense-tail bound max_tail (a grid that already has it is
    returned as is; the others are cloned at their state)."""
    done = {}
    for g in grids:
        if id(g) not in done:
            done[id(g)] = g if int(g.dims.max_tail) == int(max_tail) else g.clone(max_tail=max_tail)
    return [done[id(g)] for g in grids]


def _time(items, cfg, reps, stream) -> float:
    launch(items, cfg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        launch(items, cfg)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(items, widths=WIDTHS, shapes=SHAPES, splits=SPLITS, tails=None, reps: int = 3,
         cache_path: str | None = None) -> dict:
    """Tune rh_batch_hessvec_cfg for `items` ((Grid, W, HW, work) as rh.batch_hessvec takes).

    tails: None keeps every grid's own dense-tail bound; a tuple also tries each other bound
    (the items' grids are cloned with it for the measurement, then released).
    Returns {"width", "threads", "ctas_per_sm", "split_lanes", "max_tail", "ms",
    "table": every measured configuration with its ms, "cached": bool}."""
    k = key(items, widths, shapes, splits, tails)
    if k in _memo:
        return dict(_memo[k], cached=True)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if k in cache:
        _memo[k] = cache[k]
        return dict(cache[k], cached=True)
    stream = torch.cuda.current_stream()
    own_tail = sorted({int(g.dims.max_tail) for g, _, _, _ in items})
    # None: the grids as loaded (their own bounds); then every other candidate bound
    tail_list = [None] + ([int(t) for t in tails if int(t) not in own_tail] if tails is not None else [])
    table = []
    for t in tail_list:
        grids = [g for g, _, _, _ in items]
        tg = grids if t is None else with_tail(grids, t)
        titems = [(g2,) + tuple(it[1:]) for g2, it in zip(tg, items)]
        try:
            for w, th, sp in itertools.product(widths, shapes, splits):
                cfg = {"width": int(w), "threads": int(th), "split_lanes": int(sp)}
                ms = _time(titems, cfg, reps, stream)
                table.append(dict(cfg, max_tail=(own_tail[0] if len(own_tail) == 1 else None) if t is None
                                  else int(t), ms=ms))
        finally:
            for g2 in {id(g2): g2 for g2, g in zip(tg, grids) if g2 is not g}.values():
                g2.close()
    best = min(table, key=lambda r: r["ms"])
    res = {"width": best["width"], "threads": best["threads"], "ctas_per_sm": CTAS_PER_SM[best["threads"]],
           "split_lanes": best["split_lanes"], "max_tail": best["max_tail"], "ms": best["ms"], "table": table}
    _memo[k] = res
    if cache_path:
        cache[k] = res
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return dict(res, cached=False)
