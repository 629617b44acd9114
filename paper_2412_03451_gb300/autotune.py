"""Tile-shape autotuner.

The splat kernels take 8x8, 16x16 or 32x8 pixel tiles.  Small tiles give
shorter tile lists but more binning work; the best shape depends on the image
sizes, the plane count and the depth complexity.  pick_tile times one
projection + binning + fused splat/loss/backward step for each candidate on
the caller's actual data (CUDA events, after a warm-up step) and returns the
fastest.  Results are cached per key (image sizes, views per step, plane-count
bucket) for the life of the process, and optionally in a JSON file named by
the PS_AUTOTUNE_CACHE environment variable.
"""
from __future__ import annotations

import json
import math
import os

import torch

CANDIDATES = ((16, 16), (8, 8), (32, 8))
_cache: dict = {}


def _key(sizes, views, planes) -> str:
    bucket = int(math.log2(max(planes, 1)))
    return "%s|v%d|k%d" % (",".join("%dx%d" % hw for hw in sorted(set(sizes))), views, bucket)


def _load_file():
    path = os.environ.get("PS_AUTOTUNE_CACHE")
    if path and os.path.exists(path):
        try:
            _cache.update(json.load(open(path)))
        except (OSError, ValueError):
            pass


def _save_file():
    path = os.environ.get("PS_AUTOTUNE_CACHE")
    if path:
        try:
            json.dump(_cache, open(path, "w"), indent=1)
        except OSError:
            pass


def pick_tile(make_renderer, flat, gt_depth, gt_normal, lam, key, steps=3, candidates=CANDIDATES):
    """make_renderer(tile) -> splat.Renderer for the caller's frame.  Returns
    (best tile, {tile: ms per step}).  flat is not modified."""
    if not _cache:
        _load_file()
    if key in _cache:
        t = tuple(_cache[key]["tile"])
        return t, _cache[key]["ms"]
    times = {}
    for tile in candidates:
        r = make_renderer(tile)
        r.ensure_capacity(flat, lam, headroom=1.6)
        g = torch.zeros_like(flat)
        r.project_bin(flat, lam)
        r.fused(flat, g, gt_depth, gt_normal)          # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r.project_bin(flat, lam)
            g.zero_()
            r.fused(flat, g, gt_depth, gt_normal)
        e1.record()
        torch.cuda.synchronize()
        times["%dx%d" % tile] = e0.elapsed_time(e1) / steps
        del r
    best = min(times, key=times.get)
    tile = tuple(int(x) for x in best.split("x"))
    _cache[key] = {"tile": list(tile), "ms": times}
    _save_file()
    return tile, times


def key_for(sizes, views, planes) -> str:
    return _key(sizes, views, planes)
