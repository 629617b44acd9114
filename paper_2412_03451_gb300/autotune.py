"""Launch-shape autotuner of the splat kernels.

Two knobs change the speed of the kernels but not their results:
  * the tile shape (8x8, 16x16 or 32x8 pixels): small tiles give shorter tile
    lists but more binning work;
  * the warps per CTA (2, 4 or 8), i.e. the plane records a CTA stages per
    shared-memory batch (each warp stages 32 records of its tile list at a
    time): 2 and 4 give the same warps per SM in smaller or larger CTAs, 8 gives
    fewer, larger CTAs with more registers per thread.
pick_launch times one projection + binning + fused splat/loss/backward step for
each (tile, warps) pair on the caller's actual data (CUDA events, after a
warm-up step) and returns the fastest.  Results are cached per key (image sizes,
views per step, plane-count bucket) for the life of the process, and optionally
in a JSON file named by the PS_AUTOTUNE_CACHE environment variable.
"""
from __future__ import annotations

import json
import math
import os

import torch

TILES = ((16, 16), (8, 8), (32, 8))
WARPS = (2, 4, 8)
_cache: dict = {}


def _key(sizes, views, planes) -> str:
    bucket = int(math.log2(max(planes, 1)))
    return "%s|v%d|k%d" % (",".join("%dx%d" % hw for hw in sorted(set(sizes))), views, bucket)


def _label(tile, warps) -> str:
    return "%dx%d/w%d" % (tile[0], tile[1], warps)


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


def pick_launch(make_renderer, flat, gt_depth, gt_normal, lam, key, steps=3, tiles=TILES, warps=WARPS):
    """make_renderer(tile, warps) -> splat.Renderer for the caller's frame.
    Returns (best tile, best warps, {"WxH/wN": ms per step}).  flat is not
    modified."""
    if not _cache:
        _load_file()
    if key in _cache:
        e = _cache[key]
        return tuple(e["tile"]), int(e.get("warps", 0)), e["ms"]
    times = {}
    for tile in tiles:
        for nw in warps:
            r = make_renderer(tile, nw)
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
            times[_label(tile, nw)] = e0.elapsed_time(e1) / steps
            del r
    best = min(times, key=times.get)
    ts, ws = best.split("/w")
    tile = tuple(int(x) for x in ts.split("x"))
    _cache[key] = {"tile": list(tile), "warps": int(ws), "ms": times}
    _save_file()
    return tile, int(ws), times


def key_for(sizes, views, planes) -> str:
    return _key(sizes, views, planes)
