"""Ablations of Sec. 4.3 on synthetic rooms, measured as time to a mean depth
error of 2 cm (the paper's Tab. 3 measures reconstruction quality on ScanNetV2,
which is not available here; the mechanisms are the same).

Each fitted room is also scored like Sec. 4.1 (evaluate.py: Chamfer distance
and F-score at 5 cm against the ground truth over every 8th view, and the plane
instances after the merge of Sec. 3.3).

Variants (each fits every room on its own, 64 views of 640x480, 8 views per
step, Eq. 10 schedule from iteration 0):
  plain         random surface points, random orientation, radii 0.5 x the
                nearest-centre distance (the start used by the throughput runs);
  mono          the Sec. 3.1 start: points and normals of a degraded (monocular-
                like) depth/normal map, radii 0.5 x nearest-centre distance;
  sphere        the Sec. 4.3 sphere start: radii 0.05 m on the scene's bounding
                sphere, normals to its centre;
  single_radii  the mono start with one radius per axis (Sec. 4.3, PS_SINGLE_RADII);
  split         the mono start with plane splitting every 1,000 iterations
                (Sec. 3.3; threshold 0.2 on the radius gradient of the per-view
                mean loss);
  split_low     the same with the threshold lowered to 0.005 (the printed 0.2
                selects no plane on these rooms under this reading of the loss
                scale; this variant exercises the mechanism);
  gaussian      the mono start with the Gaussian weight of Eq. 5 instead of the
                rectangle weight (Sec. 3.2, Fig. 4), the radii as its scales.
"""
from __future__ import annotations

import numpy as np
import torch

from . import batch as BT
from . import evaluate as EV
from . import binding as B
from . import scenes as S
from . import starts as ST

VARIANTS = ("plain", "mono", "sphere", "single_radii", "split", "split_low", "gaussian")


def _gt_maps(ss: BT.SceneSet, i: int):
    c = ss.rooms[i].cams
    off = int(ss.gt_off[i][0])
    m = c.V * c.H * c.W
    d = ss.gt_depth[off:off + m].view(c.V, c.H, c.W).cpu().numpy()
    n = ss.gt_normal[off:off + m].view(c.V, c.H, c.W, 3).cpu().numpy()
    return d, n


def make_inits(name: str, rooms, ss_ref: BT.SceneSet, planes: int, seed0: int, device="cuda"):
    out = []
    for i, room in enumerate(rooms):
        seed = seed0 + 100 + i
        if name == "plain":
            out.append(ST.surface_start(room, planes, seed, device))
        elif name in ("mono", "single_radii", "split", "split_low", "gaussian"):
            d, n = _gt_maps(ss_ref, i)
            out.append(ST.mono_start(room, d, n, planes, seed, device))
        elif name == "sphere":
            out.append(S.sphere_init(room, planes, seed))
        else:
            raise ValueError(name)
    return out


def run(n_rooms: int = 4, planes: int = 2000, iters: int = 5000, seed0: int = 7000,
        variants=VARIANTS, device="cuda", tile=(16, 16), evaluate: bool = True) -> dict:
    rooms = [S.large_room(seed0 + i, n_rect=2000, n_views=64) for i in range(n_rooms)]
    ss_ref = BT.SceneSet(rooms, [ST.surface_start(r, planes, seed0 + 100 + i, device)
                                 for i, r in enumerate(rooms)], device=device, tile=tile)
    out = {"rooms": n_rooms, "planes": planes, "iteration_cap": iters,
           "what": "per variant: rooms fitted one by one; GPU seconds, iterations to mean depth "
                   "error <= 2 cm (None: not reached), error at the end"}
    for name in variants:
        inits = make_inits(name, rooms, ss_ref, planes, seed0, device)
        flags = {"single_radii": B.PS_SINGLE_RADII, "gaussian": B.PS_GAUSSIAN}.get(name, 0)
        ss = BT.SceneSet(rooms, inits, device=device, tile=tile, flags=flags)
        split = 1000 if name in ("split", "split_low") else 0
        tau = 0.005 if name == "split_low" else 0.2
        res = [BT.fit_until(ss, [s], max_iters=iters, split_every=split, split_tau=tau)
               for s in range(n_rooms)]
        its = [r["done_at"][0][0] if r["done_at"][0] is not None else None for r in res]
        ev = [EV.evaluate_fit(rooms[s], res[s]["params"][0], res[s]["planes"][0], flags=flags,
                              seed=seed0 + s) for s in range(n_rooms)] if evaluate else []
        out[name] = {"gpu_s": round(sum(r["gpu_ms"] for r in res) / 1e3, 3),
                     "iterations_to_2cm": its,
                     "reached": sum(i is not None for i in its),
                     "final_err_m": [round(float(r["err"][0]), 4) for r in res],
                     "planes_at_end": [r["planes"][0] for r in res]}
        if ev:
            for key in ("chamfer_m", "fscore", "instances_0.1cm", "instances_0.1m", "gt_instances"):
                out[name][key] = [e[key] for e in ev]
        del ss
        torch.cuda.empty_cache()
    return out
