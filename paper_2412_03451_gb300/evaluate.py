"""Geometry of a fitted room against its ground truth, and its plane instances.

Sec. 4.1 evaluates reconstructions with the Chamfer distance and F-score
(following AirPlanes); on the synthetic rooms the same quantities are taken
between points back-projected from depth maps: the fitted planes rendered
with the sharpest weight of Eq. 10 (lambda = 300) and the exact ground truth,
over the same views, so that only surfaces some view observes count.
  accuracy      mean distance from fitted points to the nearest ground-truth point;
  completeness  mean distance from ground-truth points to the nearest fitted point;
  Chamfer       their mean;
  F-score       harmonic mean of the fractions within 5 cm each way.
Plane instances come from the merge of Sec. 3.3 (ps_merge_planes: 25 degrees,
0.1 cm as printed, and 0.1 m), beside the same merge of the ground-truth
rectangles as the reference count.  The nearest-neighbour search runs on the
host (scipy); this is measurement, not part of the fitted path.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from . import splat as SP


def depth_points(depth: torch.Tensor, cams, views, n_pts: int, seed: int) -> np.ndarray:
    """World points of the valid pixels of depth [V, H, W] (views' cameras),
    a seeded uniform subsample of at most n_pts."""
    dev = depth.device
    V, H, W = depth.shape
    jj, ii = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float32),
                            torch.arange(W, device=dev, dtype=torch.float32), indexing="ij")
    pts = []
    for k, v in enumerate(views):
        fx, fy, cx, cy = (float(x) for x in cams.intr[v])
        Rt = torch.as_tensor(cams.w2c[v], dtype=torch.float32, device=dev)
        d = depth[k]
        ok = d > 0
        pc = torch.stack([(ii[ok] + 0.5 - cx) / fx * d[ok], (jj[ok] + 0.5 - cy) / fy * d[ok], d[ok]], 1)
        pts.append((pc - Rt[:, 3]) @ Rt[:, :3])           # R^T (p_c - t)
    P = torch.cat(pts).cpu().numpy().astype(np.float64)
    if len(P) > n_pts:
        P = P[np.random.default_rng(seed).choice(len(P), n_pts, replace=False)]
    return P


def chamfer_fscore(pred: np.ndarray, gt: np.ndarray, thresh: float = 0.05) -> dict:
    from scipy.spatial import cKDTree
    if len(pred) == 0 or len(gt) == 0:
        return {"accuracy_m": None, "completeness_m": None, "chamfer_m": None, "fscore": 0.0}
    d_pg, _ = cKDTree(gt).query(pred)
    d_gp, _ = cKDTree(pred).query(gt)
    prec = float((d_pg < thresh).mean())
    rec = float((d_gp < thresh).mean())
    f = 2 * prec * rec / (prec + rec) if prec + rec > 0 else 0.0
    return {"accuracy_m": round(float(d_pg.mean()), 5), "completeness_m": round(float(d_gp.mean()), 5),
            "chamfer_m": round(float(0.5 * (d_pg.mean() + d_gp.mean())), 5), "fscore": round(f, 4)}


def merged_groups(flat: torch.Tensor, K: int, centre, max_angle=25.0, max_offset=0.001) -> int:
    dev = flat.device
    g = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
    reps = torch.empty_like(g)
    n = torch.zeros(1, dtype=torch.int32, device=dev)
    B.ps_merge_planes(flat, K, centre, max_angle, max_offset, g, reps, n)
    return int(n.item())


def evaluate_fit(room, flat: torch.Tensor, K: int, views=None, n_pts: int = 200000,
                 tile=(16, 16), flags=0, seed: int = 0) -> dict:
    """Chamfer / F-score of the fitted planes (flat, K planes) against the room's
    ground truth over the given views (default: every 8th), plus merge counts."""
    cams = room.cams
    views = list(range(0, cams.V, 8)) if views is None else list(views)
    dev = flat.device
    n = len(views)
    w2c, intr = cams.w2c[views], cams.intr[views]
    r = SP.Renderer([cams.H] * n, [cams.W] * n, [0] * n, [0, K], tile=tile, device=dev, flags=flags)
    r.set_cameras(w2c, intr)
    r.ensure_capacity(flat, 300.0)
    r.forward(flat, 300.0, alpha=False)
    pred = r.depth.view(n, cams.H, cams.W).clone()
    gt_flat = SP.planes_to_flat(room.gt.center, room.gt.quat, room.gt.radii, dev)
    g = SP.Renderer([cams.H] * n, [cams.W] * n, [0] * n, [0, room.gt.K], tile=tile, device=dev,
                    flags=B.PS_HARD)
    g.set_cameras(w2c, intr)
    g.ensure_capacity(gt_flat, 300.0)
    g.forward(gt_flat, 300.0, alpha=False)
    gt = g.depth.view(n, cams.H, cams.W).clone()
    out = chamfer_fscore(depth_points(pred, cams, views, n_pts, seed),
                         depth_points(gt, cams, views, n_pts, seed + 1))
    centre = [float(x) / 2 for x in room.size]
    out["instances_0.1cm"] = merged_groups(flat, K, centre, 25.0, 0.001)
    out["instances_0.1m"] = merged_groups(flat, K, centre, 25.0, 0.1)
    out["gt_instances"] = merged_groups(gt_flat, room.gt.K, centre, 25.0, 0.001)
    return out
