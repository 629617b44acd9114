"""Plane splitting (Sec. 3.3 "Plane Splitting", App. A.2) and plane merging
(Sec. 3.3 "Plane Merge") in FP64.

TEST INFRASTRUCTURE ONLY: imported by tests; shares no code with the CUDA
path.

The paper: every 1,000 iterations, a plane whose average radius gradient on
the X axis (r^x+ and r^x-) exceeds 0.2 is split along its Y axis, and one whose
average radius gradient on the Y axis exceeds 0.2 is split along its X axis.
Readings used here (the paper gives no more):
  * "average radius gradient on the X axis" = the mean over the interval's
    iterations of (|dL/dr^x+| + |dL/dr^x-|) / 2, with L the loss of the
    iteration's views, each view's Eq. 14 taken as a per-pixel mean (the
    caller's scale: views per step / supervised pixels of the step's views);
  * "split along the Y axis" = cut along the line through the centre parallel
    to v^y: a +X half covering [0, r^x+] and a -X half covering [-r^x-, 0] of
    the plane's X range, each with both X radii equal to half its width, the Y
    radii and the rotation unchanged;
  * if both axes exceed the threshold, the axis with the larger gradient is
    split (ties: X); a plane is split at most once per round;
  * the +half keeps the parent's slot, the -halves follow the scene's planes
    in parent order; Adam moments of both halves restart at zero.
"""
from __future__ import annotations

import math

import numpy as np


def rotation(q: np.ndarray) -> np.ndarray:
    """R(q / |q|) for quaternions [n, 4] in (w, x, y, z) order (Eq. 2-3);
    columns are v^x, v^y, n."""
    q = np.asarray(q, np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):    # zero rows give NaN axes
        q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((len(q), 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def radii_grad_accum(acc: np.ndarray, g_radii: np.ndarray, scale) -> np.ndarray:
    """acc [P, 2] plus this step's per-axis mean absolute radius gradient times
    scale (a number or a per-plane array)."""
    g = np.abs(np.asarray(g_radii, np.float64))
    s = np.broadcast_to(np.asarray(scale, np.float64), (len(g),))
    out = np.array(acc, np.float64)
    out[:, 0] += s * 0.5 * (g[:, 0] + g[:, 1])
    out[:, 1] += s * 0.5 * (g[:, 2] + g[:, 3])
    return out


def split_kind(acc: np.ndarray, quat: np.ndarray, n_iter: int, tau: float) -> np.ndarray:
    """Per plane 0 (keep), 1 (X gradient: halves along v^x) or 2 (halves along v^y)."""
    q = np.asarray(quat, np.float64)
    nq = (q * q).sum(1)
    ok = np.isfinite(nq) & (nq > 0)
    g = np.asarray(acc, np.float64) / n_iter
    gx, gy = g[:, 0], g[:, 1]
    kind = np.where((gx > tau) | (gy > tau), np.where(gx >= gy, 1, 2), 0)
    return np.where(ok, kind, 0)


def split_planes(center, quat, radii, plane_ptr, acc, n_iter, tau, m=None, v=None):
    """Returns dict(center, quat, radii, plane_ptr, split_rank, count, m, v) of
    the new plane set (moments in the flat [center | quat | radii] layout)."""
    center = np.asarray(center, np.float64)
    quat = np.asarray(quat, np.float64)
    radii = np.asarray(radii, np.float64)
    plane_ptr = np.asarray(plane_ptr, np.int64)
    P = len(center)
    kind = split_kind(acc, quat, n_iter, tau) if P else np.zeros(0, int)
    flags = (kind != 0).astype(np.int64)
    rank = np.concatenate([[0], np.cumsum(flags)])
    cs, qs, rs, keep_mask = [], [], [], []
    new_ptr = [0]
    R = rotation(quat) if P else np.zeros((0, 3, 3))
    for s in range(len(plane_ptr) - 1):
        a, b = int(plane_ptr[s]), int(plane_ptr[s + 1])
        tail_c, tail_q, tail_r = [], [], []
        for i in range(a, b):
            if kind[i] == 0:
                cs.append(center[i]); qs.append(quat[i]); rs.append(radii[i]); keep_mask.append(i)
                continue
            axis = R[i][:, 0] if kind[i] == 1 else R[i][:, 1]
            o = 0 if kind[i] == 1 else 2
            rp, rm = radii[i, o], radii[i, o + 1]
            ra, rb = radii[i].copy(), radii[i].copy()
            ra[o] = ra[o + 1] = rp / 2
            rb[o] = rb[o + 1] = rm / 2
            cs.append(center[i] + rp / 2 * axis); qs.append(quat[i]); rs.append(ra); keep_mask.append(-1)
            tail_c.append(center[i] - rm / 2 * axis); tail_q.append(quat[i]); tail_r.append(rb)
        cs += tail_c; qs += tail_q; rs += tail_r
        keep_mask += [-1] * len(tail_c)
        new_ptr.append(len(cs))
    Pn = len(cs)
    out = {"center": np.array(cs).reshape(Pn, 3), "quat": np.array(qs).reshape(Pn, 4),
           "radii": np.array(rs).reshape(Pn, 4), "plane_ptr": np.array(new_ptr),
           "split_rank": rank, "count": Pn, "kind": kind}
    for name, mom in (("m", m), ("v", v)):
        if mom is None:
            out[name] = None
            continue
        mom = np.asarray(mom, np.float64)
        mc, mq, mr = mom[:3 * P].reshape(P, 3), mom[3 * P:7 * P].reshape(P, 4), mom[7 * P:].reshape(P, 4)
        nc, nq, nr = np.zeros((Pn, 3)), np.zeros((Pn, 4)), np.zeros((Pn, 4))
        for j, i in enumerate(keep_mask):
            if i >= 0:
                nc[j], nq[j], nr[j] = mc[i], mq[i], mr[i]
        out[name] = np.concatenate([nc.ravel(), nq.ravel(), nr.ravel()])
    return out


def merge_planes(center, quat, radii, scene_center, max_angle_deg=25.0, max_offset=0.001):
    """Plane merge (Sec. 3.3 "Plane Merge") read as a greedy grouping: planes by
    decreasing area (ties: lower index), each joining the first group whose
    first plane's normal is within max_angle_deg up to sign and whose offset
    (distance from scene_center along the normal oriented like the group's) is
    within max_offset.  Returns (group_of [P], first plane of each group)."""
    c = np.asarray(center, np.float64)
    r = np.asarray(radii, np.float64)
    q = np.asarray(quat, np.float64)
    P = len(c)
    area = (r[:, 0] + r[:, 1]) * (r[:, 2] + r[:, 3])
    area = np.where(area > 0, area, 0.0)
    order = sorted(range(P), key=lambda i: (-area[i], i))
    nq = (q * q).sum(1)
    R = rotation(q)
    cos_max = math.cos(math.radians(max_angle_deg))
    group_of = np.full(P, -1, np.int64)
    reps, rep_n, rep_o = [], [], []
    for i in order:
        if not (np.isfinite(nq[i]) and nq[i] > 0):
            continue
        n = R[i][:, 2]
        off = float(n @ (c[i] - np.asarray(scene_center, np.float64)))
        for g, (m, o) in enumerate(zip(rep_n, rep_o)):
            d = float(n @ m)
            s = 1.0 if d >= 0 else -1.0
            if abs(d) >= cos_max and abs(s * off - o) < max_offset:
                group_of[i] = g
                break
        else:
            group_of[i] = len(reps)
            reps.append(i); rep_n.append(n); rep_o.append(off)
    return group_of, np.asarray(reps, np.int64)
