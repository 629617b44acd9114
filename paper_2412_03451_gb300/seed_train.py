"""Training data, training and inference of the seed-proposal network.

Data: synthetic rooms are fitted by the splatting method itself (batched, a
fixed number of iterations); the converged planes cut every 64x64 patch of every
view into segments (the nearest converged plane of each pixel, ps_splat_ids).
The patch input is the ground-truth depth (divided by the patch's median depth,
minus 1) and camera-frame normal; up to 8 targets per patch are the largest
segments, each described in the camera frame by its centroid, the canonical
frame of its converged plane (normal towards the camera, x axis closest to the
image x axis) and its one-sided extents along that frame, depths relative to
the median depth.

Inference (propose_planes): the network runs on the patches of a few views of a
new room; seeds with confidence >= 0.5 become planes in world coordinates;
patches without a confident seed fall back to the plain initialisation (a
random surface point of the patch with random orientation).

python -m paper_2412_03451_gb300.seed_train writes the trained weights and
scores them on held-out rooms.  The committed weights came from
PS_SEED_ROOMS=2000 PS_SEED_CUT_VIEWS=4 PS_SEED_STEPS=16000 PS_SEED_EVAL_ROOMS=100
(about 35 minutes on one GB300: 29 fitting the 2,000 rooms, 2 training);
PS_SEED_EVAL_ONLY=1 scores the committed weights alone.
"""
from __future__ import annotations

import math
import os
import time

import numpy as np
import torch

from . import batch as BT
from . import binding as B
from . import scenes as S
from . import seednet as SN
from . import splat as SP

PATCH = SN.PATCH
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "seednet.npz")


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def canonical_frame(Rc: np.ndarray, centroid: np.ndarray):
    """Plane frame (columns v^x, v^y, n in camera coordinates) made canonical:
    n faces the camera, v^x is the in-plane axis closest to the image x axis."""
    vx, vy, n = Rc[:, 0], Rc[:, 1], Rc[:, 2]
    if n @ centroid > 0:
        n = -n
    cands = [vx, -vx, vy, -vy]
    ax = cands[int(np.argmax([c[0] for c in cands]))]
    ay = np.cross(n, ax)
    return np.stack([ax, ay, n], axis=1)


def patch_grid(H, W):
    return [(y, x) for y in range(0, H - PATCH + 1, PATCH) for x in range(0, W - PATCH + 1, PATCH)]


def patch_inputs(depth: np.ndarray, normal: np.ndarray, y0, x0):
    d = depth[y0:y0 + PATCH, x0:x0 + PATCH]
    valid = d > 0
    if valid.sum() < PATCH * PATCH // 4:
        return None, None
    z_ref = float(np.median(d[valid]))
    x = np.zeros((PATCH, PATCH, 4), np.float32)
    x[..., 0] = np.where(valid, d / z_ref - 1.0, 0.0)
    x[..., 1:] = np.where(valid[..., None], normal[y0:y0 + PATCH, x0:x0 + PATCH], 0.0)
    return x, z_ref


def patch_targets(ids, depth, intr, w2c, planes_q, y0, x0, z_ref, min_pix=64):
    """Targets [8, 12] of one patch from its plane-index map."""
    fx, fy, cx, cy = (float(v) for v in intr)
    R = w2c[:, :3].astype(np.float64)
    t = np.zeros((SN.SLOTS, 12), np.float32)
    pid = ids[y0:y0 + PATCH, x0:x0 + PATCH]
    d = depth[y0:y0 + PATCH, x0:x0 + PATCH]
    ok = (pid >= 0) & (d > 0)
    if not ok.any():
        return t
    u, c = np.unique(pid[ok], return_counts=True)
    order = np.argsort(-c)
    jj, ii = np.mgrid[0:PATCH, 0:PATCH]
    slot = 0
    for k in order:
        if c[k] < min_pix or slot >= SN.SLOTS:
            break
        m = ok & (pid == u[k])
        z = d[m].astype(np.float64)
        X = ((ii[m] + x0 + 0.5 - cx) / fx) * z
        Y = ((jj[m] + y0 + 0.5 - cy) / fy) * z
        P = np.stack([X, Y, z], axis=1)
        cen = P.mean(axis=0)
        F = canonical_frame(R @ _rot(planes_q[u[k]].astype(np.float64)), cen)
        a = (P - cen) @ F[:, 0]
        b = (P - cen) @ F[:, 1]
        half_px = 0.5 * cen[2] / fx
        ext = np.array([a.max(), -a.min(), b.max(), -b.min()]) + half_px
        ext = np.maximum(ext, 0.005 * z_ref)
        un = ((fx * cen[0] / cen[2] + cx) - (x0 + PATCH / 2)) / (PATCH / 2)
        vn = ((fy * cen[1] / cen[2] + cy) - (y0 + PATCH / 2)) / (PATCH / 2)
        t[slot, 0] = 1.0
        t[slot, 1:4] = (un, vn, math.log(cen[2] / z_ref))
        t[slot, 4:8] = S.quat_from_frame(F[:, 0], F[:, 1], F[:, 2])
        t[slot, 8:12] = np.log(ext / z_ref)
        slot += 1
    return t


def make_dataset(n_rooms=32, seed0=5000, views=16, iters=1500, device="cuda", log=print, chunk=48,
                 cut_views=None):
    """Fits n_rooms rooms with the method (batched, chunk rooms at a time) and
    cuts their views into patches (all views, or cut_views of them spread over
    the trajectory: more rooms for the same number of patches).  Returns
    (X [N, 64, 64, 4] float16, T [N, 8, 12] float32)."""
    t0 = time.time()
    rng = np.random.default_rng(seed0)
    Ks = [int(rng.integers(500, 3001)) for _ in range(n_rooms)]
    Xs, Ts = [], []
    for c0 in range(0, n_rooms, chunk):
        idx = list(range(c0, min(c0 + chunk, n_rooms)))
        _cut_patches(idx, Ks, seed0, views, iters, device, Xs, Ts, cut_views)
        log("seed data: %d of %d rooms, %d patches, %.1f s" % (idx[-1] + 1, n_rooms, len(Xs),
                                                             time.time() - t0))
    X, T = np.stack(Xs), np.stack(Ts)
    log("seed data: %d patches, %.2f targets per patch, %.1f s" %
        (len(X), float(T[..., 0].sum(1).mean()), time.time() - t0))
    return X, T


def _cut_patches(idx, Ks, seed0, views, iters, device, Xs, Ts, cut_views=None):
    rooms, inits = [], []
    for i in idx:
        room = S.large_room(seed0 + i, n_rect=2000, n_views=views)
        rooms.append(room)
        inits.append(S.surface_init_nn(room, Ks[i], seed0 + 10000 + i))
    ss = BT.SceneSet(rooms, inits, device=device)
    res = BT.fit_until(ss, list(range(len(rooms))), threshold=0.0, max_iters=iters)
    for i, room in enumerate(rooms):
        c = room.cams
        flat = res["params"][i]
        K = ss.K[i]
        r = SP.Renderer([c.H] * c.V, [c.W] * c.V, [0] * c.V, [0, K], device=device)
        r.set_cameras(c.w2c, c.intr)
        r.ensure_capacity(flat, 300.0, flags=B.PS_HARD)
        ids, _ = r.plane_ids(flat)
        ids = ids.cpu().numpy().reshape(c.V, c.H, c.W)
        q = flat[3 * K:7 * K].view(K, 4).cpu().numpy()
        off = int(ss.gt_off[i][0])
        n = c.V * c.H * c.W
        gd = ss.gt_depth[off:off + n].cpu().numpy().reshape(c.V, c.H, c.W)
        gn = ss.gt_normal[off:off + n].cpu().numpy().reshape(c.V, c.H, c.W, 3)
        step = max(1, c.V // cut_views) if cut_views else 1
        for v in range(0, c.V, step):
            for (y0, x0) in patch_grid(c.H, c.W):
                x, z_ref = patch_inputs(gd[v], gn[v], y0, x0)
                if x is None:
                    continue
                Xs.append(x.astype(np.float16))
                Ts.append(patch_targets(ids[v], gd[v], c.intr[v], c.w2c[v], q, y0, x0, z_ref))
        del r
    del ss
    torch.cuda.empty_cache()


def train(X, T, steps=3000, batch=256, lr=1e-3, seed=0, device="cuda", log=print):
    """Trains a SeedNet on (X, T) with Adam on the GPU; returns the net and the
    loss history (sums of the four terms per batch, every 100 steps)."""
    net = SN.SeedNet(device=device, seed=seed)
    net.sync_weights()
    Xd = torch.from_numpy(X).to(device).bfloat16()
    Td = torch.from_numpy(T).to(device)
    N = len(X)
    g = torch.Generator(device=device).manual_seed(seed)
    hist = []
    t0 = time.time()
    for it in range(steps):
        idx = torch.randint(0, N, (batch,), device=device, generator=g)
        net.forward(Xd[idx].contiguous())
        net.grad.zero_()
        sums = net.loss_backward(Td[idx].contiguous())
        net.adam(lr=lr if it < 0.8 * steps else lr * 0.2)
        if it % 100 == 0 or it == steps - 1:
            hist.append((it, [round(float(v) / batch, 4) for v in sums.cpu().tolist()]))
    torch.cuda.synchronize()
    log("seed net: %d steps of %d patches in %.1f s, loss terms per patch %s -> %s" %
        (steps, batch, time.time() - t0, hist[0][1], hist[-1][1]))
    return net, hist


def _rot_batch(q):
    """Rotation matrices [n, 3, 3] of quaternions [n, 4] (w, x, y, z), normalised."""
    q = q / (np.linalg.norm(q, axis=1, keepdims=True) + 1e-12)
    w, x, y, z = q.T
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)],
                    axis=1)


def _quat_batch(R):
    """Unit quaternions [n, 4] of rotation matrices [n, 3, 3] (Shepperd's method)."""
    n = len(R)
    q = np.zeros((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    cands = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], axis=1)
    k = np.argmax(cands, axis=1)
    for case in range(4):
        m = k == case
        if not m.any():
            continue
        Rm = R[m]
        if case == 0:
            s_ = np.sqrt(tr[m] + 1.0) * 2
            q[m] = np.stack([0.25 * s_, (Rm[:, 2, 1] - Rm[:, 1, 2]) / s_, (Rm[:, 0, 2] - Rm[:, 2, 0]) / s_,
                             (Rm[:, 1, 0] - Rm[:, 0, 1]) / s_], 1)
        elif case == 1:
            s_ = np.sqrt(1.0 + Rm[:, 0, 0] - Rm[:, 1, 1] - Rm[:, 2, 2]) * 2
            q[m] = np.stack([(Rm[:, 2, 1] - Rm[:, 1, 2]) / s_, 0.25 * s_, (Rm[:, 0, 1] + Rm[:, 1, 0]) / s_,
                             (Rm[:, 0, 2] + Rm[:, 2, 0]) / s_], 1)
        elif case == 2:
            s_ = np.sqrt(1.0 + Rm[:, 1, 1] - Rm[:, 0, 0] - Rm[:, 2, 2]) * 2
            q[m] = np.stack([(Rm[:, 0, 2] - Rm[:, 2, 0]) / s_, (Rm[:, 0, 1] + Rm[:, 1, 0]) / s_, 0.25 * s_,
                             (Rm[:, 1, 2] + Rm[:, 2, 1]) / s_], 1)
        else:
            s_ = np.sqrt(1.0 + Rm[:, 2, 2] - Rm[:, 0, 0] - Rm[:, 1, 1]) * 2
            q[m] = np.stack([(Rm[:, 1, 0] - Rm[:, 0, 1]) / s_, (Rm[:, 0, 2] + Rm[:, 2, 0]) / s_,
                             (Rm[:, 1, 2] + Rm[:, 2, 1]) / s_, 0.25 * s_], 1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def patches_gpu(depth: torch.Tensor, normal: torch.Tensor, views):
    """Network inputs of the full 64x64 patches of the given views, on the GPU.
    depth [V, H, W], normal [V, H, W, 3] (device tensors).  Returns
    (X [n, 64, 64, 4] bf16, meta [n, 4] numpy: view, y0, x0, z_ref); patches
    with fewer than a quarter valid pixels are dropped."""
    V, H, W = depth.shape
    ny, nx = H // PATCH, W // PATCH
    vi = torch.as_tensor(list(views), device=depth.device)
    d = depth[vi, :ny * PATCH, :nx * PATCH].reshape(len(vi), ny, PATCH, nx, PATCH)
    d = d.permute(0, 1, 3, 2, 4).reshape(-1, PATCH, PATCH)
    nrm = normal[vi, :ny * PATCH, :nx * PATCH].reshape(len(vi), ny, PATCH, nx, PATCH, 3)
    nrm = nrm.permute(0, 1, 3, 2, 4, 5).reshape(-1, PATCH, PATCH, 3)
    valid = d > 0
    ok = valid.reshape(len(d), -1).sum(1) >= PATCH * PATCH // 4
    dn = torch.where(valid, d, torch.full_like(d, float("nan"))).reshape(len(d), -1)
    z_ref = torch.nanmedian(dn, dim=1).values
    x = torch.zeros((len(d), PATCH, PATCH, 4), device=depth.device)
    x[..., 0] = torch.where(valid, d / z_ref[:, None, None] - 1.0, torch.zeros_like(d))
    x[..., 1:] = torch.where(valid[..., None], nrm, torch.zeros_like(nrm))
    vv = vi.repeat_interleave(ny * nx)
    yy = torch.arange(ny, device=depth.device).repeat_interleave(nx).repeat(len(vi)) * PATCH
    xx = torch.arange(nx, device=depth.device).repeat(ny * len(vi)) * PATCH
    meta = torch.stack([vv.float(), yy.float(), xx.float(), z_ref], 1)[ok]
    return x[ok].bfloat16(), meta.cpu().numpy().astype(np.float64)


LEARNED_LAM_OFFSET = 1000   # Eq. 10 start of a fit from network seeds (lambda = 20)


def propose_planes(net: SN.SeedNet, room, depth, normal, views, conf=0.5, seed=0, max_planes=None,
                   cell=0.4, radius_scale=0.7):
    """Planes (world coordinates) proposed by the network from the depth/normal
    maps of the given views; patches without a confident seed get one plain
    seed (random surface point, random orientation).  Seeds seen from several
    views are deduplicated: one seed (the most confident) per 3D cell of size
    `cell` and dominant normal direction.  depth [V, H, W], normal [V, H, W, 3]
    numpy.  Returns (Planes, n_learned, n_fallback)."""
    rng = np.random.default_rng(seed)
    c = room.cams
    X, meta = patches_gpu(depth, normal, views)
    pad = (-len(X)) % 64
    if pad:
        X = torch.cat([X, torch.zeros((pad,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)])
    out = net.forward(X.contiguous()).cpu().numpy()[:len(meta)]
    depth = depth.cpu().numpy()
    O = out.reshape(len(meta), SN.SLOTS, 12).astype(np.float64)
    pconf = 1.0 / (1.0 + np.exp(-O[..., 11]))
    keep = pconf >= conf                                  # [n_patch, slots]
    pi, si = np.nonzero(keep)
    S_ = O[pi, si]
    v = meta[pi, 0].astype(int)
    y0, x0, z_ref = meta[pi, 1], meta[pi, 2], meta[pi, 3]
    fx, fy, cx, cy = (c.intr[v, k].astype(np.float64) for k in range(4))
    Rv = c.w2c[v, :, :3].astype(np.float64)
    tv = c.w2c[v, :, 3].astype(np.float64)
    z = z_ref * np.exp(S_[:, 2])
    upx = x0 + PATCH / 2 + S_[:, 0] * PATCH / 2
    vpx = y0 + PATCH / 2 + S_[:, 1] * PATCH / 2
    pc = np.stack([(upx - cx) / fx * z, (vpx - cy) / fy * z, z], axis=1)
    Fw = np.einsum("nji,njk->nik", Rv, _rot_batch(S_[:, 3:7]))      # R^T F_cam
    cen = np.einsum("nji,nj->ni", Rv, pc - tv)
    rad = radius_scale * z_ref[:, None] * np.exp(np.clip(S_[:, 7:11], -6, 2))
    score = pconf[pi, si]
    # deduplicate across views: one seed per (cell, dominant normal axis and sign)
    n = Fw[:, :, 2]
    ax = np.argmax(np.abs(n), axis=1)
    sg = (n[np.arange(len(n)), ax] > 0).astype(int)
    key = np.concatenate([np.floor(cen / cell).astype(np.int64), (ax * 2 + sg)[:, None]], axis=1)
    order = np.lexsort((-score,) + tuple(key.T[::-1]))
    kk = key[order]
    first = np.ones(len(kk), bool)
    first[1:] = np.any(kk[1:] != kk[:-1], axis=1)
    sel = order[first]
    cen, Fw, rad, score = cen[sel], Fw[sel], rad[sel], score[sel]
    quat = _quat_batch(Fw)
    # fallback: patches without a confident seed get one plain seed
    fb = np.nonzero(~keep.any(axis=1))[0]
    fc, fq, fr = [], [], []
    for p_ in fb:
        vv, yy, xx, zr = int(meta[p_, 0]), int(meta[p_, 1]), int(meta[p_, 2]), meta[p_, 3]
        d = depth[vv, yy:yy + PATCH, xx:xx + PATCH]
        jj, ii = np.nonzero(d > 0)
        k = rng.integers(0, len(jj))
        zz = float(d[jj[k], ii[k]])
        fx_, fy_, cx_, cy_ = (float(t) for t in c.intr[vv])
        pcf = np.array([(xx + ii[k] + 0.5 - cx_) / fx_ * zz, (yy + jj[k] + 0.5 - cy_) / fy_ * zz, zz])
        Rt = c.w2c[vv].astype(np.float64)
        fc.append(Rt[:, :3].T @ (pcf - Rt[:, 3]))
        fq.append(S.random_quats(rng, 1)[0])
        fr.append(np.full(4, 0.25 * PATCH * zr / fx_))
    n_learned = len(cen)
    if max_planes is not None and n_learned + len(fb) > max_planes and n_learned > 0:
        take = max(max_planes - len(fb), 0)
        if take < n_learned:
            idx = np.argsort(-score)[:take]
            cen, quat, rad = cen[idx], quat[idx], rad[idx]
            n_learned = take
    if fb.size:
        cen = np.concatenate([cen, np.asarray(fc)])
        quat = np.concatenate([quat, np.asarray(fq)])
        rad = np.concatenate([rad, np.asarray(fr)])
    P = S.Planes(cen.astype(np.float32), quat.astype(np.float32), rad.astype(np.float32))
    return P, n_learned, len(fb)


def evaluate(net, n_rooms=8, seed0=9000, planes=3000, iters=5000, device="cuda", log=print,
             variants=None):
    """Time to mean depth error <= 2 cm on held-out rooms (64 views at 640x480).
    plain: random surface points and orientations, radii half the nearest-neighbour
    spacing, fitted room by room.  learned: network proposals from all 64 views,
    deduplicated and capped at `planes`, fitted room by room and all rooms
    batched; times include the network's inference.  Each variant is a dict of
    propose_planes options plus lam_offset (Eq. 10 start)."""
    variants = variants or [dict(name="learned", lam_offset=LEARNED_LAM_OFFSET)]
    rooms = [S.large_room(seed0 + i, n_rect=2000, n_views=64) for i in range(n_rooms)]
    plain = [S.surface_init_nn(room, planes, seed0 + 100 + i) for i, room in enumerate(rooms)]
    ss_p = BT.SceneSet(rooms, plain, device=device)
    pl = [BT.fit_until(ss_p, [s], max_iters=iters) for s in range(n_rooms)]
    res = {"rooms": n_rooms, "planes_plain": planes,
           "plain_one_by_one_s": round(sum(p["gpu_ms"] for p in pl) / 1e3, 3),
           "reached_plain": sum(p["done_at"][0] is not None for p in pl),
           "iterations_plain": [p["done_at"][0][0] if p["done_at"][0] else None for p in pl],
           "variants": []}
    # warm the network's kernels once (first-call set-up is not inference)
    c0 = rooms[0].cams
    propose_planes(net, rooms[0], ss_p.gt_depth[:c0.H * c0.W].view(1, c0.H, c0.W),
                   ss_p.gt_normal[:c0.H * c0.W].view(1, c0.H, c0.W, 3), [0], seed=seed0, max_planes=100)
    torch.cuda.synchronize()
    for var in variants:
        opts = {k: v for k, v in var.items() if k not in ("name", "lam_offset", "net")}
        learned, infer_ms, n_l, n_f = [], 0.0, 0, 0
        for i, room in enumerate(rooms):
            c = room.cams
            off = int(ss_p.gt_off[i][0])
            n = c.V * c.H * c.W
            gd = ss_p.gt_depth[off:off + n].view(c.V, c.H, c.W)
            gn = ss_p.gt_normal[off:off + n].view(c.V, c.H, c.W, 3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P, nl, nf = propose_planes(var.get("net", net), room, gd, gn, range(c.V), seed=seed0 + 200 + i,
                                       max_planes=planes, **opts)
            e1.record()
            torch.cuda.synchronize()
            infer_ms += e0.elapsed_time(e1)
            learned.append(P)
            n_l += nl
            n_f += nf
        ss_l = BT.SceneSet(rooms, learned, device=device)
        lo = var.get("lam_offset", 0)
        ll = [BT.fit_until(ss_l, [s], max_iters=iters, lam_offset=lo) for s in range(n_rooms)]
        lb = BT.fit_until(ss_l, list(range(n_rooms)), max_iters=iters, lam_offset=lo)
        r = {"name": var.get("name"), "options": {k: v for k, v in var.items() if k not in ("name", "net")},
             "planes_mean": round(float(np.mean([p.K for p in learned])), 1),
             "learned_seeds": n_l, "fallback_seeds": n_f, "inference_s": round(infer_ms / 1e3, 4),
             "one_by_one_s": round(sum(p["gpu_ms"] for p in ll) / 1e3 + infer_ms / 1e3, 3),
             "batched_s": round(lb["gpu_ms"] / 1e3 + infer_ms / 1e3, 3),
             "reached": sum(p["done_at"][0] is not None for p in ll),
             "reached_batched": sum(d is not None for d in lb["done_at"]),
             "iterations": [p["done_at"][0][0] if p["done_at"][0] else None for p in ll]}
        r["speedup_batched_vs_plain"] = round(res["plain_one_by_one_s"] / r["batched_s"], 3)
        res["variants"].append(r)
        log("seed eval %s: %s" % (var.get("name"), r))
    return res


def save(net: SN.SeedNet, path=WEIGHTS, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=net.params.cpu().numpy(), **(meta or {}))


def load(device="cuda", path=WEIGHTS):
    if not os.path.exists(path):
        return None
    z = np.load(path)
    net = SN.SeedNet(device=device, params=z["params"])
    net.sync_weights()
    return net


if __name__ == "__main__":
    import json
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2412_03451_gb300 import _build
    _build.build()
    n_rooms = int(os.environ.get("PS_SEED_ROOMS", "32"))
    out = os.environ.get("PS_SEED_OUT", WEIGHTS)
    previous = load()        # the weights in place before this run, if any
    if os.environ.get("PS_SEED_EVAL_ONLY", "0") == "1":
        net = previous
    else:
        cut = int(os.environ.get("PS_SEED_CUT_VIEWS", "0")) or None
        X, T = make_dataset(n_rooms=n_rooms, cut_views=cut)
        net, hist = train(X, T, steps=int(os.environ.get("PS_SEED_STEPS", "3000")))
        save(net, path=out, meta={"history": json.dumps(hist), "rooms": n_rooms, "patches": len(X)})
        print(json.dumps({"patches": len(X), "history": hist[-3:]}), flush=True)
    if os.environ.get("PS_SEED_EVAL", "1") == "1":
        variants = json.loads(os.environ.get("PS_SEED_VARIANTS", "null"))
        if variants is None:
            variants = [dict(name="learned", lam_offset=LEARNED_LAM_OFFSET)]
            if previous is not None and previous is not net and os.environ.get("PS_SEED_COMPARE", "0") == "1":
                variants.append(dict(name="previous weights", lam_offset=LEARNED_LAM_OFFSET, net=previous))
        ev = evaluate(net, n_rooms=int(os.environ.get("PS_SEED_EVAL_ROOMS", "8")), variants=variants)
        print(json.dumps(ev), flush=True)
