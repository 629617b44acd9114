"""Batched fitting of many scenes in one launch per step.

All scenes' planes live in one flat parameter buffer (CSR ranges per scene),
all scenes' ground-truth maps stay resident in HBM, and every step renders a
fixed number of views of every scene -- scenes of uneven plane counts, view
counts and resolutions -- in one persistent launch of each kernel, captured
as a CUDA graph per camera batch.  Each scene's depth error (mean |D - D*| over
its supervised pixels) comes from the fused kernel's per-view loss sums, so
checking convergence costs one small device-to-host copy per rotation.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import binding as B
from . import splat as SP


class SceneSet:
    """Scenes (rooms with initial planes), their resident ground truth and the
    per-step camera batches (views_per_step views of each scene per step)."""

    def __init__(self, rooms, inits, device="cuda", tile=(16, 16), views_per_step=8, flags=0, warps=0):
        self.rooms, self.inits = rooms, inits
        self.device = torch.device(device)
        self.tile = tile
        self.warps = int(warps)       # warps per CTA of the splat kernels (0: the library default)
        self.flags = int(flags)       # ps_settings flags of the fit (PS_SINGLE_RADII, ...)
        self.S = len(rooms)
        self.vps = views_per_step
        self.K = [p.K for p in inits]
        self.plane_ptr = np.concatenate([[0], np.cumsum(self.K)]).astype(np.int32)
        # resident ground truth of every view of every scene (library hard-rectangle mode)
        gd, gn, self.gt_off = [], [], []
        off = 0
        for room in rooms:
            c = room.cams
            r = SP.Renderer([c.H] * c.V, [c.W] * c.V, [0] * c.V, [0, room.gt.K], tile=tile,
                            device=device, flags=B.PS_HARD)
            r.set_cameras(c.w2c, c.intr)
            f = SP.planes_to_flat(room.gt.center, room.gt.quat, room.gt.radii, device)
            r.ensure_capacity(f, 300.0)
            r.forward(f, 300.0)
            gd.append(r.depth.clone())
            gn.append(r.normal.clone())
            self.gt_off.append(off + np.arange(c.V, dtype=np.int64) * c.H * c.W)
            off += c.V * c.H * c.W
            del r
        self.gt_depth = torch.cat(gd)
        self.gt_normal = torch.cat(gn)
        # supervised pixels (ground-truth depth > 0) of every view of every scene
        self.sup = [(d.view(room.cams.V, -1) > 0).sum(1).cpu().numpy()
                    for d, room in zip(gd, rooms)]
        self.n_batches = max(int(math.ceil(room.cams.V / self.vps)) for room in rooms)

    def batch_views(self, b):
        """View indices of every scene in batch b: (b * vps + j) mod V_s."""
        return [[(b * self.vps + j) % room.cams.V for j in range(self.vps)] for room in self.rooms]

    def flat_init(self):
        c = np.concatenate([p.center for p in self.inits])
        q = np.concatenate([p.quat for p in self.inits])
        r = np.concatenate([p.radii for p in self.inits])
        return SP.planes_to_flat(c, q, r, self.device)

    def split_scales(self, scenes, Ks):
        """Per camera batch, the per-plane factor [sum Ks] (device) that turns the
        summed loss of a step into a sum of per-view pixel means over the step's
        views of the plane's scene (views_per_step / supervised pixels of those
        views): the loss one view contributes when each iteration fits one view."""
        out = []
        for b in range(self.n_batches):
            vi = self.batch_views(b)
            per = [self.vps / max(int(self.sup[s][vi[s]].sum()), 1) for s in scenes]
            out.append(torch.tensor(np.repeat(per, Ks), dtype=torch.float32, device=self.device))
        return out

    def renderer(self, scenes=None, M=30, capacity=None, Ks=None):
        """A renderer for the step frame of the given scenes (all by default),
        with every camera batch planned on the device.  Ks overrides the scenes'
        plane counts (after splitting)."""
        scenes = list(range(self.S)) if scenes is None else list(scenes)
        H, W, sov = [], [], []
        for i, s in enumerate(scenes):
            c = self.rooms[s].cams
            H += [c.H] * self.vps
            W += [c.W] * self.vps
            sov += [i] * self.vps
        K = [self.K[s] for s in scenes] if Ks is None else list(Ks)
        pptr = np.concatenate([[0], np.cumsum(K)]).astype(np.int32)
        r = SP.Renderer(H, W, sov, pptr, tile=self.tile, M=M, capacity=capacity,
                        device=self.device, flags=self.flags, warps=self.warps)
        w2cs, intrs, gts = [], [], []
        for b in range(self.n_batches):
            vi = self.batch_views(b)
            w2cs.append(np.concatenate([self.rooms[s].cams.w2c[vi[s]] for s in scenes]))
            intrs.append(np.concatenate([self.rooms[s].cams.intr[vi[s]] for s in scenes]))
            gts.append(np.concatenate([self.gt_off[s][vi[s]] for s in scenes]))
        r.preplan(w2cs, intrs, gts)
        r.scenes = scenes
        return r

    def flat_for(self, scenes):
        c = np.concatenate([self.inits[s].center for s in scenes])
        q = np.concatenate([self.inits[s].quat for s in scenes])
        r = np.concatenate([self.inits[s].radii for s in scenes])
        return SP.planes_to_flat(c, q, r, self.device)


def split_flat(flat: torch.Tensor, Ks):
    """Per-scene flat buffers from a batched one ([c | q | r] over all planes)."""
    P = int(sum(Ks))
    c, q, r = flat[:3 * P].view(P, 3), flat[3 * P:7 * P].view(P, 4), flat[7 * P:].view(P, 4)
    out, o = [], 0
    for K in Ks:
        out.append(torch.cat([c[o:o + K].reshape(-1), q[o:o + K].reshape(-1), r[o:o + K].reshape(-1)]))
        o += K
    return out


def join_flat(flats, Ks):
    """Batched flat buffer from per-scene ones."""
    cs, qs, rs = [], [], []
    for f, K in zip(flats, Ks):
        cs.append(f[:3 * K]); qs.append(f[3 * K:7 * K]); rs.append(f[7 * K:])
    return torch.cat(cs + qs + rs).contiguous()


def _split_round(ss, fit, active, Ks, n_iter, tau, params, moments):
    """Sec. 3.3 plane splitting of the active scenes on the device; updates
    params, moments and returns the new plane counts and the number of splits."""
    P = int(sum(Ks))
    dev = fit.flat.device
    ptr = torch.tensor(np.concatenate([[0], np.cumsum(Ks)]), dtype=torch.int32, device=dev)
    cap = 2 * P
    out = torch.empty(11 * cap, device=dev)
    mo, vo = torch.empty_like(out), torch.empty_like(out)
    ptr_o = torch.empty_like(ptr)
    rank = torch.empty(P + 1, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    B.ps_split_planes(fit.flat, fit.m, fit.v, ptr, fit.split_acc, n_iter, tau, out, mo, vo,
                      ptr_o, cap, rank, cnt)
    Pn = int(cnt.item())
    new_ptr = ptr_o.cpu().numpy()
    nK = [int(new_ptr[i + 1] - new_ptr[i]) for i in range(len(active))]
    for s, f, m, v in zip(active, split_flat(out[:11 * Pn], nK), split_flat(mo[:11 * Pn], nK),
                          split_flat(vo[:11 * Pn], nK)):
        params[s] = f.clone()
        moments[s] = (m.clone(), v.clone())
    return nK, Pn - P


def fit_until(ss: SceneSet, scenes, threshold=0.02, max_iters=3000, capacity_headroom=1.6,
              use_graphs=True, compact=True, lam_offset=0, split_every=0, split_tau=0.2,
              grow_margin=1.1, capacity=None):
    """Fits the given scenes together (one launch per kernel per step) until
    every scene's mean depth error is <= threshold or max_iters.  With compact,
    scenes that reach the threshold leave the batch: the remaining scenes'
    parameters and Adam moments move to a smaller frame whose graphs are
    captured again.  With split_every > 0, planes are split every split_every
    iterations (Sec. 3.3; threshold split_tau on the radius gradient of the
    per-view mean loss) and the frame is rebuilt with the new plane counts.  Returns
    per-scene iterations and errors and the GPU time spent stepping (CUDA
    events; frame rebuilds, splitting and the per-rotation convergence check are
    outside the timed region).  Tile-list capacity: the frame is rebuilt with
    capacity_headroom x the current need when the last step's need x grow_margin
    passes the capacity (None: never), and a rotation whose lists overflowed
    is redone from the state before it in a rebuilt frame; capacity sets the
    smallest capacity of a new frame (default: 64 entries per tile)."""
    scenes = list(scenes)
    S = len(scenes)
    nb = ss.n_batches
    Kd = {s: ss.K[s] for s in scenes}
    splits = 0
    overflows = 0
    next_split = split_every if split_every > 0 else None
    params = {s: f for s, f in zip(scenes, split_flat(ss.flat_for(scenes), [ss.K[s] for s in scenes]))}
    moments = {s: (torch.zeros_like(params[s]), torch.zeros_like(params[s])) for s in scenes}
    latest = {}                     # (scene, view) -> (sum |D - D*|, count)
    done_at = {s: None for s in scenes}
    err = {s: float("nan") for s in scenes}
    spent_ms = 0.0
    ite = 0
    active = list(scenes)
    while ite < max_iters and active:
        Ks = [Kd[s] for s in active]
        r = ss.renderer(active, Ks=Ks, capacity=capacity)
        flat = join_flat([params[s] for s in active], Ks)
        fit = SP.Fitter(r, flat)
        fit.m.copy_(join_flat([moments[s][0] for s in active], Ks))
        fit.v.copy_(join_flat([moments[s][1] for s in active], Ks))
        fit.ite = ite
        fit.lam_offset = lam_offset
        acc_from = ite
        if next_split is not None:
            fit.enable_split(ss.split_scales(active, Ks))
        need = 0
        for b in range(nb):
            r.select(b)
            r.ensure_capacity(flat, B.lambda_schedule(ite + lam_offset), headroom=capacity_headroom)
            need = max(need, int(r.required.item()))
        if need * capacity_headroom > r.capacity:
            r._alloc_lists(int(need * capacity_headroom) + 1024)
        r.status.zero_()
        if use_graphs:
            fit.enable_graphs(max_iters + nb, list(range(nb)), [(ss.gt_depth, ss.gt_normal)] * nb)
        view_scene = np.repeat(np.arange(len(active)), ss.vps)
        rebuild = False
        while ite < max_iters and not rebuild:
            # state before the rotation: a rotation whose tile lists overflowed is redone
            snap = (fit.flat.clone(), fit.m.clone(), fit.v.clone(), ite,
                    None if fit.split_acc is None else fit.split_acc.clone())
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sums = []
            for b in range(nb):
                if use_graphs:
                    sums.append(fit.replay(b))
                else:
                    r.select(b)
                    sums.append(fit.step(ss.gt_depth, ss.gt_normal, batch=b).clone())
                ite += 1
            e1.record()
            torch.cuda.synchronize()
            spent_ms += e0.elapsed_time(e1)
            if int(r.status.item()) & (1 << B.PS_ERR_CAPACITY):
                # planes grew past the tile-list capacity: back to the state before the
                # rotation, then a frame with capacity for the current planes
                overflows += 1
                if overflows > 8:
                    raise RuntimeError("tile-list capacity overflow persists during the fit")
                fit.flat.copy_(snap[0]); fit.m.copy_(snap[1]); fit.v.copy_(snap[2])
                ite = snap[3]
                for s, f, m, v in zip(active, split_flat(fit.flat, Ks), split_flat(fit.m, Ks),
                                      split_flat(fit.v, Ks)):
                    params[s] = f.clone()
                    moments[s] = (m.clone(), v.clone())
                rebuild = True
                break
            if grow_margin is not None and int(r.required.item()) * grow_margin > r.capacity:
                # close to the capacity: rebuild with headroom before it overflows
                for s, f, m, v in zip(active, split_flat(fit.flat, Ks), split_flat(fit.m, Ks),
                                      split_flat(fit.v, Ks)):
                    params[s] = f.clone()
                    moments[s] = (m.clone(), v.clone())
                rebuild = True
            vs = torch.stack(sums).cpu().numpy()          # [nb, V, 4]
            for b in range(nb):
                vi = ss.batch_views(b)
                for v in range(len(view_scene)):
                    s = active[view_scene[v]]
                    latest[(s, vi[s][v % ss.vps])] = (vs[b, v, 2], vs[b, v, 3])
            newly = []
            for s in active:
                num = sum(val[0] for key, val in latest.items() if key[0] == s)
                den = sum(val[1] for key, val in latest.items() if key[0] == s)
                err[s] = num / max(den, 1.0)
                if done_at[s] is None and err[s] <= threshold:
                    done_at[s] = (ite, spent_ms)
                    newly.append(s)
            if newly and compact:
                for s, f in zip(active, split_flat(fit.flat, Ks)):
                    params[s] = f.clone()
                for s, m, v in zip(active, split_flat(fit.m, Ks), split_flat(fit.v, Ks)):
                    moments[s] = (m.clone(), v.clone())
                active = [s for s in active if done_at[s] is None]
                rebuild = True
            elif all(done_at[s] is not None for s in active):
                for s, f in zip(active, split_flat(fit.flat, Ks)):
                    params[s] = f.clone()
                active = []
                break
            elif next_split is not None and ite >= next_split:
                nK, n_split = _split_round(ss, fit, active, Ks, ite - acc_from, split_tau,
                                           params, moments)
                splits += n_split
                for s, k in zip(active, nK):
                    Kd[s] = k
                next_split += split_every
                rebuild = True
        if not rebuild and active:
            for s, f in zip(active, split_flat(fit.flat, Ks)):
                params[s] = f.clone()
        del fit, r
    return {"iterations": ite, "gpu_ms": spent_ms, "done_at": [done_at[s] for s in scenes],
            "err": [err[s] for s in scenes], "params": [params[s] for s in scenes],
            "planes": [Kd[s] for s in scenes], "splits": splits, "overflows": overflows}
