"""PyTorch driver of libps: buffers, one optimisation step, autograd wrapper.

PyTorch provides device memory and streams; every step of the rendering path
(projection, binning, forward splat, loss, backward splat, Adam) is a call into
libps through ``binding``.  The plane parameters of all scenes live in one flat
float32 buffer laid out as [center P*3 | quat P*4 | radii P*4], so that Adam
runs as two launches (the radii group is clamped to stay positive, Eq. 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B

R_MIN = 1e-3          # radii are clamped to >= 1 mm after each Adam step (Eq. 1: r in R^4_+)


def planes_to_flat(center, quat, radii, device) -> torch.Tensor:
    P = int(np.asarray(center).shape[0])
    flat = np.concatenate([np.asarray(center, np.float32).reshape(-1),
                           np.asarray(quat, np.float32).reshape(-1),
                           np.asarray(radii, np.float32).reshape(-1)])
    assert flat.size == 11 * P
    return torch.from_numpy(flat).to(device)


def flat_views(flat: torch.Tensor, P: int):
    return flat[:3 * P].view(P, 3), flat[3 * P:7 * P].view(P, 4), flat[7 * P:].view(P, 4)


@dataclass
class StepStats:
    view_sums: torch.Tensor      # [V,4] f64 (device)
    required: torch.Tensor       # [1] i64 (device)
    status: torch.Tensor         # [1] i32 (device)


class Renderer:
    """Owns every buffer of one batch shape (a fixed set of view sizes and
    scene plane counts) and runs the libps calls on the current stream."""

    def __init__(self, H, W, scene_of_view, plane_ptr, tile=(16, 16), M=30, capacity=None,
                 device="cuda", flags=0, warps=0):
        self.device = torch.device(device)
        self.H = np.asarray(H, np.int32).reshape(-1)
        self.W = np.asarray(W, np.int32).reshape(-1)
        self.V = int(self.H.size)
        self.scene_of_view = np.asarray(scene_of_view, np.int32).reshape(-1)
        self.plane_ptr = np.asarray(plane_ptr, np.int32).reshape(-1)
        self.P = int(self.plane_ptr[-1])
        self.tile = (int(tile[0]), int(tile[1]))
        self.M = int(M)
        self.flags = int(flags)
        self.warps = int(warps)       # warps per CTA of the splat kernels (0: the library default)
        # plan once with identity cameras to learn the totals
        eye = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32),
                      (self.V, 1, 1))
        intr = np.tile(np.array([1, 1, 0, 0], np.float32), (self.V, 1))
        self._views_host, self.frame = B.ps_plan_views(self.H, self.W, self.scene_of_view,
                                                       self.plane_ptr, eye, intr, *self.tile)
        f = self.frame
        dev = self.device
        self.views_dev = torch.zeros(self.V * 128, dtype=torch.uint8, device=dev)
        self.frame.views = self.views_dev.data_ptr()
        R = f.n_records
        self.rec = torch.zeros((max(R, 1), 16), dtype=torch.float32, device=dev)
        self.rect = torch.zeros((max(R, 1), 4), dtype=torch.int32, device=dev)
        self.key = torch.zeros(max(R, 1), dtype=torch.float32, device=dev)
        self.tile_ptr = torch.zeros(f.n_tiles + 1, dtype=torch.int32, device=dev)
        if capacity is None:
            capacity = max(1 << 16, 64 * f.n_tiles)
        self._alloc_lists(int(capacity))
        self.required = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        npix = int(f.n_pixels)
        self.depth = torch.zeros(npix, dtype=torch.float32, device=dev)
        self.normal = torch.zeros((npix, 3), dtype=torch.float32, device=dev)
        self.alpha = torch.zeros(npix, dtype=torch.float32, device=dev)
        self.dLdD = torch.zeros(npix, dtype=torch.float32, device=dev)
        self.dLdN = torch.zeros((npix, 3), dtype=torch.float32, device=dev)
        self.view_sums = torch.zeros((self.V, 4), dtype=torch.float64, device=dev)
        self.bwd_ws = torch.zeros((B.ps_bwd_workspace_bytes(f) + 255) // 256 * 64,
                                  dtype=torch.float32, device=dev)
        self.fwd_ws = torch.zeros((B.ps_fwd_workspace_bytes(f) + 255) // 256 * 64,
                                  dtype=torch.float32, device=dev)
        self._batches = None
        self._views_tensor = self.views_dev
        self.settings = None
        # bumped whenever the records / tile lists or the camera descriptors change, so a
        # holder of an earlier render (PlaneSplatFunction) can tell that they are stale
        self.generation = 0

    # -- buffers ---------------------------------------------------------------
    def _alloc_lists(self, capacity: int):
        self.capacity = int(capacity)
        self.tile_ent = torch.zeros(max(self.capacity, 1), dtype=torch.int32, device=self.device)
        self.tile_key = torch.zeros(max(self.capacity, 1), dtype=torch.float32, device=self.device)
        nbytes = B.ps_bin_workspace_bytes(self.frame, self.capacity)
        self.bin_ws = torch.zeros((nbytes + 255) // 256 * 64, dtype=torch.float32,
                                  device=self.device)

    def set_cameras(self, w2c, intr):
        """Re-plans the views with new poses/intrinsics (host) and uploads the
        128-byte descriptors (synchronous copy of V * 128 bytes)."""
        self._views_host, fr = B.ps_plan_views(self.H, self.W, self.scene_of_view, self.plane_ptr,
                                               w2c, intr, *self.tile)
        raw = np.frombuffer(bytes(self._views_host), dtype=np.uint8).copy()
        self.views_dev.copy_(torch.from_numpy(raw))
        self.frame.views = self.views_dev.data_ptr()
        self._views_tensor = self.views_dev
        self.generation += 1

    def preplan(self, w2c_batches, intr_batches, gt_off_batches=None):
        """Plans several camera batches of this renderer's shape once and keeps
        their descriptors on the device; select(i) then switches batches with no
        host-to-device traffic (and so can run inside a captured graph).
        gt_off_batches (optional) gives every view of every batch the offset of its
        supervision image in resident ground-truth arrays."""
        raws = []
        for i, (w2c, intr) in enumerate(zip(w2c_batches, intr_batches)):
            go = None if gt_off_batches is None else gt_off_batches[i]
            vh, _ = B.ps_plan_views(self.H, self.W, self.scene_of_view, self.plane_ptr, w2c, intr,
                                    *self.tile, gt_off=go)
            raws.append(np.frombuffer(bytes(vh), dtype=np.uint8))
        self._batches = torch.from_numpy(np.stack(raws)).to(self.device)
        self.select(0)

    def select(self, i: int):
        self.frame.views = self._batches[i].data_ptr()
        self._views_tensor = self._batches[i]
        self.generation += 1

    def views_snapshot(self) -> torch.Tensor:
        """Device copy of the current view descriptors (V x 128 bytes)."""
        return self._views_tensor.clone()

    def make_settings(self, lam, flags=None, d_state=None):
        fl = self.flags if flags is None else flags
        if fl & B.PS_HARD:
            delta = 0.0
        elif fl & B.PS_GAUSSIAN:
            delta = B.gauss_extent()
        else:
            delta = B.filter_margin(float(np.float32(lam)))
        self.settings = B.make_settings(lam, delta, M=self.M, tile_w=self.tile[0],
                                        tile_h=self.tile[1], flags=fl, d_state=d_state,
                                        cta_warps=self.warps)
        return self.settings

    def planes_struct(self, flat: torch.Tensor) -> B.PsPlanes:
        c, q, r = flat_views(flat, self.P)
        p = B.PsPlanes()
        p.n_planes = self.P
        p.center, p.quat, p.radii = c.data_ptr(), q.data_ptr(), r.data_ptr()
        return p

    # -- the path ----------------------------------------------------------------
    def project_bin(self, flat: torch.Tensor, lam: float, flags=None, d_state=None):
        self.generation += 1
        s = self.make_settings(lam, flags, d_state)
        pl = self.planes_struct(flat)
        B.ps_project_cull(pl, self.frame, s, self.rec, self.rect, self.key, self.status)
        B.ps_bin_tiles(self.frame, s, self.rec, self.rect, self.key, self.tile_ptr, self.tile_ent,
                       self.tile_key, self.capacity, self.required, self.bin_ws, self.status)

    def ensure_capacity(self, flat, lam, flags=None, headroom=1.5) -> bool:
        """Runs projection + binning once and grows the tile-list capacity if it
        was too small (synchronises).  Returns True if it grew."""
        self.project_bin(flat, lam, flags)
        need = int(self.required.item())
        if need > self.capacity:
            self._alloc_lists(int(need * headroom) + 1024)
            self.status.zero_()
            return True
        return False

    def splat_forward(self, alpha=True):
        B.ps_splat_fwd(self.frame, self.settings, self.rec, self.tile_key, self.tile_ptr, self.tile_ent,
                       self.capacity, self.depth, self.normal, self.alpha if alpha else None,
                       self.fwd_ws, self.status)
        return self.depth, self.normal

    def forward(self, flat: torch.Tensor, lam: float, flags=None, alpha=True):
        self.project_bin(flat, lam, flags)
        return self.splat_forward(alpha)

    def plane_ids(self, flat: torch.Tensor, lam: float = 300.0, hard: bool = True):
        """Per-pixel index of the nearest composited plane (-1: none) and depth."""
        fl = B.PS_HARD if hard else 0
        self.project_bin(flat, lam, flags=fl)
        ids = torch.empty(int(self.frame.n_pixels), dtype=torch.int32, device=self.device)
        B.ps_splat_ids(self.frame, self.settings, self.rec, self.tile_key, self.tile_ptr, self.tile_ent,
                       self.capacity, ids, self.depth, self.fwd_ws, self.status)
        return ids, self.depth

    def count_pairs(self, counts: torch.Tensor):
        """Work counts of the current tile lists (tested, candidate, composited pairs)."""
        B.ps_count_pairs(self.frame, self.settings, self.rec, self.tile_key, self.tile_ptr,
                         self.tile_ent, self.capacity, counts)

    def loss(self, gt_depth, gt_normal):
        B.ps_loss(self.frame, self.settings, self.depth, self.normal, gt_depth, gt_normal,
                  self.dLdD, self.dLdN, self.view_sums)
        return self.view_sums

    def fused(self, flat: torch.Tensor, grad_flat: torch.Tensor, gt_depth, gt_normal,
              write_maps: bool = False, view_sums=None):
        """Forward + Eq. 14 loss + backward in one pass (after project_bin).
        Accumulates the loss gradient into grad_flat; fills view_sums; writes
        depth/normal/dL maps only if write_maps."""
        pl = self.planes_struct(flat)
        gc, gq, gr = flat_views(grad_flat, self.P)
        m = write_maps
        B.ps_splat_fused(pl, self.frame, self.settings, self.rec, self.tile_key, self.tile_ptr,
                         self.tile_ent, self.capacity, gt_depth, gt_normal,
                         self.depth if m else None, self.normal if m else None,
                         self.dLdD if m else None, self.dLdN if m else None,
                         self.view_sums if view_sums is None else view_sums,
                         gc, gq, gr, self.bwd_ws, self.status)
        return self.view_sums if view_sums is None else view_sums

    def backward(self, flat: torch.Tensor, grad_flat: torch.Tensor, dLdD=None, dLdN=None):
        """Accumulates d(sum dLdD*D + dLdN.N)/dparams into grad_flat (same layout)."""
        pl = self.planes_struct(flat)
        gc, gq, gr = flat_views(grad_flat, self.P)
        B.ps_splat_bwd(pl, self.frame, self.settings, self.rec, self.tile_key, self.tile_ptr,
                       self.tile_ent, self.capacity, self.dLdD if dLdD is None else dLdD,
                       self.dLdN if dLdN is None else dLdN, gc, gq, gr, self.bwd_ws, self.status)


class PlaneSplatFunction(torch.autograd.Function):
    """(planes) -> (depth, normal) through libps, as a torch.autograd.Function
    whose backward is the hand-written adjoint kernel ps_splat_bwd.

    apply(flat, renderer, lam, flags=None): flat is the [11 P] float32 parameter
    buffer of the renderer's scenes ([center P*3 | quat P*4 | radii P*4]); lam the
    Eq. 10 value.  The forward grows the renderer's tile-list capacity when needed
    (one host synchronisation), projects, bins and splats the renderer's current
    views, and returns copies of depth [n_pixels] and normal [n_pixels, 3].

    The backward recomputes every pixel's compositing state from the tile lists;
    nothing per pixel is kept.  If the renderer has projected, binned or switched
    cameras since this forward (another render before .backward()), the backward
    first rebuilds this forward's records and tile lists from the saved planes,
    camera descriptors and lambda: binning is deterministic, so they are the
    forward's own lists bit for bit.  The renderer's buffers then hold this
    rebuilt state and its generation moves on, so later holders rebuild theirs."""

    @staticmethod
    def forward(ctx, flat, renderer: Renderer, lam: float, flags=None):
        if renderer.ensure_capacity(flat, lam, flags):
            renderer.project_bin(flat, lam, flags)      # the lists of the grown buffers
        renderer.splat_forward(alpha=False)
        ctx.renderer = renderer
        ctx.lam, ctx.flags = lam, flags
        ctx.generation = renderer.generation
        ctx.views = renderer.views_snapshot()
        ctx.save_for_backward(flat)
        return renderer.depth.clone(), renderer.normal.clone()

    @staticmethod
    def backward(ctx, gD, gN):
        (flat,) = ctx.saved_tensors
        r = ctx.renderer
        g = torch.zeros_like(flat)
        if r.generation == ctx.generation:
            r.backward(flat, g, gD.contiguous(), gN.contiguous())
            return g, None, None, None
        cur_views, cur_tensor = r.frame.views, r._views_tensor
        try:
            r.frame.views = ctx.views.data_ptr()
            r._views_tensor = ctx.views
            r.project_bin(flat, ctx.lam, ctx.flags)
            r.backward(flat, g, gD.contiguous(), gN.contiguous())
        finally:
            r.frame.views, r._views_tensor = cur_views, cur_tensor
            r.generation += 1
        return g, None, None, None


class Fitter:
    """Adam fit of the planes of a batch (Sec. 3.3): per step, lambda from
    Eq. 10, render, Eq. 14 loss, backward, Adam with lr 1e-3 for every group."""

    def __init__(self, renderer: Renderer, flat: torch.Tensor, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8,
                 fused: bool = True):
        self.r = renderer
        self.fused = fused
        self.flat = flat
        self.grad = torch.zeros_like(flat)
        self.m = torch.zeros_like(flat)
        self.v = torch.zeros_like(flat)
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.ite = 0
        # Eq. 10 is evaluated at ite + lam_offset: a fit from a good initialisation
        # may skip the schedule's blurry start (Adam's step count is unaffected)
        self.lam_offset = 0
        # plane splitting (Sec. 3.3): running per-axis radius-gradient sums [P, 2] and, per
        # camera batch, the per-plane scale to the per-pixel mean loss
        self.split_acc = None
        self.split_scale = None

    def enable_split(self, plane_scales):
        """Accumulates the radius gradients of every step for plane splitting;
        plane_scales[b] ([P] device) is used at steps of camera batch b."""
        self.split_acc = torch.zeros((self.r.P, 2), device=self.flat.device)
        self.split_scale = list(plane_scales)

    def _accumulate(self, batch):
        if self.split_acc is not None:
            P = self.r.P
            B.ps_radii_grad_accum(self.grad[7 * P:], self.split_acc,
                                  plane_scale=self.split_scale[batch or 0])

    # -- captured CUDA graphs ------------------------------------------------------
    def enable_graphs(self, n_iters: int, batches, gt_slices, host_stream=None):
        """Captures one CUDA graph per camera batch of a full optimisation step
        (schedule advance, projection, binning, fused splat/loss/backward, Adam),
        with lambda, the binning margin and Adam's bias corrections read from a
        device-side per-iteration schedule, so that replaying graph s % n_batches
        at iteration s reproduces the eager step.  Capacity must already suffice
        (checked after replays through the status word).

        host_stream (optional) streams the supervision from pinned host memory:
        a dict with host_depth [n] and host_normal [n, 3] (pinned CPU tensors),
        offsets (the first pixel of each batch's supervision in them) and
        sums_host (pinned f64 [n_batches, V, 4]).  gt_slices are then two device
        buffer pairs used alternately (batch b reads gt_slices[b]; consecutive
        batches must use different buffers), and the graph of batch b also copies
        the next batch's supervision into the other buffer on a parallel branch
        (overlapping the step) and the step's loss sums to sums_host[b]."""
        dev = self.flat.device
        sched = B.step_schedule(n_iters, lam_offset=self.lam_offset)
        self.d_sched = torch.frombuffer(bytearray(sched), dtype=torch.uint8).to(dev)
        self.n_sched = n_iters
        self.d_state = torch.zeros(32, dtype=torch.uint8, device=dev)
        self.d_iter = torch.tensor([self.ite], dtype=torch.int32, device=dev)
        self.graphs = []
        r = self.r
        # each graph writes its own loss sums, so a host check after a rotation sees every batch
        self.graph_sums = [torch.zeros_like(r.view_sums) for _ in batches]
        stream = torch.cuda.Stream(device=dev)
        stream.wait_stream(torch.cuda.current_stream())
        # warm the library's per-device launch caches outside capture
        with torch.cuda.stream(stream):
            r.select(batches[0])
            saved = (self.flat.clone(), self.m.clone(), self.v.clone(), int(self.d_iter.item()),
                     None if self.split_acc is None else self.split_acc.clone())
            self._graph_body(*gt_slices[0], self.graph_sums[0], batches[0])
            torch.cuda.synchronize()
            self.flat.copy_(saved[0]); self.m.copy_(saved[1]); self.v.copy_(saved[2])
            self.d_iter.fill_(saved[3])
            if saved[4] is not None:
                self.split_acc.copy_(saved[4])
        side = torch.cuda.Stream(device=dev) if host_stream is not None else None
        for i, (b, (gd, gn)) in enumerate(zip(batches, gt_slices)):
            r.select(b)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                if host_stream is not None:
                    j = (i + 1) % len(batches)
                    nd, nn = gt_slices[j]
                    if nd.data_ptr() == gd.data_ptr():
                        raise ValueError("consecutive batches must read different supervision buffers")
                    o, m = host_stream["offsets"][j], nd.numel()
                    side.wait_stream(stream)
                    with torch.cuda.stream(side):
                        nd.copy_(host_stream["host_depth"][o:o + m], non_blocking=True)
                        nn.copy_(host_stream["host_normal"][o:o + m], non_blocking=True)
                self._graph_body(gd, gn, self.graph_sums[i], b)
                if host_stream is not None:
                    stream.wait_stream(side)
                    host_stream["sums_host"][i].copy_(self.graph_sums[i], non_blocking=True)
            self.graphs.append(g)
        torch.cuda.synchronize()

    def _graph_body(self, gt_depth, gt_normal, view_sums, batch=0):
        r = self.r
        P = r.P
        B.ps_step_advance(self.d_state, self.d_sched, self.n_sched, self.d_iter)
        r.project_bin(self.flat, 1.0, d_state=self.d_state)
        self.grad.zero_()
        r.fused(self.flat, self.grad, gt_depth, gt_normal, view_sums=view_sums)
        self._accumulate(batch)
        # one launch for all parameters; the radii (the last 4 P) are clamped below at R_MIN
        B.ps_adam_step_state(self.flat, self.grad, self.m, self.v, self.lr, self.b1, self.b2, self.eps,
                             self.d_state, clamp_min=R_MIN, clamp_from=7 * P)

    def replay(self, batch_index: int):
        """One optimisation step by graph replay (iteration counter on the device)."""
        self.graphs[batch_index].replay()
        self.ite += 1
        return self.graph_sums[batch_index]

    def step(self, gt_depth, gt_normal, lam=None, marks=None, batch=None):
        """One iteration.  If marks is a list, CUDA events are recorded on the
        current stream after each stage as (name, event) pairs."""
        def mark(tag):
            if marks is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                marks.append((tag, e))

        lam = B.lambda_schedule(self.ite + self.lam_offset) if lam is None else lam
        r = self.r
        mark("start")
        r.project_bin(self.flat, lam)
        mark("project_bin")
        self.grad.zero_()
        if self.fused:
            r.fused(self.flat, self.grad, gt_depth, gt_normal)
            mark("splat_fused")
        else:
            r.splat_forward(alpha=False)
            mark("splat_fwd")
            r.loss(gt_depth, gt_normal)
            mark("loss")
            r.backward(self.flat, self.grad)
            mark("splat_bwd")
        self._accumulate(batch)
        P = r.P
        t = self.ite + 1
        B.ps_adam_step(self.flat[:7 * P], self.grad[:7 * P], self.m[:7 * P], self.v[:7 * P],
                       self.lr, self.b1, self.b2, self.eps, t)
        B.ps_adam_step(self.flat[7 * P:], self.grad[7 * P:], self.m[7 * P:], self.v[7 * P:],
                       self.lr, self.b1, self.b2, self.eps, t, clamp_min=R_MIN)
        mark("adam")
        self.ite += 1
        return r.view_sums
