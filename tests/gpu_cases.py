"""Shared helpers of the GPU parity tests: run the libps path and the oracle on
the same seeded inputs and collect comparable numpy arrays."""
from __future__ import annotations

import json
import os

import numpy as np

from oracle import oracle as O
from paper_2412_03451_gb300 import scenes as S

Z_NEAR32 = float(np.float32(0.01))     # the library takes z_near as f32; the oracle gets the same value
Z_FAR32 = 100.0


def f32(x: float) -> float:
    return float(np.float32(x))


# measured parity figures are appended to $PS_REPORT_DIR/parity_report.jsonl when it is set
REPORT = (os.path.join(os.environ["PS_REPORT_DIR"], "parity_report.jsonl")
          if os.environ.get("PS_REPORT_DIR") else None)


def record(name, **kw):
    """Appends one line of measured parity figures to the run's report (best effort)."""
    if REPORT is None:
        return
    try:
        os.makedirs(os.path.dirname(REPORT), exist_ok=True)
        with open(REPORT, "a") as f:
            f.write(json.dumps(dict(test=name, **kw)) + "\n")
    except OSError:
        pass


def gpu_run(planes: S.Planes, cams: S.Cameras, lam: float, tile=(16, 16), M=30, flags=0,
            capacity=None, dLdD=None, dLdN=None, backward=False):
    """Runs project -> bin -> fwd (-> bwd) on cuda:0 for one scene.  Returns numpy arrays."""
    import torch
    from paper_2412_03451_gb300 import splat as SP
    V = cams.V
    r = SP.Renderer([cams.H] * V, [cams.W] * V, [0] * V, [0, planes.K], tile=tile, M=M,
                    capacity=capacity, flags=flags)
    r.set_cameras(cams.w2c, cams.intr)
    flat = SP.planes_to_flat(planes.center, planes.quat, planes.radii, "cuda")
    if capacity is None:
        r.ensure_capacity(flat, lam)
    r.status.zero_()
    r.forward(flat, lam)
    out = {}
    if backward:
        g = torch.zeros_like(flat)
        gD = torch.from_numpy(np.asarray(dLdD, np.float32).reshape(-1)).cuda()
        gN = torch.from_numpy(np.asarray(dLdN, np.float32).reshape(-1, 3)).cuda()
        r.backward(flat, g, gD, gN)
        gc, gq, gr = SP.flat_views(g, planes.K)
        out.update(g_center=gc.cpu().numpy(), g_quat=gq.cpu().numpy(), g_radii=gr.cpu().numpy())
    torch.cuda.synchronize()
    H, W = cams.H, cams.W
    out.update(
        rect=r.rect.cpu().numpy().reshape(V, planes.K, 4),
        key=r.key.cpu().numpy().reshape(V, planes.K),
        tile_ptr=r.tile_ptr.cpu().numpy(),
        tile_ent=r.tile_ent.cpu().numpy()[: int(r.tile_ptr[-1].item())],
        tile_key=r.tile_key.cpu().numpy()[: int(r.tile_ptr[-1].item())],
        required=int(r.required.item()),
        status=int(r.status.item()),
        depth=r.depth.cpu().numpy().reshape(V, H, W),
        normal=r.normal.cpu().numpy().reshape(V, H, W, 3),
        alpha=r.alpha.cpu().numpy().reshape(V, H, W),
        delta=r.settings.delta,
    )
    return out


def oracle_bins(planes, cams, delta, tile, gaussian=False):
    rect, key, key32 = O.bin_records(planes.center, planes.quat, planes.radii, cams.w2c, cams.intr,
                                     cams.H, cams.W, tile[0], tile[1], delta, z_near=Z_NEAR32,
                                     z_far=Z_FAR32, gaussian=gaussian)
    ns = O.records_ns(planes.center, planes.quat, planes.radii, cams.w2c)
    ptr, ent, ekey = O.tile_lists(rect, key32, ns, cams.intr, cams.H, cams.W, tile[0], tile[1],
                                  z_near=Z_NEAR32)
    return rect, key32, ptr, ent, ekey


def oracle_render(planes, cams, lam, M=30, rows=None, gaussian=False, single_radii=False):
    return O.render(planes.center, planes.quat, planes.radii, cams.w2c, cams.intr, cams.H, cams.W,
                    f32(lam), M=M, z_near=Z_NEAR32, z_far=Z_FAR32, rows=rows, gaussian=gaussian,
                    single_radii=single_radii)


def loss_mask(o, gt_depth, gt_normal, tol_d=1e-4, tol_n=1e-5):
    """Pixels to leave unsupervised on both sides (ground-truth depth set to 0) when
    the GPU computes the Eq. 14 gradient from its own FP32 render (the fused kernel):
    pixels where FP32 rounding could flip a min / sign branch, the filter, the depth
    order or the z range (oracle flag bits 2 and 3), and pixels where the sign of
    D - D*, of a component of N - N* or of 1 - N.N* could differ between the FP32
    render and the oracle's, because the oracle's value lies within twice the bar the
    render is held to (max(tol, 2 x the oracle's rounding-sensitivity estimate))."""
    bd = np.maximum(tol_d, 2.0 * o["sens_d"])
    bn = np.maximum(tol_n, 2.0 * o["sens_n"])
    m = (o["ill"] & 12) != 0
    m |= np.abs(o["depth"] - gt_depth) <= 2.0 * bd
    m |= (np.abs(o["normal"] - gt_normal) <= 2.0 * bn[..., None]).any(axis=-1)
    m |= np.abs(1.0 - (o["normal"] * gt_normal).sum(axis=-1)) <= 6.0 * bn
    return m


def compare_maps(g, o, rows=None, tol_d=1e-4, tol_n=1e-5):
    """Max depth / normal error over well-conditioned pixels (oracle ill bit 0
    clear) and the count of ill-conditioned pixels.  Of those, the pixels where
    only the size of the rounding effect is the issue (bit 2 clear: no filter,
    order or range flip) are checked against the oracle's own first-order
    estimate of it: |D - D*| <= max(tol_d, 2 sens_d), likewise N."""
    sl = slice(None) if rows is None else slice(rows[0], rows[1])
    ill = o["ill"][:, sl]
    well = (ill & 1) == 0
    sens = ((ill & 1) != 0) & ((ill & 4) == 0)
    dd = np.abs(g["depth"][:, sl].astype(np.float64) - o["depth"][:, sl])
    dn = np.abs(g["normal"][:, sl].astype(np.float64) - o["normal"][:, sl]).max(axis=-1)
    bd = np.maximum(tol_d, 2.0 * o["sens_d"][:, sl])
    bn = np.maximum(tol_n, 2.0 * o["sens_n"][:, sl])
    return dict(
        n_pix=int(well.size), n_ill=int((~well).sum()), n_sens=int(sens.sum()),
        n_flip=int(((ill & 4) != 0).sum()),
        max_dd_well=float(dd[well].max()) if well.any() else 0.0,
        max_dn_well=float(dn[well].max()) if well.any() else 0.0,
        max_dd_ill=float(dd[~well].max()) if (~well).any() else 0.0,
        n_bad_d=int((dd[well] > tol_d).sum()), n_bad_n=int((dn[well] > tol_n).sum()),
        n_bad_sens_d=int((dd[sens] > bd[sens]).sum()), n_bad_sens_n=int((dn[sens] > bn[sens]).sum()),
        worst_sens_ratio_d=float((dd[sens] / bd[sens]).max()) if sens.any() else 0.0,
        worst_sens_ratio_n=float((dn[sens] / bn[sens]).max()) if sens.any() else 0.0,
    )


def grad_errors(g_gpu, g_or, rel=1e-3, floor=1e-6):
    """Per-plane gradient check of one parameter group: ||g - g*|| <=
    rel ||g*|| + floor max_planes ||g*||.  Returns (n_bad, worst ratio)."""
    n_or = np.linalg.norm(g_or, axis=1)
    err = np.linalg.norm(g_gpu.astype(np.float64) - g_or, axis=1)
    bound = rel * n_or + floor * max(n_or.max(), 1e-30)
    ratio = err / np.maximum(bound, 1e-300)
    return int((err > bound).sum()), float(ratio.max())


def gpu_fused_vs_split(planes: S.Planes, cams: S.Cameras, lam: float, gt_depth, gt_normal,
                       tile=(16, 16), M=30, flags=0):
    """Runs the fused forward+loss+backward and the separate fwd -> loss -> bwd
    calls on the same inputs; returns both results as numpy arrays."""
    import torch
    from paper_2412_03451_gb300 import splat as SP
    V = cams.V
    r = SP.Renderer([cams.H] * V, [cams.W] * V, [0] * V, [0, planes.K], tile=tile, M=M, flags=flags)
    r.set_cameras(cams.w2c, cams.intr)
    flat = SP.planes_to_flat(planes.center, planes.quat, planes.radii, "cuda")
    r.ensure_capacity(flat, lam)
    gD = torch.from_numpy(np.asarray(gt_depth, np.float32).reshape(-1)).cuda()
    gN = torch.from_numpy(np.asarray(gt_normal, np.float32).reshape(-1, 3)).cuda()
    r.status.zero_()
    # separate path
    r.forward(flat, lam)
    r.loss(gD, gN)
    g_split = torch.zeros_like(flat)
    r.backward(flat, g_split)
    split = dict(depth=r.depth.clone(), normal=r.normal.clone(), dLdD=r.dLdD.clone(),
                 dLdN=r.dLdN.clone(), sums=r.view_sums.clone(), grad=g_split)
    # fused path
    r.depth.zero_(); r.normal.zero_(); r.dLdD.zero_(); r.dLdN.zero_()
    r.project_bin(flat, lam)
    g_fused = torch.zeros_like(flat)
    r.fused(flat, g_fused, gD, gN, write_maps=True)
    fused = dict(depth=r.depth.clone(), normal=r.normal.clone(), dLdD=r.dLdD.clone(),
                 dLdN=r.dLdN.clone(), sums=r.view_sums.clone(), grad=g_fused)
    torch.cuda.synchronize()
    status = int(r.status.item())
    to_np = lambda d: {k: v.cpu().numpy() for k, v in d.items()}
    return to_np(split), to_np(fused), status
