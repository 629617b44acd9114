"""ctypes binding of libps (include/ps.h), with the same function names.

Argument marshalling only: every step of the rendering path runs in the CUDA
kernels of libps.so.  Tensors are passed by data pointer; the stream is the
current PyTorch stream unless one is given.  If the compiled library is
missing, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libps.so")

PS_OK, PS_ERR_ARG, PS_ERR_CUDA, PS_ERR_CAPACITY, PS_ERR_TIMEOUT, PS_ERR_NONFINITE = range(6)
PS_SINGLE_RADII = 1
PS_HARD = 2
PS_GAUSSIAN = 4
PS_MAX_M = 64

EXPORTS = ("ps_plan_views", "ps_project_cull", "ps_bin_workspace_bytes", "ps_bin_tiles",
           "ps_fwd_workspace_bytes", "ps_splat_fwd", "ps_splat_ids", "ps_loss", "ps_bwd_workspace_bytes", "ps_splat_bwd",
           "ps_splat_fused", "ps_adam_step",
           "ps_count_pairs", "ps_step_advance", "ps_adam_step_state", "ps_gemm_bf16", "ps_wait_selftest",
           "ps_seed_im2col", "ps_seed_col2im", "ps_seed_relu_bwd", "ps_seed_transpose",
           "ps_seed_colsum", "ps_seed_pool", "ps_seed_pool_bwd", "ps_seed_loss", "ps_cast_bf16",
           "ps_radii_grad_accum", "ps_split_planes", "ps_merge_planes", "ps_status_string",
           "ps_version", "ps_lambda_schedule", "ps_filter_margin", "ps_gauss_extent",
           "ps_step_schedule", "ps_nn_workspace_bytes", "ps_nn_distance")


class PsSettings(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("w_min", ctypes.c_float),
                ("z_near", ctypes.c_float), ("z_far", ctypes.c_float),
                ("delta", ctypes.c_double), ("M", ctypes.c_int),
                ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("flags", ctypes.c_int),
                ("a_cos", ctypes.c_float), ("a_l1n", ctypes.c_float), ("a_depth", ctypes.c_float),
                ("cta_warps", ctypes.c_int), ("d_state", ctypes.c_void_p)]


class PsStepState(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("lambda_", ctypes.c_float), ("step", ctypes.c_int),
                ("bc1", ctypes.c_float), ("bc2", ctypes.c_float)]


class PsView(ctypes.Structure):
    _fields_ = [("w2c", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("tiles_x", ctypes.c_int), ("tiles_y", ctypes.c_int),
                ("tile_off", ctypes.c_int), ("rec_off", ctypes.c_int), ("plane_off", ctypes.c_int),
                ("K", ctypes.c_int), ("pix_off", ctypes.c_longlong), ("scene", ctypes.c_int),
                ("reserved", ctypes.c_int), ("gt_off", ctypes.c_longlong),
                ("reserved2", ctypes.c_int * 2)]


class PsFrame(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("n_records", ctypes.c_int),
                ("n_tiles", ctypes.c_int), ("max_K", ctypes.c_int),
                ("n_pixels", ctypes.c_longlong), ("views", ctypes.c_void_p)]


class PsPlanes(ctypes.Structure):
    _fields_ = [("n_planes", ctypes.c_int), ("reserved", ctypes.c_int),
                ("center", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("radii", ctypes.c_void_p)]


assert ctypes.sizeof(PsView) == 128
assert ctypes.sizeof(PsSettings) == 64
assert ctypes.sizeof(PsStepState) == 24

_lock = threading.Lock()
_lib = None


class PsError(RuntimeError):
    pass


def load():
    """Loads libps.so (built by paper_2412_03451_gb300._build); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise PsError("libps.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        P, I, LL, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t
        F, D = ctypes.c_float, ctypes.c_double
        sig = {
            "ps_plan_views": ([I, P, P, P, I, P, P, P, I, I, P, P], I),
            "ps_project_cull": ([P, P, P, P, P, P, P, P], I),
            "ps_bin_workspace_bytes": ([P, LL], SZ),
            "ps_bin_tiles": ([P, P, P, P, P, P, P, P, LL, P, P, SZ, P, P], I),
            "ps_fwd_workspace_bytes": ([P], SZ),
            "ps_splat_fwd": ([P, P, P, P, P, P, LL, P, P, P, P, SZ, P, P], I),
            "ps_splat_ids": ([P, P, P, P, P, P, LL, P, P, P, SZ, P, P], I),
            "ps_loss": ([P, P, P, P, P, P, P, P, P, P], I),
            "ps_bwd_workspace_bytes": ([P], SZ),
            "ps_splat_bwd": ([P, P, P, P, P, P, P, LL, P, P, P, P, P, P, SZ, P, P], I),
            "ps_splat_fused": ([P, P, P, P, P, P, P, LL, P, P, P, P, P, P, P, P, P, P, P, SZ, P, P], I),
            "ps_adam_step": ([P, P, P, P, LL, F, F, F, F, I, F, P], I),
            "ps_count_pairs": ([P, P, P, P, P, P, LL, P, P], I),
            "ps_step_advance": ([P, P, I, P, P], I),
            "ps_gemm_bf16": ([P, P, P, P, P, I, I, I, I, I, I, P, P], I),
            "ps_wait_selftest": ([P, LL, P], I),
            "ps_seed_im2col": ([P, I, I, I, I, I, P, P], I),
            "ps_seed_col2im": ([P, I, I, I, I, I, P, P], I),
            "ps_seed_relu_bwd": ([P, P, LL, F, P, P, P], I),
            "ps_seed_transpose": ([P, I, I, I, I, P, I, P], I),
            "ps_seed_colsum": ([P, LL, I, P, P], I),
            "ps_seed_pool": ([P, I, I, I, P, P, P], I),
            "ps_seed_pool_bwd": ([P, I, I, I, P, P], I),
            "ps_seed_loss": ([P, P, I, I, P, P, P], I),
            "ps_cast_bf16": ([P, I, I, I, P, P], I),
            "ps_adam_step_state": ([P, P, P, P, LL, F, F, F, F, P, F, LL, P], I),
            "ps_radii_grad_accum": ([P, P, F, I, P, P], I),
            "ps_split_planes": ([P, P, P, I, P, I, P, I, F, P, P, P, P, I, P, P, P], I),
            "ps_merge_planes": ([P, I, P, F, F, P, P, P, P], I),
            "ps_status_string": ([I], ctypes.c_char_p),
            "ps_version": ([], I),
            "ps_lambda_schedule": ([I], D),
            "ps_filter_margin": ([D, D], D),
            "ps_gauss_extent": ([D], D),
            "ps_step_schedule": ([I, I, I, F, F, D, P], I),
            "ps_nn_workspace_bytes": ([I], SZ),
            "ps_nn_distance": ([P, I, F, F, F, P, P, P, SZ, P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(code: int, what: str):
    if code != PS_OK:
        msg = load().ps_status_string(code).decode()
        raise PsError("%s failed: %s (%d)" % (what, msg, code))


def _ptr(t) -> int | None:
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# Host planning.

def ps_plan_views(H, W, scene_of_view, plane_ptr, w2c, intr, tile_w, tile_h, gt_off=None):
    """Plans a batch of views.  Returns (PsView array (host), PsFrame with views=NULL).
    gt_off (optional, per view) points each view at its supervision pixels."""
    lib = load()
    V = len(H)
    Ha = np.ascontiguousarray(H, dtype=np.int32)
    Wa = np.ascontiguousarray(W, dtype=np.int32)
    sc = np.ascontiguousarray(scene_of_view, dtype=np.int32)
    pp = np.ascontiguousarray(plane_ptr, dtype=np.int32)
    w2 = np.ascontiguousarray(np.asarray(w2c, dtype=np.float32).reshape(V, 12))
    it = np.ascontiguousarray(np.asarray(intr, dtype=np.float32).reshape(V, 4))
    views = (PsView * V)()
    frame = PsFrame()
    code = lib.ps_plan_views(V, Ha.ctypes.data, Wa.ctypes.data, sc.ctypes.data, len(pp) - 1,
                             pp.ctypes.data, w2.ctypes.data, it.ctypes.data, int(tile_w),
                             int(tile_h), ctypes.byref(views), ctypes.byref(frame))
    _check(code, "ps_plan_views")
    if gt_off is not None:
        for v in range(V):
            views[v].gt_off = int(gt_off[v])
    return views, frame


def make_settings(lam, delta, M=30, tile_w=16, tile_h=16, flags=0, w_min=1e-4, z_near=0.01,
                  z_far=100.0, a_cos=5.0, a_l1n=5.0, a_depth=1.0, d_state=None, cta_warps=0) -> PsSettings:
    s = PsSettings()
    s.lambda_ = float(lam)
    s.w_min = float(w_min)
    s.z_near = float(z_near)
    s.z_far = float(z_far)
    s.delta = float(delta)
    s.M = int(M)
    s.tile_w, s.tile_h = int(tile_w), int(tile_h)
    s.flags = int(flags)
    s.a_cos, s.a_l1n, s.a_depth = float(a_cos), float(a_l1n), float(a_depth)
    s.cta_warps = int(cta_warps)
    s.d_state = None if d_state is None else d_state.data_ptr()
    return s


def step_schedule(n: int, first: int = 0, b1: float = 0.9, b2: float = 0.999,
                  lam_offset: int = 0, w_min: float = 1e-4) -> bytes:
    """Packed ps_step_state entries for optimisation steps first .. first + n - 1
    (ps_step_schedule: Eq. 10 lambda, its binning margin, Adam's step number and
    bias corrections)."""
    arr = (PsStepState * n)()
    _check(load().ps_step_schedule(int(first), int(n), int(lam_offset), float(b1), float(b2),
                                   float(w_min), arr), "ps_step_schedule")
    return bytes(arr)


def filter_margin(lam: float, w_min: float = 1e-4) -> float:
    """ps_filter_margin: delta with 2 sigmoid(-5 lam delta) = w_min (Eq. 7-8, Sec. 3.2)."""
    return float(load().ps_filter_margin(float(lam), float(w_min)))


def gauss_extent(w_min: float = 1e-4) -> float:
    """ps_gauss_extent: the radius factor kappa of the Eq. 5 binning."""
    return float(load().ps_gauss_extent(float(w_min)))


def lambda_schedule(ite: int) -> float:
    """ps_lambda_schedule: Eq. 10 at iteration ite (from 0)."""
    return float(load().ps_lambda_schedule(int(ite)))


# ---------------------------------------------------------------------------
# Device calls.

def ps_project_cull(planes: PsPlanes, frame: PsFrame, settings: PsSettings, rec, rect, key,
                    status, stream=None):
    _check(load().ps_project_cull(ctypes.byref(planes), ctypes.byref(frame), ctypes.byref(settings),
                                  _ptr(rec), _ptr(rect), _ptr(key), _ptr(status), _stream(stream)),
           "ps_project_cull")


def ps_bin_workspace_bytes(frame: PsFrame, capacity: int) -> int:
    return int(load().ps_bin_workspace_bytes(ctypes.byref(frame), int(capacity)))


def ps_bin_tiles(frame, settings, rec, rect, key, tile_ptr, tile_ent, tile_key, capacity, required,
                 ws, status, stream=None):
    nbytes = ws.numel() * ws.element_size()
    _check(load().ps_bin_tiles(ctypes.byref(frame), ctypes.byref(settings), _ptr(rec), _ptr(rect),
                               _ptr(key), _ptr(tile_ptr), _ptr(tile_ent), _ptr(tile_key),
                               int(capacity), _ptr(required), _ptr(ws), nbytes, _ptr(status),
                               _stream(stream)), "ps_bin_tiles")


def ps_fwd_workspace_bytes(frame: PsFrame) -> int:
    return int(load().ps_fwd_workspace_bytes(ctypes.byref(frame)))


def ps_splat_fwd(frame, settings, rec, key, tile_ptr, tile_ent, capacity, depth, normal, alpha,
                 ws, status, stream=None):
    nbytes = ws.numel() * ws.element_size()
    _check(load().ps_splat_fwd(ctypes.byref(frame), ctypes.byref(settings), _ptr(rec), _ptr(key),
                               _ptr(tile_ptr), _ptr(tile_ent), int(capacity), _ptr(depth),
                               _ptr(normal), _ptr(alpha), _ptr(ws), nbytes, _ptr(status),
                               _stream(stream)),
           "ps_splat_fwd")


def ps_splat_ids(frame, settings, rec, key, tile_ptr, tile_ent, capacity, ids, depth, ws, status,
                 stream=None):
    nbytes = ws.numel() * ws.element_size()
    _check(load().ps_splat_ids(ctypes.byref(frame), ctypes.byref(settings), _ptr(rec), _ptr(key),
                               _ptr(tile_ptr), _ptr(tile_ent), int(capacity), _ptr(ids), _ptr(depth),
                               _ptr(ws), nbytes, _ptr(status), _stream(stream)), "ps_splat_ids")


def ps_loss(frame, settings, depth, normal, gt_depth, gt_normal, dLdD, dLdN, view_sums, stream=None):
    _check(load().ps_loss(ctypes.byref(frame), ctypes.byref(settings), _ptr(depth), _ptr(normal),
                          _ptr(gt_depth), _ptr(gt_normal), _ptr(dLdD), _ptr(dLdN),
                          _ptr(view_sums), _stream(stream)), "ps_loss")


def ps_bwd_workspace_bytes(frame: PsFrame) -> int:
    return int(load().ps_bwd_workspace_bytes(ctypes.byref(frame)))


def ps_splat_bwd(planes, frame, settings, rec, key, tile_ptr, tile_ent, capacity, dLdD, dLdN,
                 g_center, g_quat, g_radii, ws, status, stream=None):
    nbytes = ws.numel() * ws.element_size()
    _check(load().ps_splat_bwd(ctypes.byref(planes), ctypes.byref(frame), ctypes.byref(settings),
                               _ptr(rec), _ptr(key), _ptr(tile_ptr), _ptr(tile_ent), int(capacity),
                               _ptr(dLdD), _ptr(dLdN), _ptr(g_center), _ptr(g_quat),
                               _ptr(g_radii), _ptr(ws), nbytes, _ptr(status), _stream(stream)),
           "ps_splat_bwd")


def ps_splat_fused(planes, frame, settings, rec, key, tile_ptr, tile_ent, capacity, gt_depth,
                   gt_normal, depth, normal, dLdD, dLdN, view_sums, g_center, g_quat, g_radii, ws,
                   status, stream=None):
    nbytes = ws.numel() * ws.element_size()
    _check(load().ps_splat_fused(ctypes.byref(planes), ctypes.byref(frame), ctypes.byref(settings),
                                 _ptr(rec), _ptr(key), _ptr(tile_ptr), _ptr(tile_ent),
                                 int(capacity), _ptr(gt_depth), _ptr(gt_normal), _ptr(depth),
                                 _ptr(normal), _ptr(dLdD), _ptr(dLdN), _ptr(view_sums),
                                 _ptr(g_center), _ptr(g_quat), _ptr(g_radii), _ptr(ws), nbytes,
                                 _ptr(status), _stream(stream)), "ps_splat_fused")


def ps_adam_step(param, grad, m, v, lr, b1, b2, eps, step, clamp_min=float("nan"), stream=None):
    _check(load().ps_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(),
                               float(lr), float(b1), float(b2), float(eps), int(step),
                               float(clamp_min), _stream(stream)), "ps_adam_step")


def ps_count_pairs(frame, settings, rec, key, tile_ptr, tile_ent, capacity, counts, stream=None):
    _check(load().ps_count_pairs(ctypes.byref(frame), ctypes.byref(settings), _ptr(rec), _ptr(key),
                                 _ptr(tile_ptr), _ptr(tile_ent), int(capacity), _ptr(counts),
                                 _stream(stream)), "ps_count_pairs")


def ps_step_advance(d_state, d_sched, n_sched, d_iter, stream=None):
    _check(load().ps_step_advance(_ptr(d_state), _ptr(d_sched), int(n_sched), _ptr(d_iter),
                                  _stream(stream)), "ps_step_advance")


def ps_adam_step_state(param, grad, m, v, lr, b1, b2, eps, d_state, clamp_min=float("nan"),
                       clamp_from=0, stream=None):
    _check(load().ps_adam_step_state(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(),
                                     float(lr), float(b1), float(b2), float(eps), _ptr(d_state),
                                     float(clamp_min), int(clamp_from), _stream(stream)),
           "ps_adam_step_state")


def ps_radii_grad_accum(g_radii, acc, scale=1.0, plane_scale=None, stream=None):
    """acc [P, 2] += per-axis mean |dL/dr| of g_radii [P, 4] (times scale or plane_scale[P])."""
    n = acc.numel() // 2
    _check(load().ps_radii_grad_accum(_ptr(g_radii), _ptr(plane_scale), float(scale), int(n),
                                      _ptr(acc), _stream(stream)), "ps_radii_grad_accum")


def ps_split_planes(params, m, v, plane_ptr, acc, n_iter, tau, params_out, m_out, v_out,
                    plane_ptr_out, capacity, split_rank, d_count, stream=None):
    """Sec. 3.3 plane splitting on device buffers (see ps.h)."""
    n_planes = acc.numel() // 2
    _check(load().ps_split_planes(_ptr(params), _ptr(m), _ptr(v), int(plane_ptr.numel() - 1),
                                  _ptr(plane_ptr), int(n_planes), _ptr(acc), int(n_iter), float(tau),
                                  _ptr(params_out), _ptr(m_out), _ptr(v_out), _ptr(plane_ptr_out),
                                  int(capacity), _ptr(split_rank), _ptr(d_count), _stream(stream)),
           "ps_split_planes")


def ps_merge_planes(params, n_planes, scene_center, max_angle_deg, max_offset, group_of,
                    rep_of_group, d_groups, stream=None):
    """Sec. 3.3 plane merge on device buffers (see ps.h); scene_center is 3 host floats."""
    c = (ctypes.c_float * 3)(*[float(x) for x in scene_center])
    _check(load().ps_merge_planes(_ptr(params), int(n_planes), c, float(max_angle_deg),
                                  float(max_offset), _ptr(group_of), _ptr(rep_of_group),
                                  _ptr(d_groups), _stream(stream)), "ps_merge_planes")


def ps_nn_distance(points, dist=None, radii=None, scale=0.5, r_lo=0.0, r_hi=float("inf"), ws=None,
                   stream=None):
    """Nearest-other-point distances of points [n, 3] (device f32) into dist [n]
    and/or the Sec. 3.1 initial radii clamp(scale * dist, r_lo, r_hi) into radii
    [n, 4]; scratch is allocated here when ws is None."""
    import torch
    n = int(points.shape[0])
    need = int(load().ps_nn_workspace_bytes(n))
    if ws is None:
        ws = torch.empty((need + 15) // 16 * 4, dtype=torch.float32, device=points.device)
    _check(load().ps_nn_distance(_ptr(points), n, float(scale), float(r_lo), float(r_hi), _ptr(dist),
                                 _ptr(radii), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "ps_nn_distance")


def ps_wait_selftest(status, polls: int, stream=None):
    """One bounded device wait that runs out (nothing arrives): ORs
    1 << PS_ERR_TIMEOUT into the status word (device int32)."""
    _check(load().ps_wait_selftest(_ptr(status), int(polls), _stream(stream)), "ps_wait_selftest")


def ps_gemm_bf16(A, B, bias, C32, C16, relu=False, accumulate=False, err=None, stream=None):
    """C = A . B^T (+ bias) (ReLU) on the tensor cores; A [M, K], B [N, K] bf16."""
    M, K = A.shape
    N = B.shape[0]
    C = C32 if C32 is not None else C16
    _check(load().ps_gemm_bf16(_ptr(A), _ptr(B), _ptr(bias), _ptr(C32), _ptr(C16), int(M), int(N),
                               int(K), int(C.stride(0)), int(bool(relu)), int(bool(accumulate)),
                               _ptr(err), _stream(stream)), "ps_gemm_bf16")


def ps_seed_im2col(x, B, H, W, C, Kp, A, stream=None):
    _check(load().ps_seed_im2col(_ptr(x), B, H, W, C, Kp, _ptr(A), _stream(stream)), "ps_seed_im2col")


def ps_seed_col2im(dA, B, H, W, C, Kp, dx, stream=None):
    _check(load().ps_seed_col2im(_ptr(dA), B, H, W, C, Kp, _ptr(dx), _stream(stream)), "ps_seed_col2im")


def ps_seed_relu_bwd(dy, y, scale, dz16=None, dz32=None, stream=None):
    _check(load().ps_seed_relu_bwd(_ptr(dy), _ptr(y), dy.numel(), float(scale), _ptr(dz16),
                                   _ptr(dz32), _stream(stream)), "ps_seed_relu_bwd")


def ps_seed_transpose(inp, out, R=None, stream=None):
    """out[c, r] = inp[r, c] for the 2-D tensor inp; out must be [C, ldo >= R]."""
    Rr, C = inp.shape
    R = Rr if R is None else R
    _check(load().ps_seed_transpose(_ptr(inp), int(inp.dtype != __import__("torch").float32), R, C,
                                    inp.stride(0), _ptr(out), out.stride(0), _stream(stream)),
           "ps_seed_transpose")


def ps_seed_colsum(dz, db, stream=None):
    R, C = dz.shape
    _check(load().ps_seed_colsum(_ptr(dz), R, C, _ptr(db), _stream(stream)), "ps_seed_colsum")


def ps_seed_pool(y, B, S, C, h32=None, h16=None, stream=None):
    _check(load().ps_seed_pool(_ptr(y), B, S, C, _ptr(h32), _ptr(h16), _stream(stream)), "ps_seed_pool")


def ps_seed_pool_bwd(dh, B, S, C, dy, stream=None):
    _check(load().ps_seed_pool_bwd(_ptr(dh), B, S, C, _ptr(dy), _stream(stream)), "ps_seed_pool_bwd")


def ps_seed_loss(out, tgt, B, slots, dout, sums=None, stream=None):
    _check(load().ps_seed_loss(_ptr(out), _ptr(tgt), B, slots, _ptr(dout), _ptr(sums),
                               _stream(stream)), "ps_seed_loss")


def ps_cast_bf16(inp, out, stream=None):
    R, Cin = inp.shape
    _check(load().ps_cast_bf16(_ptr(inp), R, Cin, out.shape[1], _ptr(out), _stream(stream)),
           "ps_cast_bf16")


def ps_status_string(code: int) -> str:
    return load().ps_status_string(int(code)).decode()


def ps_version() -> int:
    return int(load().ps_version())


def decode_status(word: int) -> list:
    """Names of the device status bits set in a status word."""
    return [ps_status_string(c) for c in range(1, 6) if word & (1 << c)]
