"""FP64 CPU oracle of PlanarSplatting's differentiable plane rendering.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The CUDA library never
loads it and shares no code with it; the two meet only through the seeded
input generators in ``paper_2412_03451_gb300.scenes``.

The arithmetic lives in ``ps_oracle.c`` (plain C, FP64, brute force over every
plane at every pixel, compiled with ``-ffp-contract=off``).  This module builds
that file with gcc, marshals numpy arrays into it and adds the few steps that
are plain definitions in numpy:

* ``lambda_schedule`` -- Eq. 10, lambda = min(20 exp(-(1 - 0.001 ite)), 300).
* ``filter_margin`` -- the distance delta outside the rectangle edge at which
  the splat weight 2 sigmoid(5 lambda m) of Eq. 7-8 falls to the filter
  threshold w_min of Sec. 3.2 ("Blending Composition").
* ``tile_lists`` -- per-tile lists of the planes whose binning rectangle covers
  the tile, sorted by (depth key, plane id): the near-to-far order of Sec. 3.2
  applied to a conservative per-plane key.
* ``total_loss`` -- Eq. 14 of the Eq. 11-13 render, for finite differences.

Parity: every function here is pinned by ``tests/test_oracle_pins.py`` to
closed forms, brute force on tiny inputs, invariants, a library routine (Adam
against ``torch.optim.Adam``) or central finite differences.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libps_oracle.so")
_lock = threading.Lock()
_lib = None

# Hyperparameters printed in the paper (Sec. 3.2 and Eq. 14, Sec. 3.3, App. A.2).
M_DEFAULT = 30          # nearest intersections kept per ray (Sec. 3.2)
W_MIN = 1e-4            # weights below this are filtered (Sec. 3.2)
ALPHA1 = 5.0            # normal terms of Eq. 14
ALPHA2 = 1.0            # depth term of Eq. 14
LR = 1e-3               # Adam learning rate for centers, radii, rotation (App. A.2)
Z_NEAR = 0.01           # not in the paper: near limit of a valid intersection
Z_FAR = 100.0           # not in the paper: far limit
R_MIN = 1e-3            # not in the paper: radii kept positive (Eq. 1 says R^4_+)


def build(force: bool = False) -> str:
    """Compile ps_oracle.c into a shared library (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            L = ctypes.c_long
            lib.or_bin_records.argtypes = [I, I, P, P, P, P, P, I, I, I, I, D, D, D, I, P, P, P]
            lib.or_records_ns.argtypes = [I, I, P, P, P, P, P]
            lib.or_render.argtypes = [I, I, P, P, P, P, P, I, I, D, D, D, D, I, I, D, D, D, D,
                                      I, I, P, P, P, P, P, P, P]
            lib.or_loss.argtypes = [I, I, I, P, P, P, P, D, D, D, P, P, P]
            lib.or_loss.restype = D
            lib.or_backward.argtypes = [I, I, P, P, P, P, P, I, I, D, D, D, D, I, I, P, P, P, P, P, P]
            lib.or_raycast.argtypes = [I, I, P, P, P, P, P, I, I, D, D, I, I, P, P, P]
            lib.or_adam.argtypes = [L, P, P, P, P, D, D, D, D, I, D]
            lib.or_num_threads.restype = I
            lib.or_set_num_threads.argtypes = [I]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (OpenMP)."""
    _load().or_set_num_threads(int(n))


# --------------------------------------------------------------------------
# Eq. 10 and the filter margin.

def lambda_schedule(ite: int) -> float:
    """Eq. 10: lambda = min(20 e^{-(1 - 0.001 ite)}, 300), ite counted from 0."""
    return min(20.0 * math.exp(-(1.0 - 0.001 * ite)), 300.0)


def filter_margin(lam: float, w_min: float = W_MIN) -> float:
    """delta > 0 with 2 sigmoid(-5 lam delta) = w_min (Eq. 7-8 and the 1e-4 filter)."""
    h = 0.5 * w_min
    return math.log((1.0 - h) / h) / (5.0 * lam)


def gauss_extent(w_min: float = W_MIN) -> float:
    """kappa with exp(-kappa^2 / 2) = w_min: the Gaussian weight of Eq. 5 passes the
    filter only within kappa sigma of the centre on each axis."""
    return math.sqrt(2.0 * math.log(1.0 / w_min))


def _flags(single_radii, gaussian) -> int:
    return (1 if single_radii else 0) | (4 if gaussian else 0)


# --------------------------------------------------------------------------
# Binning (per-plane screen bounds) and tile lists.

def bin_records(center, quat, radii, w2c, intr, H, W, tile_w, tile_h, delta,
                z_near=Z_NEAR, z_far=Z_FAR, single_radii=False, gaussian=False):
    """Tile rectangle and depth key of every (view, plane); see ps_oracle.c.
    The binning formula runs in FP32 on inputs rounded to float (delta
    included); key is the FP32 key as a double, key32 the same value.
    With gaussian, delta multiplies the radii (gauss_extent) instead of widening them."""
    c, q, r = _f64(center), _f64(quat), _f64(radii)
    Rt, K_ = _f64(w2c).reshape(-1, 12), _f64(intr).reshape(-1, 4)
    K, V = c.shape[0], Rt.shape[0]
    rect = np.zeros((V, K, 4), dtype=np.int32)
    key = np.zeros((V, K), dtype=np.float64)
    key32 = np.zeros((V, K), dtype=np.float32)
    _load().or_bin_records(K, V, _ptr(c), _ptr(q), _ptr(r), _ptr(Rt), _ptr(K_), H, W,
                           tile_w, tile_h, float(delta), float(z_near), float(z_far),
                           _flags(single_radii, gaussian), _ptr(rect), _ptr(key), _ptr(key32))
    return rect, key, key32


def records_ns(center, quat, radii, w2c):
    """f32 (n_c, n_c . p_c) of every (view, plane) record [V, K, 4], from the same
    FP32 operations as the bins (see ps_oracle.c)."""
    c, q, r = _f64(center), _f64(quat), _f64(radii)
    Rt = _f64(w2c).reshape(-1, 12)
    K, V = c.shape[0], Rt.shape[0]
    ns = np.zeros((V, K, 4), dtype=np.float32)
    _load().or_records_ns(K, V, _ptr(c), _ptr(q), _ptr(r), _ptr(Rt), _ptr(ns))
    return ns


def entry_keys(ns, intr, tx, ty, tile_w, tile_h, z_near=Z_NEAR, rec_key=None):
    """Entry keys of tile-list entries (records with f32 normal/offset ns [E, 4],
    intrinsics [E, 4], tile coordinates tx, ty [E]): the depth of the plane on
    the rays through the pixel centres at the tile's four corner pixels, all
    in f32 with correctly rounded + - * / (numpy float32, no contraction).  If
    the denominators d . n_c share one sign and are each > 0.01 of the sum of
    the magnitudes of their terms, c = max(min t, z_near), or +inf if
    max t <= z_near; otherwise c = z_near.  The key is max(c, rec_key) (the
    record's f32 quad key, if given): a lower bound of every depth the plane
    takes on a ray of the tile."""
    f32 = np.float32
    ns = np.asarray(ns, f32)
    intr = np.asarray(intr, f32)
    fx, fy, cx, cy = intr[:, 0], intr[:, 1], intr[:, 2], intr[:, 3]
    tx = np.asarray(tx, np.int64)
    ty = np.asarray(ty, np.int64)
    xs = [(tx * tile_w).astype(f32), (tx * tile_w + tile_w - 1).astype(f32)]
    ys = [(ty * tile_h).astype(f32), (ty * tile_h + tile_h - 1).astype(f32)]
    zn = f32(z_near)
    tmin = np.full(len(tx), np.inf, f32)
    tmax = np.full(len(tx), -np.inf, f32)
    npos = np.zeros(len(tx), np.int64)
    nneg = np.zeros(len(tx), np.int64)
    weak = np.zeros(len(tx), bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        for xa in xs:
            dx = ((xa + f32(0.5)) - cx) / fx
            for yb in ys:
                dy = ((yb + f32(0.5)) - cy) / fy
                p1 = ns[:, 0] * dx
                p2 = ns[:, 1] * dy
                den = (p1 + p2) + ns[:, 2]
                mag = (np.abs(p1) + np.abs(p2)) + np.abs(ns[:, 2])
                weak |= ~(np.abs(den) > f32(0.01) * mag)
                npos += den > 0
                nneg += den < 0
                t = ns[:, 3] / den
                tmin = np.fmin(tmin, t)
                tmax = np.fmax(tmax, t)
    key = np.where(tmax > zn, np.maximum(tmin, zn), f32(np.inf)).astype(f32)
    key = np.where(weak | ((npos != 4) & (nneg != 4)), zn, key).astype(f32)
    if rec_key is not None:
        key = np.maximum(key, np.asarray(rec_key, f32))
    return key


def tile_lists(rect, key32, ns, intr, H, W, tile_w, tile_h, z_near=Z_NEAR):
    """CSR tile lists: tiles numbered v*T + ty*tiles_x + tx, entries are record
    ids v*K + k with their entry keys (entry_keys with the record keys key32
    [V, K]), each list sorted by (key, record id).  ns [V, K, 4] from
    records_ns, intr [V, 4].  Returns (ptr, ent, key)."""
    V, K = rect.shape[0], rect.shape[1]
    tx_n = (W + tile_w - 1) // tile_w
    ty_n = (H + tile_h - 1) // tile_h
    T = tx_n * ty_n
    tiles, recs, txs, tys, vs = [], [], [], [], []
    for v in range(V):
        for k in range(K):
            x0, y0, x1, y1 = (int(a) for a in rect[v, k])
            if x1 < x0 or y1 < y0:
                continue
            for yy in range(y0, y1 + 1):
                for xx in range(x0, x1 + 1):
                    tiles.append(v * T + yy * tx_n + xx)
                    recs.append(v * K + k)
                    txs.append(xx); tys.append(yy); vs.append(v)
    tiles = np.asarray(tiles, dtype=np.int64)
    recs = np.asarray(recs, dtype=np.int64)
    if tiles.size:
        vs = np.asarray(vs)
        keys = entry_keys(ns.reshape(-1, 4)[recs], np.asarray(intr, np.float32).reshape(-1, 4)[vs],
                          np.asarray(txs), np.asarray(tys), tile_w, tile_h, z_near,
                          rec_key=np.asarray(key32, np.float32).reshape(-1)[recs])
    else:
        keys = np.zeros(0, np.float32)
    order = np.lexsort((recs, keys.view(np.uint32).astype(np.int64), tiles))
    counts = np.bincount(tiles, minlength=V * T) if tiles.size else np.zeros(V * T, np.int64)
    ptr = np.zeros(V * T + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(counts)
    return ptr.astype(np.int32), recs[order].astype(np.int32), keys[order]


# --------------------------------------------------------------------------
# Render, loss, backward.

def render(center, quat, radii, w2c, intr, H, W, lam, M=M_DEFAULT, w_min=W_MIN,
           z_near=Z_NEAR, z_far=Z_FAR, single_radii=False, eta=1e-6, tol_d=1e-4,
           tol_n=1e-5, rows=None, gaussian=False):
    """Brute-force forward of Eq. 11-13.  Returns a dict of per-pixel arrays:
    depth [V,H,W], normal [V,H,W,3], alpha, n_sel, n_cand, ill, and sens_d, sens_n
    (the first-order FP32 rounding sensitivity of D and N; see ps_oracle.c)."""
    c, q, r = _f64(center), _f64(quat), _f64(radii)
    Rt, K_ = _f64(w2c).reshape(-1, 12), _f64(intr).reshape(-1, 4)
    K, V = c.shape[0], Rt.shape[0]
    row0, row1 = (0, H) if rows is None else rows
    out = dict(depth=np.zeros((V, H, W)), normal=np.zeros((V, H, W, 3)),
               alpha=np.zeros((V, H, W)), n_sel=np.zeros((V, H, W), np.int32),
               n_cand=np.zeros((V, H, W), np.int32), ill=np.zeros((V, H, W), np.int32))
    sens = np.zeros((V, H, W, 2))
    delta = filter_margin(lam, w_min)
    _load().or_render(K, V, _ptr(c), _ptr(q), _ptr(r), _ptr(Rt), _ptr(K_), H, W,
                      float(lam), float(w_min), float(z_near), float(z_far), int(M),
                      _flags(single_radii, gaussian), float(delta), float(eta), float(tol_d),
                      float(tol_n), int(row0), int(row1),
                      _ptr(out["depth"]), _ptr(out["normal"]), _ptr(out["alpha"]),
                      _ptr(out["n_sel"]), _ptr(out["n_cand"]), _ptr(out["ill"]), _ptr(sens))
    out["sens_d"], out["sens_n"] = sens[..., 0], sens[..., 1]
    return out


def loss(depth, normal, gt_depth, gt_normal, a_cos=ALPHA1, a_l1n=ALPHA1, a_depth=ALPHA2):
    """Eq. 14 summed over pixels with gt_depth > 0.  Returns
    (total, dL/dD [V,H,W], dL/dN [V,H,W,3], view_sums [V,4])."""
    D, N = _f64(depth), _f64(normal)
    Dg, Ng = _f64(gt_depth), _f64(gt_normal)
    V, H, W = D.shape
    dD = np.zeros_like(D)
    dN = np.zeros_like(N)
    sums = np.zeros((V, 4))
    tot = _load().or_loss(V, H, W, _ptr(D), _ptr(N), _ptr(Dg), _ptr(Ng), float(a_cos),
                          float(a_l1n), float(a_depth), _ptr(dD), _ptr(dN), _ptr(sums))
    return float(tot), dD, dN, sums


def backward(center, quat, radii, w2c, intr, H, W, lam, dLdD, dLdN, M=M_DEFAULT,
             w_min=W_MIN, z_near=Z_NEAR, z_far=Z_FAR, single_radii=False, gaussian=False,
             with_abs=False):
    """Analytic FP64 gradient of sum(dLdD * D + dLdN . N) with respect to the
    plane centers [K,3], quaternions [K,4] and radii [K,4].  With with_abs, a fourth
    array [K,11] holds per plane and parameter the sum of the absolute per-pixel
    contributions (how much the sum cancels)."""
    c, q, r = _f64(center), _f64(quat), _f64(radii)
    Rt, K_ = _f64(w2c).reshape(-1, 12), _f64(intr).reshape(-1, 4)
    K, V = c.shape[0], Rt.shape[0]
    gD, gN = _f64(dLdD), _f64(dLdN)
    gc, gq, gr = np.zeros((K, 3)), np.zeros((K, 4)), np.zeros((K, 4))
    ga = np.zeros((K, 11)) if with_abs else None
    _load().or_backward(K, V, _ptr(c), _ptr(q), _ptr(r), _ptr(Rt), _ptr(K_), H, W,
                        float(lam), float(w_min), float(z_near), float(z_far), int(M),
                        _flags(single_radii, gaussian), _ptr(gD), _ptr(gN), _ptr(gc), _ptr(gq),
                        _ptr(gr), None if ga is None else _ptr(ga))
    if with_abs:
        return gc, gq, gr, ga
    return gc, gq, gr


def total_loss(center, quat, radii, w2c, intr, H, W, lam, gt_depth, gt_normal, **kw):
    """Scalar Eq. 14 loss of the Eq. 11-13 render (used for finite differences)."""
    out = render(center, quat, radii, w2c, intr, H, W, lam, **kw)
    return loss(out["depth"], out["normal"], gt_depth, gt_normal)[0]


def raycast(center, quat, radii, w2c, intr, H, W, z_near=Z_NEAR, z_far=Z_FAR, rows=None):
    """Exact hard-rectangle ray casting (ground truth for synthetic rooms).
    Only rows [rows[0], rows[1]) are cast when rows is given (others stay 0)."""
    c, q, r = _f64(center), _f64(quat), _f64(radii)
    Rt, K_ = _f64(w2c).reshape(-1, 12), _f64(intr).reshape(-1, 4)
    K, V = c.shape[0], Rt.shape[0]
    D = np.zeros((V, H, W))
    N = np.zeros((V, H, W, 3))
    pid = np.full((V, H, W), -1, np.int32)
    row0, row1 = (0, H) if rows is None else rows
    _load().or_raycast(K, V, _ptr(c), _ptr(q), _ptr(r), _ptr(Rt), _ptr(K_), H, W,
                       float(z_near), float(z_far), int(row0), int(row1), _ptr(D), _ptr(N),
                       _ptr(pid))
    return D, N, pid


def adam(param, grad, m, v, step, lr=LR, b1=0.9, b2=0.999, eps=1e-8, clamp_min=float("nan")):
    """In-place FP64 Adam step on flat arrays (returns them for convenience)."""
    p, g, mm, vv = (np.ascontiguousarray(a, dtype=np.float64) for a in (param, grad, m, v))
    _load().or_adam(p.size, _ptr(p), _ptr(g), _ptr(mm), _ptr(vv), float(lr), float(b1),
                    float(b2), float(eps), int(step), float(clamp_min))
    return p, mm, vv
