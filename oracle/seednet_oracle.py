"""FP64 reference of the seed-proposal network and its set loss.

TEST INFRASTRUCTURE ONLY (imported by tests and the smoke check).  Shares no
code with the CUDA path.  Shapes are generic (any patch size divisible by 16,
any channel count) so that the pins can use tiny networks.

Network: 4 x [conv 3x3, stride 2, padding 1, ReLU] -> global mean pool ->
linear.  Convolutions are written as im2col + matmul (a library primitive) and
pinned below against direct loops.  Stored activations may be rounded to bf16
(round to nearest even) to take the same decisions as the GPU, which keeps its
activations in bf16; arithmetic is FP64.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP64/FP32 values to the nearest bf16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def im2col(x: np.ndarray) -> np.ndarray:
    """x [B, H, W, C] -> [B*Ho*Wo, 9C], columns ordered (ky, kx, c); stride 2, pad 1."""
    Bn, H, W, C = x.shape
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    xp = np.zeros((Bn, H + 2, W + 2, C))
    xp[:, 1:H + 1, 1:W + 1] = x
    cols = []
    for ky in range(3):
        for kx in range(3):
            cols.append(xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :])
    return np.concatenate(cols, axis=-1).reshape(Bn * Ho * Wo, 9 * C)


def col2im(dA: np.ndarray, shape) -> np.ndarray:
    """Adjoint of im2col."""
    Bn, H, W, C = shape
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    d = dA.reshape(Bn, Ho, Wo, 9, C)
    dxp = np.zeros((Bn, H + 2, W + 2, C))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :] += d[:, :, :, ky * 3 + kx, :]
    return dxp[:, 1:H + 1, 1:W + 1]


def split(params: np.ndarray, cin: int, ch: int, out: int, n_conv: int = 4):
    """Flat parameters -> list of (W [ch, 9 cin'], b [ch]) and (Wfc [out, ch], bfc)."""
    p = np.asarray(params, np.float64)
    o = 0
    layers = []
    c = cin
    for _ in range(n_conv):
        W = p[o:o + ch * 9 * c].reshape(ch, 9 * c); o += ch * 9 * c
        b = p[o:o + ch]; o += ch
        layers.append((W, b))
        c = ch
    Wfc = p[o:o + out * ch].reshape(out, ch); o += out * ch
    bfc = p[o:o + out]; o += out
    assert o == p.size
    return layers, (Wfc, bfc)


def forward(params, x, cin=4, ch=64, out=96, bf16_acts=True):
    """x [B, H, W, cin].  Returns (out [B, out], cache)."""
    layers, (Wfc, bfc) = split(params, cin, ch, out)
    rnd = bf16_round if bf16_acts else (lambda a: a)
    if bf16_acts:
        layers = [(bf16_round(W), b) for W, b in layers]
        Wfc = bf16_round(Wfc)
    a = rnd(np.asarray(x, np.float64))
    cache = []
    for W, b in layers:
        Bn, H, Wd, C = a.shape
        A = im2col(a)
        y = np.maximum(A @ W.T + b, 0.0)
        y = rnd(y)
        cache.append((a.shape, A, y))
        a = y.reshape(Bn, (H + 1) // 2, (Wd + 1) // 2, ch)
    h = a.reshape(a.shape[0], -1, ch).mean(axis=1)
    h = rnd(h)
    o = h @ Wfc.T + bfc
    return o, dict(layers=layers, Wfc=Wfc, h=h, cache=cache, last=a)


def backward(params, fwd_cache, dout, cin=4, ch=64, out=96, bf16_grads=False):
    """Gradient of sum(dout * out) w.r.t. the flat parameters.

    With bf16_grads, the upstream gradient of every matrix product (dout, and
    each layer's gradient behind its ReLU) is rounded to bf16 before it enters
    the product, as on a tensor-core path whose operands are bf16; the bias
    gradients sum the unrounded values.  Arithmetic stays FP64."""
    c = fwd_cache
    layers, Wfc, h = c["layers"], c["Wfc"], c["h"]
    rnd = bf16_round if bf16_grads else (lambda a: a)
    grads = []
    dout_m = rnd(dout)
    gWfc = dout_m.T @ h
    gbfc = dout.sum(axis=0)
    dh = dout_m @ Wfc
    last = c["last"]
    Bn, Ho, Wo, _ = last.shape
    dy = np.repeat(dh[:, None, :] / (Ho * Wo), Ho * Wo, axis=1).reshape(-1, ch)
    conv_grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        shape, A, y = c["cache"][i]
        dz = dy * (y > 0)
        dz_m = rnd(dz)
        gW = dz_m.T @ A
        gb = dz.sum(axis=0)
        conv_grads.append((gW, gb))
        if i > 0:
            dA = dz_m @ W
            dy = col2im(dA, shape).reshape(-1, shape[-1])
    conv_grads.reverse()
    for gW, gb in conv_grads:
        grads += [gW.ravel(), gb]
    grads += [gWfc.ravel(), gbfc]
    return np.concatenate(grads)


def seed_loss(o: np.ndarray, tgt: np.ndarray, slots: int = 8):
    """Set loss per slot (mean over the batch) and its gradient w.r.t. o.
    o [B, slots*12]: centre 3, quaternion 4, log extents 4, confidence logit.
    tgt [B, slots, 12]: valid, centre 3, unit quaternion 4, log extents 4."""
    Bn = o.shape[0]
    O = o.reshape(Bn, slots, 12)
    d = np.zeros_like(O)
    valid = tgt[..., 0]
    z = O[..., 11]
    bce = np.maximum(z, 0) - z * valid + np.log1p(np.exp(-np.abs(z)))
    d[..., 11] = 1.0 / (1.0 + np.exp(-z)) - valid
    ec = O[..., 0:3] - tgt[..., 1:4]
    q = O[..., 3:7]
    qn = np.linalg.norm(q, axis=-1, keepdims=True) + 1e-12
    qh = q / qn
    dot = (qh * tgt[..., 4:8]).sum(-1)
    ee = O[..., 7:11] - tgt[..., 8:12]
    v = valid[..., None]
    lc = np.abs(ec).sum(-1) * valid
    lq = (1.0 - np.abs(dot)) * valid
    le = 0.5 * np.abs(ee).sum(-1) * valid
    d[..., 0:3] = np.sign(ec) * v
    gqh = -np.sign(dot)[..., None] * tgt[..., 4:8]
    proj = (gqh * qh).sum(-1, keepdims=True)
    d[..., 3:7] = (gqh - qh * proj) / qn * v
    d[..., 7:11] = 0.5 * np.sign(ee) * v
    total = (bce.sum() + lc.sum() + lq.sum() + le.sum()) / Bn
    return total, d.reshape(Bn, -1) / Bn, np.array([bce.sum(), lc.sum(), lq.sum(), le.sum()])
