"""Seed-proposal network: a learned initialiser of the plane primitives.

The paper initialises planes from monocular depth (Sec. 3.1).  This network
maps a 64x64 patch of depth and camera-frame normals to up to 8 plane seeds
(centre, orientation, extents, confidence); seeds whose confidence is below 0.5
fall back to the plain initialisation.  It is trained on planes converged by
the splatting method itself.

Architecture: conv 3x3 stride 2 (4 -> 64) -> ReLU -> 3 x [conv 3x3 stride 2
(64 -> 64) -> ReLU] -> global average pool -> linear 64 -> 96.  Every
convolution is im2col + a tcgen05 BF16 GEMM with FP32 accumulation (libps);
the backward pass is the same kernels run on transposed operands.  Parameters
are FP32 masters (Adam in libps) with BF16 copies for the tensor cores.

Output slot j of a patch (12 floats): centre (u, v in [-1, 1] patch
coordinates, log(z / z_ref)), quaternion of the plane frame in camera
coordinates (normalised by the consumer), log(extent / z_ref) for x+, x-, y+,
y- and a confidence logit.  z_ref is the patch's median depth.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

PATCH = 64
CH = 64
SLOTS = 8
OUT = SLOTS * 12
IN_C = 4
# (H_in, C_in, Kp) of the four convolutions
LAYERS = [(64, IN_C, 64), (32, CH, 9 * CH), (16, CH, 9 * CH), (8, CH, 9 * CH)]


def param_shapes():
    shapes = []
    for (_, cin, _) in LAYERS:
        shapes += [("W", (CH, 9 * cin)), ("b", (CH,))]
    shapes += [("W", (OUT, CH)), ("b", (OUT,))]
    return shapes


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (confidence bias -2: seeds start unsure)."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, shp in param_shapes():
        if kind == "W":
            fan_in = shp[1]
            parts.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), size=shp).ravel())
        else:
            parts.append(np.zeros(shp))
    flat = np.concatenate(parts).astype(np.float32)
    # confidence logits of every slot
    o = flat.size - OUT
    flat[o + 11::12] = -2.0
    return flat


class SeedNet:
    """Forward, backward and Adam of the seed network on the GPU."""

    def __init__(self, device="cuda", seed: int = 0, params: np.ndarray | None = None):
        self.device = torch.device(device)
        p = init_params(seed) if params is None else np.asarray(params, np.float32)
        self.params = torch.from_numpy(p.copy()).to(self.device)
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        self.err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._views()
        self._bf16 = [torch.zeros((CH, kp), dtype=torch.bfloat16, device=self.device)
                      for (_, _, kp) in LAYERS] + [torch.zeros((OUT, CH), dtype=torch.bfloat16,
                                                               device=self.device)]
        self.B = 0

    def _views(self):
        self.W, self.b, self.gW, self.gb = [], [], [], []
        o = 0
        for kind, shp in param_shapes():
            n = int(np.prod(shp))
            (self.W if kind == "W" else self.b).append(self.params[o:o + n].view(*shp))
            (self.gW if kind == "W" else self.gb).append(self.grad[o:o + n].view(*shp))
            o += n

    def _alloc(self, Bn: int):
        if Bn == self.B:
            return
        assert Bn % 64 == 0, "batch must be a multiple of 64"
        dev, bf = self.device, torch.bfloat16
        self.B = Bn
        self.A, self.Y = [], []
        for (h, cin, kp) in LAYERS:
            ho = h // 2
            self.A.append(torch.empty((Bn * ho * ho, kp), dtype=bf, device=dev))
            self.Y.append(torch.empty((Bn * ho * ho, CH), dtype=bf, device=dev))
        self.h32 = torch.empty((Bn, CH), device=dev)
        self.h16 = torch.empty((Bn, CH), dtype=bf, device=dev)
        self.out = torch.empty((Bn, OUT), device=dev)
        self.dout = torch.empty((Bn, OUT), device=dev)
        self.loss_sums = torch.zeros(4, device=dev)

    def sync_weights(self):
        """BF16 copies of the FP32 master weights (zero-padded to the GEMM K)."""
        for i, (_, cin, kp) in enumerate(LAYERS):
            B.ps_cast_bf16(self.W[i], self._bf16[i])
        B.ps_cast_bf16(self.W[4], self._bf16[4])

    # -- forward -------------------------------------------------------------
    def forward(self, x16: torch.Tensor) -> torch.Tensor:
        """x16: [B, 64, 64, 4] bf16 (NHWC).  Returns out [B, 96] fp32."""
        Bn = x16.shape[0]
        self._alloc(Bn)
        self.x16 = x16
        inp = x16
        for i, (h, cin, kp) in enumerate(LAYERS):
            B.ps_seed_im2col(inp, Bn, h, h, cin, kp, self.A[i])
            B.ps_gemm_bf16(self.A[i], self._bf16[i], self.b[i], None, self.Y[i], relu=True, err=self.err)
            inp = self.Y[i]
        B.ps_seed_pool(self.Y[3], Bn, 16, CH, self.h32, self.h16)
        B.ps_gemm_bf16(self.h16, self._bf16[4], self.b[4], self.out, None, err=self.err)
        return self.out

    # -- backward ------------------------------------------------------------
    def backward(self, dout: torch.Tensor):
        """Gradient of sum(dout * out) w.r.t. every parameter, into self.grad."""
        Bn, dev, bf = self.B, self.device, torch.bfloat16
        f32 = torch.float32
        # linear layer
        doutT = torch.empty((OUT, Bn), dtype=bf, device=dev)
        hT = torch.empty((CH, Bn), dtype=bf, device=dev)
        B.ps_seed_transpose(dout, doutT)
        B.ps_seed_transpose(self.h16, hT)
        B.ps_gemm_bf16(doutT, hT, None, self.gW[4], None, err=self.err)
        B.ps_seed_colsum(dout, self.gb[4])
        dout16 = torch.empty((Bn, 128), dtype=bf, device=dev)
        B.ps_cast_bf16(dout, dout16)
        WfcT = torch.empty((CH, 128), dtype=bf, device=dev)
        B.ps_seed_transpose(self.W[4], WfcT)
        dh = torch.empty((Bn, CH), dtype=f32, device=dev)
        B.ps_gemm_bf16(dout16, WfcT, None, dh, None, err=self.err)
        # pooling + ReLU of the last convolution
        dy = torch.empty((Bn * 16, CH), dtype=f32, device=dev)
        B.ps_seed_pool_bwd(dh, Bn, 16, CH, dy)
        for i in range(3, -1, -1):
            h, cin, kp = LAYERS[i]
            P = self.Y[i].shape[0]
            dz16 = torch.empty((P, CH), dtype=bf, device=dev)
            dz32 = torch.empty((P, CH), dtype=f32, device=dev)
            B.ps_seed_relu_bwd(dy, self.Y[i], 1.0, dz16, dz32)
            dzT = torch.empty((CH, P), dtype=bf, device=dev)
            AT = torch.empty((kp, P), dtype=bf, device=dev)
            B.ps_seed_transpose(dz16, dzT)
            B.ps_seed_transpose(self.A[i], AT)
            gWp = torch.empty((CH, kp), dtype=f32, device=dev)
            B.ps_gemm_bf16(dzT, AT, None, gWp, None, err=self.err)
            self.gW[i].copy_(gWp[:, :9 * cin])
            B.ps_seed_colsum(dz32, self.gb[i])
            if i > 0:
                WT = torch.empty((kp, CH), dtype=bf, device=dev)
                B.ps_seed_transpose(self._bf16[i], WT)
                dA = torch.empty((P, kp), dtype=f32, device=dev)
                B.ps_gemm_bf16(dz16, WT, None, dA, None, err=self.err)
                hp = LAYERS[i - 1][0] // 2
                dy = torch.empty((Bn * hp * hp, CH), dtype=f32, device=dev)
                B.ps_seed_col2im(dA, Bn, h, h, cin, kp, dy)

    def loss_backward(self, tgt: torch.Tensor):
        """Set loss of the current outputs against tgt [B, 8, 12]; fills dout and
        backpropagates.  Returns the four loss sums (device)."""
        B.ps_seed_loss(self.out, tgt, self.B, SLOTS, self.dout, self.loss_sums)
        self.backward(self.dout)
        return self.loss_sums

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        B.ps_adam_step(self.params, self.grad, self.m, self.v, lr, b1, b2, eps, self.step_count)
        self.sync_weights()
