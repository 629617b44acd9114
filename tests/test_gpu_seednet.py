"""Seed network on the GPU (tcgen05 GEMMs + libps kernels) against the FP64 oracle.

The oracle stores activations in bf16 like the kernels, rounds the gradients
that enter the backward matrix products to bf16 as the kernels do, and computes
in FP64.  What remains is FP32 accumulation and the bf16 roundings that its
small differences send the other way.  A bf16 rounding moves a value by at most
u = 2^-9 of itself, and a value crosses at most four of them (one per layer) on
its way to the output or, backwards, to the first layer's weights: the bar is
4u = 7.8e-3 relative per block, the first-order effect of one unmatched rounding
per layer.  Measured: output 3.7e-4, gradient blocks 4e-4 (linear layer) to
2.0e-3 (first layer, the end of the longest chain), 1 - cosine <= 2e-6 (against
the oracle without its rounding of the gradients: 1.4e-3 to 4.1e-3).  Wrong
operands, layouts or layers give errors of order one."""
REL_BAR = 4 * 2.0 ** -9
import numpy as np
import pytest

from oracle import seednet_oracle as SO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _inputs(seed, Bn=64):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(Bn, 64, 64, 4)).astype(np.float32)
    x = SO.bf16_round(x).astype(np.float32)
    tgt = np.zeros((Bn, 8, 12), np.float32)
    tgt[..., 0] = rng.integers(0, 2, size=(Bn, 8))
    tgt[..., 1:4] = rng.normal(size=(Bn, 8, 3))
    q = rng.normal(size=(Bn, 8, 4))
    tgt[..., 4:8] = q / np.linalg.norm(q, axis=-1, keepdims=True)
    tgt[..., 8:12] = rng.normal(size=(Bn, 8, 4))
    return x, tgt


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_backward_and_loss_match_oracle(torch):
    from paper_2412_03451_gb300 import seednet as SN
    net = SN.SeedNet(seed=3)
    net.sync_weights()
    x, tgt = _inputs(5)
    x16 = torch.from_numpy(x).cuda().bfloat16()
    out = net.forward(x16).clone()
    torch.cuda.synchronize()
    params = net.params.cpu().numpy().astype(np.float64)
    o_ref, cache = SO.forward(params, x)
    assert int(net.err.item()) == 0
    assert _rel(out.cpu().numpy(), o_ref) < REL_BAR
    # backward with one upstream gradient on both sides
    rng = np.random.default_rng(6)
    dout = rng.normal(size=o_ref.shape).astype(np.float32)
    net.grad.zero_()
    net.backward(torch.from_numpy(dout).cuda())
    torch.cuda.synchronize()
    g = net.grad.cpu().numpy().astype(np.float64)
    g_ref = SO.backward(params, cache, dout.astype(np.float64), bf16_grads=True)
    o = 0
    for kind, shp in SN.param_shapes():
        n = int(np.prod(shp))
        a, b = g[o:o + n], g_ref[o:o + n]
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert cos > 0.99999 and _rel(a, b) < REL_BAR, (kind, shp, cos, _rel(a, b))
        o += n
    # set loss on the GPU's own outputs
    t = torch.from_numpy(tgt).cuda()
    sums = net.loss_backward(t)
    torch.cuda.synchronize()
    L, d_ref, s_ref = SO.seed_loss(out.cpu().numpy().astype(np.float64), tgt.astype(np.float64))
    assert np.allclose(sums.cpu().numpy(), s_ref, rtol=1e-4)
    assert _rel(net.dout.cpu().numpy(), d_ref) < 1e-5


def test_training_reduces_loss(torch):
    from paper_2412_03451_gb300 import seednet as SN
    net = SN.SeedNet(seed=1)
    net.sync_weights()
    x, tgt = _inputs(7)
    x16 = torch.from_numpy(x).cuda().bfloat16()
    t = torch.from_numpy(tgt).cuda()
    losses = []
    for it in range(60):
        net.forward(x16)
        net.grad.zero_()
        s = net.loss_backward(t)
        losses.append(float(s.sum().item()))
        net.adam(lr=3e-3)
    assert losses[-1] < 0.7 * losses[0], losses[::10]
