"""Pins of the seed-network oracle: im2col convolution against direct loops,
the adjoint against central finite differences, the set loss against finite
differences and closed forms."""
import numpy as np
import pytest

from oracle import seednet_oracle as SO


def direct_conv(x, W, b):
    """3x3, stride 2, padding 1 convolution by explicit loops; W [co, (ky, kx, ci)]."""
    Bn, H, Wd, C = x.shape
    co = W.shape[0]
    Wk = W.reshape(co, 3, 3, C)
    Ho, Wo = (H + 1) // 2, (Wd + 1) // 2
    y = np.zeros((Bn, Ho, Wo, co))
    for n in range(Bn):
        for oy in range(Ho):
            for ox in range(Wo):
                for ky in range(3):
                    for kx in range(3):
                        iy, ix = 2 * oy - 1 + ky, 2 * ox - 1 + kx
                        if 0 <= iy < H and 0 <= ix < Wd:
                            y[n, oy, ox] += Wk[:, ky, kx, :] @ x[n, iy, ix]
    return y + b


def test_im2col_convolution_equals_direct_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 6, 3))
    W = rng.normal(size=(5, 27))
    b = rng.normal(size=5)
    y = (SO.im2col(x) @ W.T + b).reshape(2, 4, 3, 5)
    assert np.allclose(y, direct_conv(x, W, b), atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 8, 8, 3))
    g = rng.normal(size=SO.im2col(x).shape)
    lhs = (SO.im2col(x) * g).sum()
    rhs = (x * SO.col2im(g, x.shape)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _tiny(seed):
    rng = np.random.default_rng(seed)
    cin, ch, out = 3, 6, 12
    n = 0
    c = cin
    for _ in range(4):
        n += ch * 9 * c + ch
        c = ch
    n += out * ch + out
    params = rng.normal(0, 0.5, size=n)
    x = rng.normal(size=(2, 16, 16, cin))
    return params, x, cin, ch, out


def test_backward_matches_central_differences():
    params, x, cin, ch, out = _tiny(2)
    rng = np.random.default_rng(3)
    dout = rng.normal(size=(2, out))
    o, cache = SO.forward(params, x, cin, ch, out, bf16_acts=False)
    g = SO.backward(params, cache, dout, cin, ch, out)
    h = 1e-6
    idx = rng.choice(params.size, size=60, replace=False)
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        f1 = (SO.forward(p1, x, cin, ch, out, bf16_acts=False)[0] * dout).sum()
        f2 = (SO.forward(p2, x, cin, ch, out, bf16_acts=False)[0] * dout).sum()
        fd = (f1 - f2) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-7), i


def test_backward_with_bf16_gradient_operands():
    # rounding the products' upstream gradients to bf16 (unit roundoff 2^-8) moves each
    # parameter block by a few roundoffs of the exact (finite-difference-pinned) gradient;
    # with a bf16-exact dout the linear layer's gradients do not move at all
    params, x, cin, ch, out = _tiny(5)
    rng = np.random.default_rng(6)
    dout = SO.bf16_round(rng.normal(size=(2, out)))
    o, cache = SO.forward(params, x, cin, ch, out, bf16_acts=False)
    g = SO.backward(params, cache, dout, cin, ch, out)
    gr = SO.backward(params, cache, dout, cin, ch, out, bf16_grads=True)
    n_fc = out * ch + out
    assert np.array_equal(g[-n_fc:], gr[-n_fc:])
    o_ = 0
    c = cin
    moved = 0
    for _ in range(4):
        for n in (ch * 9 * c, ch):
            a, b = gr[o_:o_ + n], g[o_:o_ + n]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel < 4 * 2.0 ** -8, rel
            moved += rel > 0
            o_ += n
        c = ch
    assert moved >= 4


def test_seed_loss_gradient_and_closed_forms():
    rng = np.random.default_rng(4)
    Bn, S = 3, 8
    o = rng.normal(size=(Bn, S * 12))
    tgt = np.zeros((Bn, S, 12))
    tgt[..., 0] = rng.integers(0, 2, size=(Bn, S))
    tgt[..., 1:4] = rng.normal(size=(Bn, S, 3))
    q = rng.normal(size=(Bn, S, 4))
    tgt[..., 4:8] = q / np.linalg.norm(q, axis=-1, keepdims=True)
    tgt[..., 8:12] = rng.normal(size=(Bn, S, 4))
    L, d, sums = SO.seed_loss(o, tgt)
    h = 1e-7
    for i in rng.choice(o.size, size=40, replace=False):
        e = np.zeros_like(o).ravel()
        e[i] = h
        e = e.reshape(o.shape)
        fd = (SO.seed_loss(o + e, tgt)[0] - SO.seed_loss(o - e, tgt)[0]) / (2 * h)
        assert fd == pytest.approx(d.ravel()[i], rel=1e-5, abs=1e-8)
    # a perfect prediction with a confident logit costs only the BCE of the logit
    perfect = np.zeros((1, S * 12))
    t1 = np.zeros((1, S, 12))
    t1[0, :, 0] = 1
    t1[0, :, 4] = 1                      # identity quaternion
    perfect.reshape(1, S, 12)[0, :, 3] = 2.0   # any positive scale of the same quaternion
    perfect.reshape(1, S, 12)[0, :, 11] = 30.0
    Lp, _, sp = SO.seed_loss(perfect, t1)
    assert sp[1] == 0 and sp[2] == pytest.approx(0, abs=1e-10) and sp[3] == 0
    assert Lp == pytest.approx(S * np.log1p(np.exp(-30.0)), abs=1e-10)


def test_bf16_rounding_ties_to_even():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: rounds to even (1)
    assert SO.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert SO.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert SO.bf16_round(np.array([1.0 + 2 ** -7]))[0] == 1.0 + 2 ** -7
