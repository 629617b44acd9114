"""Pins of the oracle's Gaussian splatting weight (Eq. 5, the ablation of
Sec. 3.2 / Fig. 4): a plane aligned with the camera axes renders the textbook
2D Gaussian of the pixel's in-plane offset, the filter keeps exactly the
pixels where it is >= 1e-4, the analytic adjoint matches central differences,
and the binning (radii times sqrt(2 ln 1e4)) contains every surviving pixel.
CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_03451_gb300 import scenes as S


def _cams(H=48, W=64, f=50.0):
    w2c = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)[None]
    intr = np.array([[f, f, W / 2.0, H / 2.0]])
    return w2c, intr


def test_aligned_plane_renders_the_textbook_gaussian():
    H, W, f = 48, 64, 50.0
    w2c, intr = _cams(H, W, f)
    Z, cx0, cy0 = 2.0, 0.1, -0.05
    r = np.array([0.3, 0.5, 0.2, 0.4])           # one-sided scales x+, x-, y+, y-
    out = O.render([[cx0, cy0, Z]], [[1, 0, 0, 0]], [r], w2c, intr, H, W, lam=20.0, gaussian=True)
    jj, ii = np.mgrid[0:H, 0:W]
    x = Z * (ii + 0.5 - W / 2.0) / f - cx0
    y = Z * (jj + 0.5 - H / 2.0) / f - cy0
    sx = np.where(x > 0, r[0], r[1])
    sy = np.where(y > 0, r[2], r[3])
    w = np.exp(-0.5 * (x * x / (sx * sx) + y * y / (sy * sy)))
    w = np.where(w >= 1e-4, w, 0.0)
    assert np.abs(out["depth"][0] - Z * w).max() < 1e-12
    assert np.abs(out["alpha"][0] - w).max() < 1e-12
    assert np.abs(out["normal"][0][..., 2] - w).max() < 1e-12
    assert (out["n_sel"][0] == (w > 0)).all()
    # lambda plays no part in Eq. 5
    out2 = O.render([[cx0, cy0, Z]], [[1, 0, 0, 0]], [r], w2c, intr, H, W, lam=300.0, gaussian=True)
    assert np.array_equal(out["depth"], out2["depth"])


def test_gauss_extent_is_the_filter_edge():
    k = O.gauss_extent()
    assert math.isclose(math.exp(-0.5 * k * k), 1e-4, rel_tol=1e-12)


def test_two_gaussian_planes_composite_by_hand():
    H, W, f = 8, 8, 10.0
    w2c, intr = _cams(H, W, f)
    # pixel (4, 4) looks along (0.05, 0.05, 1); two planes centred on that ray
    d = np.array([0.05, 0.05, 1.0])
    p1, p2 = 1.0 * d + [0.02, 0, 0], 2.0 * d + [0, -0.03, 0]
    r1, r2 = np.full(4, 0.1), np.full(4, 0.2)
    out = O.render([p1, p2], [[1, 0, 0, 0]] * 2, [r1, r2], w2c, intr, H, W, lam=20.0, gaussian=True)
    w1 = math.exp(-0.5 * (0.02 / 0.1) ** 2)
    w2 = math.exp(-0.5 * (0.03 / 0.2) ** 2)
    D = w1 * 1.0 + (1 - w1) * w2 * 2.0
    assert math.isclose(out["depth"][0, 4, 4], D, rel_tol=1e-12)


def _fd_check_gauss(seed, h=1e-6, rtol=2e-5):
    p = S.random_planes_in_view(seed, 6)
    cams = S.identity_cameras(2, 24, 32, 25.0, seed=seed, jitter=0.05)
    rng = np.random.default_rng(seed)
    V, H, W = cams.V, cams.H, cams.W
    gD = rng.normal(size=(V, H, W))
    gN = rng.normal(size=(V, H, W, 3))

    def J(c, q, r):
        o = O.render(c, q, r, cams.w2c, cams.intr, H, W, 20.0, gaussian=True)
        return float(np.sum(gD * o["depth"]) + np.sum(gN * o["normal"]))

    base = [p.center.astype(np.float64), p.quat.astype(np.float64) * 0.8,
            p.radii.astype(np.float64) * 0.5]
    gc, gq, gr = O.backward(*base, cams.w2c, cams.intr, H, W, 20.0, gD, gN, gaussian=True)
    an = np.concatenate([gc.ravel(), gq.ravel(), gr.ravel()])
    scale = np.abs(an).max()
    assert scale > 0
    fd = []
    for g in range(3):
        for i in range(base[g].size):
            plus = [b.copy() for b in base]
            minus = [b.copy() for b in base]
            plus[g].reshape(-1)[i] += h
            minus[g].reshape(-1)[i] -= h
            fd.append((J(*plus) - J(*minus)) / (2 * h))
    fd = np.array(fd)
    bad = np.abs(fd - an) > rtol * np.abs(an) + 1e-5 * scale
    assert not bad.any(), (np.nonzero(bad), fd[bad], an[bad])


@pytest.mark.parametrize("seed", [21, 22])
def test_gaussian_backward_matches_central_differences(seed):
    _fd_check_gauss(seed)


def test_gaussian_binning_covers_every_surviving_pair():
    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 2)
    init.radii *= 0.3                 # Gaussian scales: the support is ~4.3 sigma
    cams = room.cams
    tw, th = 8, 8
    rect, key, key32 = O.bin_records(init.center, init.quat, init.radii, cams.w2c, cams.intr,
                                     cams.H, cams.W, tw, th, O.gauss_extent(), gaussian=True)
    n_checked = 0
    for k in range(init.K):
        o = O.render(init.center[k:k + 1], init.quat[k:k + 1], init.radii[k:k + 1], cams.w2c,
                     cams.intr, cams.H, cams.W, 20.0, gaussian=True)
        for v in range(cams.V):
            vj, vi = np.nonzero(o["alpha"][v] > 0)
            if vj.size == 0:
                continue
            x0, y0, x1, y1 = rect[v, k]
            assert x1 >= x0 and y1 >= y0
            assert (vi // tw).min() >= x0 and (vi // tw).max() <= x1
            assert (vj // th).min() >= y0 and (vj // th).max() <= y1
            t = o["depth"][v][vj, vi] / o["alpha"][v][vj, vi]
            assert t.min() >= key[v, k] * (1 - 1e-12)
            n_checked += vj.size
    assert n_checked > 5000
