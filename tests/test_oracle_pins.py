"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test states which passage of the paper (arxiv 2412.03451) it checks and
against what: a closed form derived here independently, brute force on a tiny
input, an invariant of Eq. 11-13, a library routine, or central finite
differences.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_03451_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def ident_cams(V=1, H=96, W=128, f=100.0):
    w2c = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1), (V, 1, 1))
    intr = np.tile(np.array([f, f, W / 2.0, H / 2.0]), (V, 1))
    return w2c, intr


def rot_z_quat(theta):
    return np.array([math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2)])


def plane(center, quat, radii):
    return (np.asarray(center, float)[None], np.asarray(quat, float)[None],
            np.asarray(radii, float)[None])


def cat(*ps):
    return tuple(np.concatenate([p[i] for p in ps], axis=0) for i in range(3))


def pix_ray(i, j, f, cx, cy):
    return (i + 0.5 - cx) / f, (j + 0.5 - cy) / f


# ---------------------------------------------------------------------------
# Constants printed in the paper.

def test_paper_constants_match_golden():
    g = json.load(open(GOLDEN))
    assert O.M_DEFAULT == g["M"]["value"]
    assert O.W_MIN == g["w_min"]["value"]
    assert O.ALPHA1 == g["alpha1"]["value"] and O.ALPHA2 == g["alpha2"]["value"]
    assert O.LR == g["lr"]["value"]
    for ite, lam in g["lambda_at"]["value"].items():
        assert O.lambda_schedule(int(ite)) == pytest.approx(lam, rel=1e-12)


def test_lambda_schedule_endpoints():
    # Eq. 10: 20/e at ite 0, 20 at ite 1000, capped at 300 from ite ~3708 on
    assert O.lambda_schedule(0) == pytest.approx(20.0 / math.e, rel=1e-15)
    assert O.lambda_schedule(1000) == pytest.approx(20.0, rel=1e-15)
    assert O.lambda_schedule(3708) < 300.0
    assert O.lambda_schedule(3709) == 300.0
    assert O.lambda_schedule(5000) == 300.0


def test_filter_margin_against_library_sigmoid():
    from scipy.special import expit
    for lam in (7.36, 20.0, 300.0):
        d = O.filter_margin(lam)
        assert 2.0 * expit(-5.0 * lam * d) == pytest.approx(1e-4, rel=1e-12)


# ---------------------------------------------------------------------------
# Eq. 4 and Eq. 11-12: closed forms.

@pytest.mark.parametrize("lam", [7.36, 20.0, 300.0])
def test_fronto_parallel_plane_constant_depth_and_normal(lam):
    H, W, f = 48, 64, 50.0
    w2c, intr = ident_cams(2, H, W, f)
    w2c[1, :, 3] = [0.1, -0.2, 0.0]          # a translated second view
    c, q, r = plane([0.3, -0.1, 2.5], [1, 0, 0, 0], [100, 100, 100, 100])
    out = O.render(c, q, r, w2c, intr, H, W, lam)
    assert np.abs(out["depth"] - 2.5).max() < 1e-12          # z-depth, not ray length
    assert np.abs(out["normal"] - np.array([0, 0, 1.0])).max() < 1e-12
    assert np.abs(out["alpha"] - 1.0).max() < 1e-15
    assert (out["n_sel"] == 1).all()


def test_tilted_plane_depth_matches_plane_equation():
    # camera-frame plane z = a x + b y + c; along the ray t (dx, dy, 1):
    # t = a t dx + b t dy + c  =>  t = c / (1 - a dx - b dy)
    H, W, f = 24, 32, 40.0
    a, b, c0 = 0.3, -0.2, 3.0
    n = np.array([-a, -b, 1.0]) / np.linalg.norm([-a, -b, 1.0])
    vx = np.cross([0.0, 1.0, 0.0], n)
    vx /= np.linalg.norm(vx)
    vy = np.cross(n, vx)
    q = S.quat_from_frame(vx, vy, n)
    w2c, intr = ident_cams(1, H, W, f)
    out = O.render(*plane([0, 0, c0], q, [50, 50, 50, 50]), w2c, intr, H, W, 20.0)
    jj, ii = np.mgrid[0:H, 0:W]
    dx, dy = pix_ray(ii, jj, f, W / 2, H / 2)
    expect = c0 / (1 - a * dx - b * dy)
    assert np.abs(out["depth"][0] - expect).max() < 1e-11
    assert np.abs(out["normal"][0] - n).max() < 1e-12


def test_quaternion_x_axis_follows_textbook_rotation():
    # Eq. 2: v^x = R(q)[1,0,0]^T.  A rotation by theta about z maps e_x to
    # (cos theta, sin theta, 0).  One-sided radii make the footprint asymmetric
    # so a transposed or sign-flipped rotation fails.
    H, W, f, Z, th = 96, 128, 100.0, 2.0, math.radians(30)
    rxp, rxm, ry = 0.6, 0.1, 0.05
    lam = 300.0
    d = O.filter_margin(lam)
    w2c, intr = ident_cams(1, H, W, f)
    out = O.render(*plane([0, 0, Z], rot_z_quat(th), [rxp, rxm, ry, ry]), w2c, intr, H, W, lam)
    jj, ii = np.mgrid[0:H, 0:W]
    dx, dy = pix_ray(ii, jj, f, W / 2, H / 2)
    X, Y = Z * dx, Z * dy
    PX = X * math.cos(th) + Y * math.sin(th)
    PY = -X * math.sin(th) + Y * math.cos(th)
    mX = np.where(PX > 0, rxp, rxm) - np.abs(PX)
    mY = ry - np.abs(PY)
    m = np.minimum(mX, mY)
    alpha = out["alpha"][0]
    assert (m > 0).sum() > 50
    assert np.all(alpha[m > 0] == 1.0)
    assert np.all(alpha[m < -1.5 * d] == 0.0)


# ---------------------------------------------------------------------------
# Eq. 7-9 and the 1e-4 filter: closed forms from the threshold definition.

def _band_pixel_setup(lam, Z=2.0, i0=100, j0=48, H=96, W=128, f=100.0, frac=0.5):
    d = O.filter_margin(lam)
    dx, dy = pix_ray(i0, j0, f, W / 2, H / 2)
    X0 = Z * dx
    rx = X0 - frac * d
    return d, X0, rx


def test_edge_band_weight_closed_form():
    # at margin m = -delta/2: e^{5 lam delta} = (1-h)/h with h = w_min/2, so
    # w = 2 sigmoid(-5 lam delta/2) = 2 / (1 + sqrt(19999))
    lam, Z, i0, j0 = 50.0, 2.0, 100, 48
    d, X0, rx = _band_pixel_setup(lam, Z, i0, j0)
    w2c, intr = ident_cams(1)
    out = O.render(*plane([0, 0, Z], [1, 0, 0, 0], [rx, 1.0, 0.5, 0.5]), w2c, intr, 96, 128, lam)
    w_expect = 2.0 / (1.0 + math.sqrt(19999.0))
    assert out["alpha"][0, j0, i0] == pytest.approx(w_expect, rel=1e-10)
    assert out["depth"][0, j0, i0] == pytest.approx(w_expect * Z, rel=1e-10)
    # three pixels further out the margin is below -delta: filtered to exactly 0
    assert out["alpha"][0, j0, i0 + 3] == 0.0
    # one pixel inside the edge the weight is clamped to exactly 1
    assert out["alpha"][0, j0, i0 - 1] == 1.0


def test_filter_threshold_is_inclusive_side():
    lam, Z, i0, j0 = 50.0, 2.0, 100, 48
    d, X0, _ = _band_pixel_setup(lam, Z, i0, j0)
    w2c, intr = ident_cams(1)
    below = O.render(*plane([0, 0, Z], [1, 0, 0, 0], [X0 - d * (1 + 1e-6), 1, .5, .5]),
                     w2c, intr, 96, 128, lam)
    above = O.render(*plane([0, 0, Z], [1, 0, 0, 0], [X0 - d * (1 - 1e-6), 1, .5, .5]),
                     w2c, intr, 96, 128, lam)
    assert below["alpha"][0, j0, i0] == 0.0
    assert above["alpha"][0, j0, i0] == pytest.approx(1e-4, rel=1e-4)


def test_min_of_two_sides():
    # Eq. 9 takes the smaller side weight: margins -delta/2 on X and -delta/4 on Y
    lam, Z, i0, j0 = 50.0, 2.0, 100, 70
    H, W, f = 96, 128, 100.0
    d = O.filter_margin(lam)
    dx, dy = pix_ray(i0, j0, f, W / 2, H / 2)
    rx, ry = Z * dx - 0.5 * d, Z * dy - 0.25 * d
    w2c, intr = ident_cams(1)
    out = O.render(*plane([0, 0, Z], [1, 0, 0, 0], [rx, 1, ry, 1]), w2c, intr, H, W, lam)
    w_expect = 2.0 / (1.0 + math.sqrt(19999.0))          # the X side
    assert out["alpha"][0, j0, i0] == pytest.approx(w_expect, rel=1e-10)


# ---------------------------------------------------------------------------
# Eq. 11-13: compositing by hand, top-M, invariants.

def test_two_planes_by_hand():
    lam, i0, j0 = 50.0, 100, 48
    Z1, Z2 = 1.5, 3.0
    d, X0, rx = _band_pixel_setup(lam, Z1, i0, j0)
    near = plane([0, 0, Z1], [1, 0, 0, 0], [rx, 1.0, 0.5, 0.5])         # n = +z
    far = plane([0, 0, Z2], [0, 1, 0, 0], [50, 50, 50, 50])              # 180 deg about x: n = -z
    w2c, intr = ident_cams(1)
    out = O.render(*cat(near, far), w2c, intr, 96, 128, lam)
    w1 = 2.0 / (1.0 + math.sqrt(19999.0))
    assert out["depth"][0, j0, i0] == pytest.approx(w1 * Z1 + (1 - w1) * Z2, rel=1e-10)
    assert out["normal"][0, j0, i0, 2] == pytest.approx(w1 - (1 - w1), rel=1e-10)
    assert out["alpha"][0, j0, i0] == pytest.approx(1.0, abs=1e-14)
    # where the near plane is opaque (w = 1) the far one is invisible
    assert out["depth"][0, j0, 64] == pytest.approx(Z1, rel=1e-14)


def _stack(n, lam, i0=100, j0=48, z0=1.0, dz=0.05, frac=0.5):
    ps = []
    for j in range(n):
        Z = z0 + dz * j
        _, _, rx = _band_pixel_setup(lam, Z, i0, j0, frac=frac)
        ps.append(plane([0, 0, Z], [1, 0, 0, 0], [rx, 1.0, 0.5, 0.5]))
    return cat(*ps)


def test_top_m_keeps_only_the_nearest_30():
    lam, i0, j0 = 50.0, 100, 48
    w0 = 2.0 / (1.0 + math.sqrt(19999.0))
    planes40 = _stack(40, lam)
    w2c, intr = ident_cams(1)
    o30 = O.render(*planes40, w2c, intr, 96, 128, lam, M=30)
    o40 = O.render(*planes40, w2c, intr, 96, 128, lam, M=40)
    Zs = 1.0 + 0.05 * np.arange(40)
    Tj = (1 - w0) ** np.arange(40)
    assert o30["depth"][0, j0, i0] == pytest.approx(np.sum(Tj[:30] * w0 * Zs[:30]), rel=1e-12)
    assert o30["alpha"][0, j0, i0] == pytest.approx(1 - (1 - w0) ** 30, rel=1e-12)
    assert o40["alpha"][0, j0, i0] == pytest.approx(1 - (1 - w0) ** 40, rel=1e-12)
    assert o30["n_cand"][0, j0, i0] == 40 and o30["n_sel"][0, j0, i0] == 30
    # removing the 10 farthest planes does not change the M = 30 render
    near30 = tuple(a[:30] for a in planes40)
    o_near = O.render(*near30, w2c, intr, 96, 128, lam, M=30)
    assert np.array_equal(o_near["depth"], o30["depth"])
    assert np.array_equal(o_near["normal"], o30["normal"])


def test_top_m_of_thousands_of_candidates_keeps_the_nearest():
    # Sec. 3.2 keeps the M nearest intersections of a ray, however many pass the
    # filter.  5,000 stacked planes all pass at one pixel with the same band weight
    # w0; plane j sits at Z = 6 - 0.001 j, so the nearest 30 have the highest
    # indices.  A gather that stopped early in plane-index order would keep the
    # farthest planes instead and miss this geometric series.
    lam, i0, j0, n = 50.0, 100, 48, 5000
    w0 = 2.0 / (1.0 + math.sqrt(19999.0))
    Zs = 6.0 - 0.001 * np.arange(n)
    ps = []
    for Z in Zs:
        _, _, rx = _band_pixel_setup(lam, Z, i0, j0)
        ps.append(plane([0, 0, Z], [1, 0, 0, 0], [rx, 1.0, 0.5, 0.5]))
    planes = cat(*ps)
    w2c, intr = ident_cams(1)
    o = O.render(*planes, w2c, intr, 96, 128, lam, M=30, rows=(j0, j0 + 1))
    near = np.sort(Zs)[:30]
    Tj = (1 - w0) ** np.arange(30)
    assert o["n_cand"][0, j0, i0] == n and o["n_sel"][0, j0, i0] == 30
    assert o["depth"][0, j0, i0] == pytest.approx(np.sum(Tj * w0 * near), rel=1e-12)
    assert o["alpha"][0, j0, i0] == pytest.approx(1 - (1 - w0) ** 30, rel=1e-12)
    # the backward differentiates exactly the same 30 planes: an upstream gradient at
    # that pixel alone reaches the 30 highest indices and no other plane
    gD = np.zeros((1, 96, 128))
    gD[0, j0, i0] = 1.0
    gc, gq, gr = O.backward(*planes, w2c, intr, 96, 128, lam, gD, np.zeros((1, 96, 128, 3)), M=30)
    touched = np.flatnonzero(np.abs(gc).sum(1) + np.abs(gr).sum(1) > 0)
    assert touched.tolist() == list(range(n - 30, n))


def _random_scene(seed, K=12, V=2, H=48, W=64, f=50.0):
    p = S.random_planes_in_view(seed, K)
    cams = S.identity_cameras(V, H, W, f, seed=seed, jitter=0.05)
    return p, cams


def test_permutation_invariance_and_alpha_bound():
    p, cams = _random_scene(3, K=16)
    lam = 20.0
    a = O.render(p.center, p.quat, p.radii, cams.w2c, cams.intr, cams.H, cams.W, lam)
    perm = np.random.default_rng(0).permutation(p.K)
    b = O.render(p.center[perm], p.quat[perm], p.radii[perm], cams.w2c, cams.intr, cams.H,
                 cams.W, lam)
    assert np.abs(a["depth"] - b["depth"]).max() < 1e-12
    assert np.abs(a["normal"] - b["normal"]).max() < 1e-12
    assert a["alpha"].max() <= 1.0 + 1e-15 and a["alpha"].min() >= 0.0
    assert (a["n_sel"] > 1).mean() > 0.05          # overlaps exist
    empty = a["n_sel"] == 0
    assert np.all(a["depth"][empty] == 0) and np.all(a["alpha"][empty] == 0)


def test_disjoint_planes_add():
    lam = 20.0
    H, W, f = 48, 64, 50.0
    w2c, intr = ident_cams(1, H, W, f)
    left = cat(plane([-0.8, 0.0, 2.0], [1, 0, 0, 0], [0.3, 0.2, 0.4, 0.3]),
               plane([-0.7, 0.2, 2.6], rot_z_quat(0.3), [0.2, 0.3, 0.2, 0.2]))
    right = cat(plane([0.8, 0.0, 2.2], [0, 1, 0, 0], [0.3, 0.3, 0.3, 0.3]))
    both = O.render(*cat(left, right), w2c, intr, H, W, lam)
    a = O.render(*left, w2c, intr, H, W, lam)
    b = O.render(*right, w2c, intr, H, W, lam)
    assert ((a["alpha"] > 0) & (b["alpha"] > 0)).sum() == 0
    assert np.abs(both["depth"] - (a["depth"] + b["depth"])).max() < 1e-12
    assert np.abs(both["normal"] - (a["normal"] + b["normal"])).max() < 1e-12


def test_single_radii_option_equals_symmetric_radii():
    p, cams = _random_scene(5)
    sym = p.radii.copy()
    sym[:, 1] = sym[:, 0]
    sym[:, 3] = sym[:, 2]
    a = O.render(p.center, p.quat, p.radii, cams.w2c, cams.intr, cams.H, cams.W, 20.0,
                 single_radii=True)
    b = O.render(p.center, p.quat, sym, cams.w2c, cams.intr, cams.H, cams.W, 20.0)
    assert np.array_equal(a["depth"], b["depth"]) and np.array_equal(a["normal"], b["normal"])


def test_scaled_quaternion_gives_same_render():
    p, cams = _random_scene(6)
    a = O.render(p.center, p.quat, p.radii, cams.w2c, cams.intr, cams.H, cams.W, 20.0)
    b = O.render(p.center, p.quat.astype(np.float64) * 4.0, p.radii, cams.w2c, cams.intr,
                 cams.H, cams.W, 20.0)
    assert np.abs(a["depth"] - b["depth"]).max() < 1e-12


# ---------------------------------------------------------------------------
# Eq. 14: loss values and gradient.

def test_loss_closed_forms():
    rng = np.random.default_rng(1)
    V, H, W = 2, 5, 7
    Ng = rng.normal(size=(V, H, W, 3))
    Ng /= np.linalg.norm(Ng, axis=-1, keepdims=True)
    Dg = rng.uniform(1, 3, size=(V, H, W))
    off = rng.normal(size=(V, H, W))
    tot, dD, dN, sums = O.loss(Dg + off, Ng, Dg, Ng)
    assert tot == pytest.approx(np.abs(off).sum(), rel=1e-13)   # normal terms vanish
    assert sums[:, 3].sum() == V * H * W
    tot2, _, _, sums2 = O.loss(Dg, -Ng, Dg, Ng)
    # N = -N*: |1 - N.N*| = 2 per pixel and ||N - N*||_1 = 2 ||N*||_1
    assert sums2[:, 0].sum() == pytest.approx(2.0 * V * H * W, rel=1e-13)
    assert sums2[:, 1].sum() == pytest.approx(2.0 * np.abs(Ng).sum(), rel=1e-13)
    assert tot2 == pytest.approx(5 * (2.0 * V * H * W + 2.0 * np.abs(Ng).sum()), rel=1e-13)
    # invalid pixels (gt depth 0) are not supervised
    Dz = Dg.copy()
    Dz[0] = 0
    tot3, dD3, _, sums3 = O.loss(Dg + off, Ng, Dz, Ng)
    assert sums3[0, 3] == 0 and np.all(dD3[0] == 0)


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(2)
    V, H, W = 1, 3, 4
    D = rng.uniform(1, 3, size=(V, H, W))
    N = rng.normal(size=(V, H, W, 3)) * 0.5
    Dg = rng.uniform(1, 3, size=(V, H, W))
    Ng = rng.normal(size=(V, H, W, 3))
    _, dD, dN, _ = O.loss(D, N, Dg, Ng)
    h = 1e-7
    for idx in np.ndindex(D.shape):
        e = np.zeros_like(D)
        e[idx] = h
        fd = (O.loss(D + e, N, Dg, Ng)[0] - O.loss(D - e, N, Dg, Ng)[0]) / (2 * h)
        assert fd == pytest.approx(dD[idx], abs=1e-6)
    for idx in np.ndindex(N.shape):
        e = np.zeros_like(N)
        e[idx] = h
        fd = (O.loss(D, N + e, Dg, Ng)[0] - O.loss(D, N - e, Dg, Ng)[0]) / (2 * h)
        assert fd == pytest.approx(dN[idx], abs=1e-6)


# ---------------------------------------------------------------------------
# Backward: central finite differences on a smooth functional of the render.

def _fd_check(p, cams, lam, seed, h=1e-6, rtol=2e-5, M=30, single_radii=False):
    rng = np.random.default_rng(seed)
    V, H, W = cams.V, cams.H, cams.W
    gD = rng.normal(size=(V, H, W))
    gN = rng.normal(size=(V, H, W, 3))

    def J(c, q, r):
        o = O.render(c, q, r, cams.w2c, cams.intr, H, W, lam, M=M, single_radii=single_radii)
        return float(np.sum(gD * o["depth"]) + np.sum(gN * o["normal"]))

    c0 = p.center.astype(np.float64)
    q0 = p.quat.astype(np.float64) * 1.3        # non-unit: exercises the normalisation
    r0 = p.radii.astype(np.float64)
    gc, gq, gr = O.backward(c0, q0, r0, cams.w2c, cams.intr, H, W, lam, gD, gN, M=M,
                            single_radii=single_radii)
    an = np.concatenate([gc.ravel(), gq.ravel(), gr.ravel()])
    scale = np.abs(an).max()
    assert scale > 0
    fd = np.zeros_like(an)
    shapes = [c0.shape, q0.shape, r0.shape]
    sizes = [c0.size, q0.size, r0.size]
    base = [c0, q0, r0]
    pos = 0
    for g, (shp, sz) in enumerate(zip(shapes, sizes)):
        for i in range(sz):
            plus = [b.copy() for b in base]
            minus = [b.copy() for b in base]
            plus[g].reshape(-1)[i] += h
            minus[g].reshape(-1)[i] -= h
            fd[pos + i] = (J(*plus) - J(*minus)) / (2 * h)
        pos += sz
    err = np.abs(fd - an)
    bad = err > rtol * np.abs(an) + 1e-5 * scale
    assert not bad.any(), (np.nonzero(bad), fd[bad], an[bad])


@pytest.mark.parametrize("lam", [7.36, 20.0, 60.0])
def test_backward_matches_central_differences(lam):
    p, cams = _random_scene(11, K=6, V=2, H=24, W=32, f=25.0)
    _fd_check(p, cams, lam, seed=4)


def test_backward_single_radii_and_small_m():
    p, cams = _random_scene(12, K=6, V=2, H=24, W=32, f=25.0)
    _fd_check(p, cams, 20.0, seed=5, single_radii=True)
    _fd_check(p, cams, 20.0, seed=6, M=2)


def test_rounding_sensitivity_matches_finite_differences():
    # sens_d is sum_j |dD/dm_j| eta (1 + t + |p_c|): for one fronto-parallel plane whose
    # right edge band crosses the centre row, dD/dm = dD/dr^x+ (m = r^x+ - P_X there);
    # central differences of the render in r^x+ must give the same slope
    w2c, intr = ident_cams()
    Z, lam, eta = 2.0, 20.0, 1e-6
    c, q, r = plane([0.0, 0.0, Z], [1, 0, 0, 0], [0.3, 0.6, 0.6, 0.6])
    o = O.render(c, q, r, w2c, intr, 96, 128, lam, eta=eta)
    h = 1e-5
    rp, rm = r.copy(), r.copy()
    rp[0, 0] += h
    rm[0, 0] -= h
    fd = (O.render(c, q, rp, w2c, intr, 96, 128, lam)["depth"] -
          O.render(c, q, rm, w2c, intr, 96, 128, lam)["depth"]) / (2 * h)
    j = 48
    band = [i for i in range(64, 128) if 1e-3 < o["alpha"][0, j, i] < 0.999]
    assert len(band) >= 3
    pc = np.array([0.0, 0.0, Z])
    for i in band:
        e = eta * (1.0 + o["depth"][0, j, i] / o["alpha"][0, j, i] + np.linalg.norm(pc))
        assert o["sens_d"][0, j, i] == pytest.approx(abs(fd[0, j, i]) * e, rel=1e-4)
        assert o["ill"][0, j, i] & 4 == 0
    # interior pixels (w = 1) have no first-order sensitivity
    assert o["sens_d"][0, j, 64] == 0.0


# ---------------------------------------------------------------------------
# Binning: conservativeness against single-plane brute force, list contents.

def test_binning_covers_every_surviving_pair_and_key_bounds_depth():
    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 1)
    cams = room.cams
    lam = 20.0
    tw, th = 16, 16
    delta = O.filter_margin(lam)
    rect, key, key32 = O.bin_records(init.center, init.quat, init.radii, cams.w2c, cams.intr,
                                     cams.H, cams.W, tw, th, delta)
    n_checked = 0
    for k in range(init.K):
        o = O.render(init.center[k:k + 1], init.quat[k:k + 1], init.radii[k:k + 1], cams.w2c,
                     cams.intr, cams.H, cams.W, lam)
        for v in range(cams.V):
            vj, vi = np.nonzero(o["alpha"][v] > 0)
            if vj.size == 0:
                continue
            x0, y0, x1, y1 = rect[v, k]
            assert x1 >= x0 and y1 >= y0, "plane with surviving pixels was culled"
            assert (vi // tw).min() >= x0 and (vi // tw).max() <= x1
            assert (vj // th).min() >= y0 and (vj // th).max() <= y1
            t = o["depth"][v][vj, vi] / o["alpha"][v][vj, vi]
            # the key is the FP32 formula's: a bound up to its few roundings (relative
            # 1e-6 here; the splat kernels allow 1/4096)
            assert t.min() >= key[v, k] * (1 - 1e-6)
            assert float(key32[v, k]) == key[v, k]
            n_checked += vj.size
    assert n_checked > 10000


def test_tile_lists_brute_force():
    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 2)
    cams = room.cams
    tw, th = 16, 8
    rect, key, key32 = O.bin_records(init.center, init.quat, init.radii, cams.w2c, cams.intr,
                                     cams.H, cams.W, tw, th, O.filter_margin(7.36))
    ns = O.records_ns(init.center, init.quat, init.radii, cams.w2c)
    ptr, ent, ekey = O.tile_lists(rect, key32, ns, cams.intr, cams.H, cams.W, tw, th)
    txn, tyn = (cams.W + tw - 1) // tw, (cams.H + th - 1) // th
    K = init.K
    for v in range(cams.V):
        for ty in range(tyn):
            for tx in range(txn):
                t = v * txn * tyn + ty * txn + tx
                expect = [v * K + k for k in range(K)
                          if rect[v, k, 0] <= tx <= rect[v, k, 2] and rect[v, k, 1] <= ty <= rect[v, k, 3]]
                kk = {r: float(O.entry_keys(ns[v, r - v * K][None], cams.intr[v][None], [tx], [ty],
                                            tw, th, rec_key=[key32[v, r - v * K]])[0])
                      for r in expect}
                expect.sort(key=lambda r: (kk[r], r))
                assert list(ent[ptr[t]:ptr[t + 1]]) == expect
                assert [kk[r] for r in expect] == list(ekey[ptr[t]:ptr[t + 1]])


def test_entry_keys_bound_every_depth_of_the_tile():
    # the entry key of a (plane, tile) pair is below the depth of every candidate pixel of
    # the tile (single-plane brute-force renders); for most pairs it is well above the
    # record's quad key (the tile sees only part of the plane)
    room = S.tiny_room(0)
    init = S.perturb_planes(room.gt, 3)
    cams = room.cams
    tw, th = 8, 8
    lam = 7.36
    rect, key, key32 = O.bin_records(init.center, init.quat, init.radii, cams.w2c, cams.intr,
                                     cams.H, cams.W, tw, th, O.filter_margin(lam))
    ns = O.records_ns(init.center, init.quat, init.radii, cams.w2c)
    tighter, checked = 0, 0
    for k in range(init.K):
        o = O.render(init.center[k:k + 1], init.quat[k:k + 1], init.radii[k:k + 1], cams.w2c,
                     cams.intr, cams.H, cams.W, lam)
        for v in range(cams.V):
            vj, vi = np.nonzero(o["alpha"][v] > 0)
            if vj.size == 0:
                continue
            t = o["depth"][v][vj, vi] / o["alpha"][v][vj, vi]
            tx, ty = vi // tw, vj // th
            ek = O.entry_keys(np.repeat(ns[v, k][None], len(tx), 0),
                              np.repeat(cams.intr[v][None], len(tx), 0), tx, ty, tw, th,
                              rec_key=np.full(len(tx), key32[v, k]))
            assert np.all(t >= ek.astype(np.float64) * (1 - 1e-6)), (k, v)
            assert np.all(ek >= key32[v, k])
            tighter += int((ek > key32[v, k] * 1.01).sum())
            checked += len(t)
    assert checked > 10000 and tighter > 0.3 * checked


def test_binning_culls_plane_behind_camera():
    w2c, intr = ident_cams(1)
    c, q, r = plane([0, 0, -2.0], [1, 0, 0, 0], [0.5, 0.5, 0.5, 0.5])
    rect, key, _ = O.bin_records(c, q, r, w2c, intr, 96, 128, 16, 16, 0.01)
    assert rect[0, 0, 2] < rect[0, 0, 0] and math.isinf(key[0, 0])
    # a plane crossing z = 0 is clipped, not culled, and its key is z_near (as a float)
    c, q, r = plane([0, 0, 0.5], [math.cos(math.pi / 4), math.sin(math.pi / 4), 0, 0], [1, 1, 1, 1])
    rect, key, _ = O.bin_records(c, q, r, w2c, intr, 96, 128, 16, 16, 0.01)
    assert rect[0, 0, 2] >= rect[0, 0, 0] and key[0, 0] == float(np.float32(O.Z_NEAR))


# ---------------------------------------------------------------------------
# Ground-truth ray caster and Adam.

def test_raycast_room_center_pixel():
    room = S.tiny_room(0)
    D, N, pid = O.raycast(room.gt.center, room.gt.quat, room.gt.radii, room.cams.w2c,
                          room.cams.intr, room.cams.H, room.cams.W)
    assert (pid >= 0).all()                        # closed room: every ray hits
    # view 0 sits at (3, 2.5, 1.5) looking at -x: the wall x = 0 is 3 m ahead and
    # faces +x (towards the camera): camera-frame normal (0, 0, -1)
    assert D[0, 47:49, 63:65] == pytest.approx(3.0, abs=1e-9)
    assert N[0, 48, 64] == pytest.approx([0, 0, -1], abs=1e-9)


def test_sharp_render_approaches_raycast():
    room = S.tiny_room(0)
    g = room.gt
    D, N, pid = O.raycast(g.center, g.quat, g.radii, room.cams.w2c, room.cams.intr,
                          room.cams.H, room.cams.W)
    o = O.render(g.center, g.quat, g.radii, room.cams.w2c, room.cams.intr, room.cams.H,
                 room.cams.W, 1e7)
    close = np.abs(o["depth"] - D) < 1e-6
    assert close.mean() > 0.99


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(5)]
    pt = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for s, g in enumerate(grads, 1):
        opt.zero_grad()
        pt.grad = torch.tensor(g)
        opt.step()
        O.adam(p, g, m, v, s)
    assert np.abs(p - pt.detach().numpy()).max() < 1e-14
    # clamp keeps values at or above the bound
    p2 = np.full(4, 1e-3)
    O.adam(p2, np.ones(4), np.zeros(4), np.zeros(4), 1, clamp_min=1e-3)
    assert np.all(p2 == 1e-3)


def test_grazing_incidence_flags_gradient_pixels():
    # Eq. 4 divides by d . n; where a pixel ray nearly lies in a composited plane the
    # FP32 evaluation loses about log2(kappa) bits, kappa = sum |d_i n_i| / |d . n|.
    # The oracle marks those pixels (kappa > 100) as not comparable for gradients
    # (flag bit 3).  Here a plane is tilted 0.002 rad out of the pixel ray of one
    # column and centred where that ray meets it at 5 m; kappa is computed in the
    # test from the plane equation alone.
    lam = 50.0
    H, W, f = 48, 64, 50.0
    i0 = 17
    d0 = np.array([(i0 + 0.5 - W / 2.0) / f, 0.0, 1.0])
    u = d0 / np.linalg.norm(d0)
    n = np.array([u[2], 0.0, -u[0]]) + 0.002 * u
    n /= np.linalg.norm(n)
    vy = np.array([0.0, 1.0, 0.0])
    vx = np.cross(vy, n)
    quat = S.quat_from_frame(vx, vy, n)
    t0 = 5.0
    center = t0 * d0
    w2c, intr = ident_cams(1, H, W, f)
    o = O.render(*plane(center, quat, [5.0, 5.0, 5.0, 5.0]), w2c, intr, H, W, lam)
    grazing = other = 0
    for j in range(H):
        for i in range(W):
            if not o["alpha"][0, j, i] > 0:
                continue
            dx, dy = pix_ray(i, j, f, W / 2.0, H / 2.0)
            den = dx * n[0] + dy * n[1] + n[2]
            kappa = (abs(dx * n[0]) + abs(dy * n[1]) + abs(n[2])) / abs(den)
            if kappa > 100.0:
                grazing += 1
                assert o["ill"][0, j, i] & 8, (i, j, kappa)
                assert o["depth"][0, j, i] / o["alpha"][0, j, i] == pytest.approx(t0, rel=1e-9)
            else:
                other += 1
    assert grazing >= H // 2 and other >= 1
