"""Pins of the plane-splitting oracle (Sec. 3.3 "Plane Splitting").

The geometry is checked against rectangles built from scipy's rotation of the
same quaternions (an independent implementation of R(q)): the two halves of a
split plane tile the parent rectangle exactly."""
import math

import numpy as np
import pytest

from oracle import split_oracle as SO

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def _planes(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(n, 3))
    q = rng.normal(size=(n, 4))
    r = rng.uniform(0.1, 1.0, size=(n, 4))
    return c, q, r


def _axes_scipy(q):
    # scipy takes (x, y, z, w); columns of the matrix are the plane's v^x, v^y, n
    R = Rotation.from_quat(np.roll(q / np.linalg.norm(q), -1)).as_matrix()
    return R[:, 0], R[:, 1]


def _corners(c, q, r):
    """(x+, y+), (x+, y-), (x-, y+), (x-, y-) corners of a rectangle."""
    vx, vy = _axes_scipy(q)
    return {(sx, sy): c + (r[0] if sx > 0 else -r[1]) * vx + (r[2] if sy > 0 else -r[3]) * vy
            for sx in (1, -1) for sy in (1, -1)}


def test_rotation_matches_scipy():
    _, q, _ = _planes(20, 1)
    R = SO.rotation(q)
    for i in range(20):
        ref = Rotation.from_quat(np.roll(q[i] / np.linalg.norm(q[i]), -1)).as_matrix()
        assert np.allclose(R[i], ref, atol=1e-12)


def test_below_threshold_is_identity():
    c, q, r = _planes(10, 2)
    acc = np.full((10, 2), 0.1)
    out = SO.split_planes(c, q, r, [0, 10], acc, n_iter=1, tau=0.2)
    assert out["count"] == 10
    assert np.array_equal(out["center"], c) and np.array_equal(out["radii"], r)
    assert np.array_equal(out["split_rank"], np.zeros(11))


@pytest.mark.parametrize("axis", [0, 1])
def test_halves_tile_the_parent(axis):
    c, q, r = _planes(1, 3 + axis)
    acc = np.zeros((1, 2))
    acc[0, axis] = 5.0
    out = SO.split_planes(c, q, r, [0, 1], acc, n_iter=10, tau=0.2)
    assert out["count"] == 2 and list(out["plane_ptr"]) == [0, 2]
    parent = _corners(c[0], q[0], r[0])
    A = _corners(out["center"][0], out["quat"][0], out["radii"][0])
    B = _corners(out["center"][1], out["quat"][1], out["radii"][1])
    # the +half keeps the parent's + edge, the -half its - edge; they meet on the cut
    for sy in (1, -1):
        if axis == 0:
            assert np.allclose(A[(1, sy)], parent[(1, sy)]) and np.allclose(B[(-1, sy)], parent[(-1, sy)])
            assert np.allclose(A[(-1, sy)], B[(1, sy)])
        else:
            assert np.allclose(A[(sy, 1)], parent[(sy, 1)]) and np.allclose(B[(sy, -1)], parent[(sy, -1)])
            assert np.allclose(A[(sy, -1)], B[(sy, 1)])
    area = lambda rr: (rr[0] + rr[1]) * (rr[2] + rr[3])
    assert np.isclose(area(out["radii"][0]) + area(out["radii"][1]), area(r[0]))
    # the other axis and the rotation are untouched
    o = 2 if axis == 0 else 0
    assert np.array_equal(out["radii"][:, o:o + 2], np.repeat(r[:, o:o + 2], 2, axis=0))
    assert np.array_equal(out["quat"], np.repeat(q, 2, axis=0))


def test_larger_axis_wins_and_ties_go_to_x():
    _, q, _ = _planes(3, 5)
    acc = np.array([[1.0, 2.0], [3.0, 1.0], [2.0, 2.0]])
    assert list(SO.split_kind(acc, q, 1, 0.2)) == [2, 1, 1]
    # one axis over the threshold is enough; the mean is over n_iter
    assert list(SO.split_kind(np.array([[3.0, 0.0]]), q[:1], 10, 0.2)) == [1]
    assert list(SO.split_kind(np.array([[3.0, 0.0]]), q[:1], 20, 0.2)) == [0]


def test_degenerate_quaternions_are_kept():
    q = np.array([[0.0, 0, 0, 0], [np.nan, 1, 0, 0], [1.0, 0, 0, 0]])
    assert list(SO.split_kind(np.full((3, 2), 9.0), q, 1, 0.2)) == [0, 0, 1]


def test_scene_layout_and_moments():
    c, q, r = _planes(7, 6)
    ptr = [0, 3, 3, 7]           # the middle scene is empty
    acc = np.zeros((7, 2))
    acc[[0, 2, 5], 0] = 1.0
    acc[6, 1] = 1.0
    P = 7
    m = np.arange(11 * P, dtype=float) + 1
    v = -m
    out = SO.split_planes(c, q, r, ptr, acc, 1, 0.2, m=m, v=v)
    assert out["count"] == 11
    assert list(out["plane_ptr"]) == [0, 5, 5, 11]
    assert list(out["split_rank"]) == [0, 1, 1, 2, 2, 2, 3, 4]
    # scene 0: A0, 1, A2, B0, B2; scene 2: 3, 4, A5, A6, B5, B6
    assert np.array_equal(out["center"][1], c[1]) and np.array_equal(out["center"][5], c[3])
    vx = SO.rotation(q)[:, :, 0]
    assert np.allclose(out["center"][3], c[0] - r[0, 1] / 2 * vx[0])
    assert np.allclose(out["center"][4], c[2] - r[2, 1] / 2 * vx[2])
    Pn = 11
    mc = out["m"][:3 * Pn].reshape(Pn, 3)
    mr = out["m"][7 * Pn:].reshape(Pn, 4)
    assert np.array_equal(mc[1], m[3:6]) and np.array_equal(mc[0], np.zeros(3))
    assert np.array_equal(mr[6], m[7 * P + 16:7 * P + 20])      # plane 4 moved to slot 6
    assert np.array_equal(out["v"][3 * Pn + 4:3 * Pn + 8], -m[3 * P + 4:3 * P + 8])


def test_accumulation_is_the_mean_of_the_two_sides():
    g = np.array([[1.0, -3.0, 0.5, 0.5], [0.0, 0.0, -2.0, 0.0]])
    acc = SO.radii_grad_accum(np.zeros((2, 2)), g, 0.5)
    assert np.allclose(acc, [[1.0, 0.25], [0.0, 0.5]])
    acc = SO.radii_grad_accum(acc, g, np.array([1.0, 2.0]))
    assert np.allclose(acc, [[3.0, 0.75], [0.0, 2.5]])


# ---------------------------------------------------------------------------
# Plane merge (Sec. 3.3 "Plane Merge"): 25 degrees and 0.1 cm as printed.

def _frame_quat(n, rng):
    """Quaternion (w, x, y, z) of a frame whose third column is n (scipy)."""
    a = rng.normal(size=3)
    vx = a - (a @ n) * n
    vx /= np.linalg.norm(vx)
    vy = np.cross(n, vx)
    R = np.stack([vx, vy, n], 1)
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def test_merge_groups_coplanar_pieces_and_splits_the_rest():
    rng = np.random.default_rng(8)
    c0 = np.array([1.0, 2.0, 0.5])
    n1 = np.array([0.0, 0.0, 1.0])
    n2 = np.array([1.0, 0.0, 0.0])
    # five pieces of the plane z = 0.5 + 1 (offset 1 from c0), one flipped, one tilted 20 deg,
    # one tilted 30 deg, one shifted 2 mm, and two pieces of x = 1 + 3
    tilt20 = np.array([math.sin(math.radians(20)), 0, math.cos(math.radians(20))])
    tilt30 = np.array([math.sin(math.radians(30)), 0, math.cos(math.radians(30))])
    centers = [c0 + [0, 0, 1], c0 + [2, 1, 1], c0 + [-1, 3, 1], c0 + [0.5, 0.5, 1], c0 + [3, 3, 1],
               c0 + [0, 0, 1.002], c0 + [3, 0, 0], c0 + [3, 2, 1]]
    normals = [n1, n1, -n1, tilt20, tilt30, n1, n2, n2]
    q = np.array([_frame_quat(n, rng) for n in normals])
    r = np.array([[1.0, 1, 1, 1], [0.5, 0.5, 0.5, 0.5], [0.2, 0.2, 0.2, 0.2], [0.3, 0.3, 0.3, 0.3],
                  [0.4, 0.4, 0.4, 0.4], [0.6, 0.6, 0.6, 0.6], [0.9, 0.9, 0.9, 0.9], [0.1, 0.1, 0.1, 0.1]])
    # the tilted planes pass through the point at offset 1 along their own normals
    centers[3] = c0 + tilt20 * 1.0
    centers[4] = c0 + tilt30 * 1.0
    centers[7] = c0 + n2 * 3.0 + [0, 2, 1]
    g, reps = SO.merge_planes(np.array(centers), q, r, c0, 25.0, 0.001)
    # groups by decreasing area: plane 0 (area 4), then 6, 5, 1, 4, 3, 2, 7
    assert g[0] == g[1] == g[2] == g[3] == 0        # coplanar, flipped and 20 deg pieces join
    assert g[4] != 0                                # 30 deg is beyond 25
    assert g[5] != 0                                # 2 mm is beyond 0.1 cm
    assert g[6] == g[7] != 0                        # the other wall
    assert reps[g[6]] == 6 and reps[0] == 0
    assert len(reps) == 4
    # with 0.1 m the shifted piece joins the first group
    g2, _ = SO.merge_planes(np.array(centers), q, r, c0, 25.0, 0.1)
    assert g2[5] == 0
