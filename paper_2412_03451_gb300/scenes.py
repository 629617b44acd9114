"""Seeded synthetic indoor rooms, cameras and plane initialisations.

This module is the one input generator shared by the CUDA path, the tests and
the CPU oracle.  It holds none of the rendering method's arithmetic (no ray
intersection, splat weight, compositing or loss): only room geometry, camera
poses, random noise and the conversion of an orthonormal frame to a quaternion.

The paper fits ScanNetV2 / ScanNet++ scenes at 480x640 with about 2,000
initial planes (App. A.1, Sec. 3.1); those datasets are not available, so the
rooms below stand in for them with the same image size and plane counts.

Plane convention (shared with the library): center [K,3], quaternion [K,4] in
(w, x, y, z) order whose rotation matrix has columns (v^x, v^y, n) (Eq. 2-3),
radii [K,4] = (r^x+, r^x-, r^y+, r^y-) (Eq. 1).  Cameras: world-to-camera
[R|t] [V,3,4] in the OpenCV frame (x right, y down, z forward), intrinsics
[V,4] = (fx, fy, cx, cy).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Planes:
    center: np.ndarray   # [K,3] float32
    quat: np.ndarray     # [K,4] float32 (w,x,y,z)
    radii: np.ndarray    # [K,4] float32 (x+, x-, y+, y-)

    @property
    def K(self) -> int:
        return int(self.center.shape[0])

    def copy(self) -> "Planes":
        return Planes(self.center.copy(), self.quat.copy(), self.radii.copy())

    def astype(self, dt) -> "Planes":
        return Planes(self.center.astype(dt), self.quat.astype(dt), self.radii.astype(dt))

    def subset(self, idx) -> "Planes":
        return Planes(self.center[idx], self.quat[idx], self.radii[idx])


@dataclass
class Cameras:
    w2c: np.ndarray      # [V,3,4] float32
    intr: np.ndarray     # [V,4] float32
    H: int
    W: int

    @property
    def V(self) -> int:
        return int(self.w2c.shape[0])

    def subset(self, idx) -> "Cameras":
        return Cameras(self.w2c[idx], self.intr[idx], self.H, self.W)


@dataclass
class Room:
    gt: Planes
    cams: Cameras
    size: tuple
    boxes: list = field(default_factory=list)
    axes: tuple = None     # (v^x [K,3], v^y [K,3]) of the ground-truth rectangles, float64


# --------------------------------------------------------------------------
# Small rotation helpers.

def quat_from_frame(vx: np.ndarray, vy: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Unit quaternion (w,x,y,z) of the rotation whose columns are vx, vy, n."""
    R = np.stack([vx, vy, n], axis=1).astype(np.float64)
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    if tr > 0:
        s = np.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.asarray(q)
    return q / np.linalg.norm(q)


def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product a*b for [...,4] arrays in (w,x,y,z) order."""
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def quat_axis_angle(axis: np.ndarray, angle: np.ndarray) -> np.ndarray:
    axis = axis / np.linalg.norm(axis, axis=-1, keepdims=True)
    h = 0.5 * angle[..., None]
    return np.concatenate([np.cos(h), np.sin(h) * axis], axis=-1)


def random_unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World-to-camera [R|t] of an OpenCV camera at eye looking at target (z up world)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f], axis=0)     # rows: camera axes in world
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1)


# --------------------------------------------------------------------------
# Rectangles.

class _RectList:
    def __init__(self):
        self.c, self.vx, self.vy, self.hx, self.hy = [], [], [], [], []

    def add(self, c, vx, vy, hx, hy):
        self.c.append(np.asarray(c, np.float64))
        self.vx.append(np.asarray(vx, np.float64))
        self.vy.append(np.asarray(vy, np.float64))
        self.hx.append(float(hx))
        self.hy.append(float(hy))

    def planes(self) -> Planes:
        K = len(self.c)
        center = np.stack(self.c) if K else np.zeros((0, 3))
        quat = np.zeros((K, 4))
        for k in range(K):
            n = np.cross(self.vx[k], self.vy[k])
            quat[k] = quat_from_frame(self.vx[k], self.vy[k], n)
        radii = np.stack([np.asarray(self.hx), np.asarray(self.hx),
                          np.asarray(self.hy), np.asarray(self.hy)], axis=1) if K else np.zeros((0, 4))
        return Planes(center.astype(np.float32), quat.astype(np.float32), radii.astype(np.float32))

    def axes(self):
        K = len(self.c)
        return (np.stack(self.vx) if K else np.zeros((0, 3)), np.stack(self.vy) if K else np.zeros((0, 3)))


def _room_faces(sx, sy, sz):
    """The 6 inner faces of the box [0,sx]x[0,sy]x[0,sz] as (corner, u, v, su, sv)
    with normal u x v pointing into the room."""
    ex, ey, ez = np.eye(3)
    return [
        (np.zeros(3), ex, ey, sx, sy),                     # floor, n = +z
        (np.array([0, sy, sz]), ex, -ey, sx, sy),          # ceiling, n = -z
        (np.zeros(3), ey, ez, sy, sz),                     # wall x=0, n = +x
        (np.array([sx, sy, 0]), -ey, ez, sy, sz),          # wall x=sx, n = -x
        (np.array([sx, 0, 0]), -ex, ez, sx, sz),           # wall y=0, n = +y
        (np.array([0, sy, 0]), ex, ez, sx, sz),            # wall y=sy, n = -y
    ]


def _box_faces(lo, hi, top=False):
    """Outer faces of an axis-aligned box (normal pointing away from the box)."""
    (x0, y0, z0), (x1, y1, z1) = lo, hi
    ex, ey, ez = np.eye(3)
    f = [
        (np.array([x0, y1, z0]), -ey, ez, y1 - y0, z1 - z0),   # x = x0, n = -x
        (np.array([x1, y0, z0]), ey, ez, y1 - y0, z1 - z0),    # x = x1, n = +x
        (np.array([x0, y0, z0]), ex, ez, x1 - x0, z1 - z0),    # y = y0, n = -y
        (np.array([x1, y1, z0]), -ex, ez, x1 - x0, z1 - z0),   # y = y1, n = +y
    ]
    if top:
        f.append((np.array([x0, y0, z1]), ex, ey, x1 - x0, y1 - y0))  # n = +z
    return f


def _grid_split(rl: _RectList, face, nu, nv):
    corner, u, v, su, sv = face
    du, dv = su / nu, sv / nv
    for i in range(nu):
        for j in range(nv):
            c = corner + (i + 0.5) * du * u + (j + 0.5) * dv * v
            rl.add(c, u, v, 0.5 * du, 0.5 * dv)


# --------------------------------------------------------------------------
# Tiny room: 4x5x3 m, 48 face rectangles + 4 boxes x 4 faces = 64 planes,
# 8 cameras at 128x96 (fx = fy = 100) on a 1 m circle at 1.5 m, looking in.

def tiny_room(seed: int = 0, H: int = 96, W: int = 128, f: float = 100.0, n_views: int = 8,
              n_boxes: int = 4) -> Room:
    rng = np.random.default_rng(seed)
    sx, sy, sz = 4.0, 5.0, 3.0
    rl = _RectList()
    for face in _room_faces(sx, sy, sz):
        su, sv = face[3], face[4]
        nu, nv = (4, 2) if su >= sv else (2, 4)
        _grid_split(rl, face, nu, nv)
    ctr = np.array([sx / 2, sy / 2])
    boxes = []
    while len(boxes) < n_boxes:
        size = rng.uniform(0.3, 1.0, size=3)
        lo_xy = rng.uniform([0.1, 0.1], [sx - 0.1 - size[0], sy - 0.1 - size[1]])
        # keep boxes away from the camera circle (radius 1 m around the centre)
        near = np.clip(ctr, lo_xy, lo_xy + size[:2])
        if np.linalg.norm(near - ctr) < 1.4:
            continue
        lo = np.array([lo_xy[0], lo_xy[1], 0.0])
        hi = lo + size
        boxes.append((lo, hi))
        for face in _box_faces(lo, hi, top=False):
            rl.add(face[0] + 0.5 * face[3] * face[1] + 0.5 * face[4] * face[2],
                   face[1], face[2], 0.5 * face[3], 0.5 * face[4])
    gt = rl.planes()
    w2c, intr = [], []
    target = np.array([ctr[0], ctr[1], 1.5])
    for i in range(n_views):
        a = 2 * np.pi * i / n_views
        eye = np.array([ctr[0] + np.cos(a), ctr[1] + np.sin(a), 1.5])
        # look inward: from the circle through the room centre
        w2c.append(look_at(eye, target))
        intr.append([f, f, W / 2.0, H / 2.0])
    cams = Cameras(np.asarray(w2c, np.float32), np.asarray(intr, np.float32), H, W)
    return Room(gt, cams, (sx, sy, sz), boxes, rl.axes())


def perturb_planes(gt: Planes, seed: int, center_sigma=0.1, angle_sigma_deg=10.0,
                   radius_range=(0.7, 1.3)) -> Planes:
    """Noisy initialisation: center + N(0, sigma), rotation by a uniform axis and an
    angle ~ N(0, angle_sigma), each radius times U(radius_range)."""
    rng = np.random.default_rng(seed)
    K = gt.K
    c = gt.center.astype(np.float64) + rng.normal(0.0, center_sigma, size=(K, 3))
    ax = random_unit_vectors(rng, K)
    ang = np.deg2rad(rng.normal(0.0, angle_sigma_deg, size=K))
    q = quat_mul(quat_axis_angle(ax, ang), gt.quat.astype(np.float64))
    r = gt.radii.astype(np.float64) * rng.uniform(*radius_range, size=(K, 4))
    return Planes(c.astype(np.float32), q.astype(np.float32), r.astype(np.float32))


# --------------------------------------------------------------------------
# Paper-scale room: 8x10x3 m with furniture, ~2000 GT rectangles whose
# half-extents spread over about [0.1, 2] m, 64 views at 640x480 (fx = 500)
# on a smooth random trajectory.

def _split_faces(faces, n_target, rng, min_half=0.1, max_half=2.0):
    """Random guillotine splits of the given faces until n_target rectangles.
    A splittable rectangle is chosen uniformly at random (regardless of size)
    and cut across its longer side at a random fraction, which spreads the
    half-extents over a wide range from min_half upwards (about 0.1-1 m for
    2,000 rectangles in an 8x10x3 m room: that many rectangles cannot tile the
    room with sizes log-uniform up to 2 m)."""
    rects = [list(f) for f in faces]   # corner, u, v, su, sv
    # first make every rectangle at most 2*max_half long
    i = 0
    while i < len(rects):
        corner, u, v, su, sv = rects[i]
        if su > 2 * max_half or sv > 2 * max_half:
            if su >= sv:
                rects[i] = [corner, u, v, su / 2, sv]
                rects.append([corner + (su / 2) * u, u, v, su / 2, sv])
            else:
                rects[i] = [corner, u, v, su, sv / 2]
                rects.append([corner + (sv / 2) * v, u, v, su, sv / 2])
        else:
            i += 1
    guard = 0
    while len(rects) < n_target and guard < 100000:
        guard += 1
        longest = np.array([max(r[3], r[4]) for r in rects])
        ok = longest >= 4 * min_half
        if not ok.any():
            break
        wgt = np.where(ok, rng.uniform(size=len(rects)), 0.0)
        j = int(np.argmax(wgt))
        corner, u, v, su, sv = rects[j]
        frac = rng.uniform(0.25, 0.75)
        if su >= sv:
            a = max(2 * min_half, min(su - 2 * min_half, frac * su))
            rects[j] = [corner, u, v, a, sv]
            rects.append([corner + a * u, u, v, su - a, sv])
        else:
            a = max(2 * min_half, min(sv - 2 * min_half, frac * sv))
            rects[j] = [corner, u, v, su, a]
            rects.append([corner + a * v, u, v, su, sv - a])
    return rects


def _catmull_rom(P: np.ndarray, n: int) -> tuple:
    """n samples (positions, tangents) along a closed Catmull-Rom spline through P."""
    m = len(P)
    pos, tan = [], []
    for s in np.linspace(0, m, n, endpoint=False):
        i = int(np.floor(s))
        u = s - i
        p0, p1, p2, p3 = P[(i - 1) % m], P[i % m], P[(i + 1) % m], P[(i + 2) % m]
        a = 2 * p1
        b = p2 - p0
        c = 2 * p0 - 5 * p1 + 4 * p2 - p3
        d = -p0 + 3 * p1 - 3 * p2 + p3
        pos.append(0.5 * (a + b * u + c * u * u + d * u ** 3))
        tan.append(0.5 * (b + 2 * c * u + 3 * d * u * u))
    return np.asarray(pos), np.asarray(tan)


def large_room(seed: int = 1000, n_rect: int = 2000, size=(8.0, 10.0, 3.0), n_views: int = 64,
               H: int = 480, W: int = 640, f: float = 500.0, n_boxes: int = 10) -> Room:
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    boxes = []
    guard = 0
    while len(boxes) < n_boxes and guard < 10000:
        guard += 1
        bs = np.array([rng.uniform(0.4, min(2.0, sx / 3)), rng.uniform(0.4, min(2.0, sy / 3)),
                       rng.uniform(0.4, 1.4)])
        lo = np.array([rng.uniform(0.05, sx - 0.05 - bs[0]), rng.uniform(0.05, sy - 0.05 - bs[1]), 0.0])
        hi = lo + bs
        clash = any(not (hi[0] + 0.3 < b[0][0] or b[1][0] + 0.3 < lo[0] or
                         hi[1] + 0.3 < b[0][1] or b[1][1] + 0.3 < lo[1]) for b in boxes)
        if clash:
            continue
        boxes.append((lo, hi))
    faces = list(_room_faces(sx, sy, sz))
    for lo, hi in boxes:
        faces += _box_faces(lo, hi, top=True)
    rects = _split_faces(faces, n_rect, rng)
    rl = _RectList()
    for corner, u, v, su, sv in rects:
        rl.add(corner + 0.5 * su * u + 0.5 * sv * v, u, v, 0.5 * su, 0.5 * sv)
    gt = rl.planes()
    cams = trajectory_cameras(rng, (sx, sy, sz), boxes, n_views, H, W, f)
    return Room(gt, cams, (sx, sy, sz), boxes, rl.axes())


def trajectory_cameras(rng, size, boxes, n_views, H, W, f, n_ctrl=8, margin=0.8) -> Cameras:
    sx, sy, sz = size
    pts = []
    guard = 0
    while len(pts) < n_ctrl and guard < 100000:
        guard += 1
        p = np.array([rng.uniform(margin, sx - margin), rng.uniform(margin, sy - margin),
                      rng.uniform(1.2, 1.8)])
        if any((lo[0] - 0.5 < p[0] < hi[0] + 0.5) and (lo[1] - 0.5 < p[1] < hi[1] + 0.5)
               for lo, hi in boxes):
            continue
        pts.append(p)
    pts = np.asarray(pts)
    # order the control points around the room centre so the loop is smooth
    ang = np.arctan2(pts[:, 1] - sy / 2, pts[:, 0] - sx / 2)
    pts = pts[np.argsort(ang)]
    pos, tan = _catmull_rom(pts, n_views)
    w2c, intr = [], []
    for p, t in zip(pos, tan):
        yaw = np.arctan2(t[1], t[0]) + np.deg2rad(rng.uniform(-30, 30))
        pitch = np.deg2rad(rng.uniform(-20, 5))
        d = np.array([np.cos(yaw) * np.cos(pitch), np.sin(yaw) * np.cos(pitch), np.sin(pitch)])
        w2c.append(look_at(p, p + d))
        intr.append([f, f, W / 2.0, H / 2.0])
    return Cameras(np.asarray(w2c, np.float32), np.asarray(intr, np.float32), H, W)


def backprojected_init(depth: np.ndarray, cams: Cameras, n: int, seed: int,
                       radius: float = 0.2) -> Planes:
    """n planes centred at back-projected random pixels of the given depth maps
    (pixels with depth > 0), with uniformly random orientation and all radii
    equal to `radius`."""
    rng = np.random.default_rng(seed)
    V, H, W = depth.shape
    valid = np.argwhere(depth > 0)
    pick = valid[rng.integers(0, len(valid), size=n)]
    centers = np.zeros((n, 3))
    for idx, (v, j, i) in enumerate(pick):
        fx, fy, cx, cy = cams.intr[v].astype(np.float64)
        z = float(depth[v, j, i])
        pc = np.array([(i + 0.5 - cx) / fx * z, (j + 0.5 - cy) / fy * z, z])
        Rt = cams.w2c[v].astype(np.float64)
        centers[idx] = Rt[:, :3].T @ (pc - Rt[:, 3])
    quat = random_quats(rng, n)
    radii = np.full((n, 4), radius)
    return Planes(centers.astype(np.float32), quat.astype(np.float32), radii.astype(np.float32))


def surface_init(room: Room, n: int, seed: int, radius: float = 0.2) -> Planes:
    """n planes centred at points drawn uniformly (by area) on the ground-truth
    rectangles of the room, with uniformly random orientation and all radii =
    radius.  With exact synthetic depth, back-projected depth pixels lie on these
    rectangles, so this stands in for the "random depth-backprojected points"
    initialisation without rendering anything."""
    rng = np.random.default_rng(seed)
    gt = room.gt
    vx_all, vy_all = room.axes
    area = (gt.radii[:, 0] + gt.radii[:, 1]).astype(np.float64) * (gt.radii[:, 2] + gt.radii[:, 3])
    k = rng.choice(gt.K, size=n, p=area / area.sum())
    u = rng.uniform(-gt.radii[k, 1], gt.radii[k, 0])
    v = rng.uniform(-gt.radii[k, 3], gt.radii[k, 2])
    centers = gt.center[k].astype(np.float64) + u[:, None] * vx_all[k] + v[:, None] * vy_all[k]
    quat = random_quats(rng, n)
    radii = np.full((n, 4), radius)
    return Planes(centers.astype(np.float32), quat.astype(np.float32), radii.astype(np.float32))


def surface_init_nn(room: Room, n: int, seed: int, scale: float = 0.5) -> Planes:
    """Like surface_init, but every radius is scale x the distance to the nearest
    other centre (Sec. 3.1: initial radii 0.5 Dist(pi)), so coverage follows the
    plane count."""
    p = surface_init(room, n, seed)
    from scipy.spatial import cKDTree
    d, _ = cKDTree(p.center.astype(np.float64)).query(p.center.astype(np.float64), k=2)
    r = np.clip(scale * d[:, 1], 0.02, 2.0)
    p.radii[:] = r[:, None].astype(np.float32)
    return p


def sphere_init(room: Room, n: int, seed: int, radius: float = 0.05) -> Planes:
    """The sphere initialisation of the ablation in Sec. 4.3: n planes with all
    radii = radius on the bounding sphere of the scene (centre of the room box,
    radius half its diagonal), normals pointing to the centre, random rotation
    about the normal."""
    rng = np.random.default_rng(seed)
    size = np.asarray(room.size, np.float64)
    centre = size / 2.0
    R = 0.5 * float(np.linalg.norm(size))
    u = random_unit_vectors(rng, n)
    centers = centre + R * u
    nrm = -u
    a = random_unit_vectors(rng, n)
    vx = a - (a * nrm).sum(1, keepdims=True) * nrm
    vx /= np.linalg.norm(vx, axis=1, keepdims=True)
    vy = np.cross(nrm, vx)
    quat = np.array([quat_from_frame(vx[k], vy[k], nrm[k]) for k in range(n)])
    radii = np.full((n, 4), radius)
    return Planes(centers.astype(np.float32), quat.astype(np.float32), radii.astype(np.float32))


def mono_points(room: Room, depth: np.ndarray, normal: np.ndarray, n: int, seed: int,
                scale_sigma: float = 0.03, depth_sigma: float = 0.01,
                normal_sigma_deg: float = 8.0) -> Planes:
    """Stand-in for the monocular-depth initialisation of Sec. 3.1: the
    ground-truth depth and camera-frame normal maps [V, H, W] / [V, H, W, 3] are
    degraded like a monocular prediction (a per-view depth scale error
    N(1, scale_sigma), per-pixel relative depth noise N(0, depth_sigma), normals
    tilted by N(0, normal_sigma_deg) degrees about a random axis), n random
    valid pixels are back-projected to plane centres, each plane's normal is the
    degraded normal (so its rotation comes from the coarse geometry), its
    in-plane rotation is random.  The radii are left at 0: they follow from the
    centres (mono_init here on the host, the library's nearest-neighbour kernel in
    the package)."""
    rng = np.random.default_rng(seed)
    cams = room.cams
    V = depth.shape[0]
    scale = rng.normal(1.0, scale_sigma, size=V)
    valid = np.argwhere(depth > 0)
    pick = valid[rng.integers(0, len(valid), size=n)]
    v, j, i = pick[:, 0], pick[:, 1], pick[:, 2]
    intr = cams.intr.astype(np.float64)[v]
    z = depth[v, j, i].astype(np.float64) * scale[v] * (1.0 + rng.normal(0.0, depth_sigma, size=n))
    pc = np.stack([(i + 0.5 - intr[:, 2]) / intr[:, 0] * z, (j + 0.5 - intr[:, 3]) / intr[:, 1] * z, z], 1)
    Rt = cams.w2c.astype(np.float64)[v]
    R, t = Rt[:, :, :3], Rt[:, :, 3]
    centers = np.einsum("nji,nj->ni", R, pc - t)
    nc = normal[v, j, i].astype(np.float64)
    ax = random_unit_vectors(rng, n)
    ang = np.deg2rad(rng.normal(0.0, normal_sigma_deg, size=n))
    # Rodrigues rotation of the camera-frame normal about a random axis
    cosa, sina = np.cos(ang)[:, None], np.sin(ang)[:, None]
    nc = nc * cosa + np.cross(ax, nc) * sina + ax * (ax * nc).sum(1, keepdims=True) * (1.0 - cosa)
    nw = np.einsum("nji,nj->ni", R, nc)
    nw /= np.linalg.norm(nw, axis=1, keepdims=True)
    a = random_unit_vectors(rng, n)
    vx = a - (a * nw).sum(1, keepdims=True) * nw
    vx /= np.linalg.norm(vx, axis=1, keepdims=True)
    vy = np.cross(nw, vx)
    quat = np.array([quat_from_frame(vx[k], vy[k], nw[k]) for k in range(n)])
    radii = np.zeros((n, 4))
    return Planes(centers.astype(np.float32), quat.astype(np.float32), radii.astype(np.float32))


def mono_init(room: Room, depth: np.ndarray, normal: np.ndarray, n: int, seed: int,
              radius_scale: float = 0.5, **kw) -> Planes:
    """mono_points with every radius radius_scale x the distance to the nearest
    other centre (clipped to [0.02, 2] m), computed on the host."""
    p = mono_points(room, depth, normal, n, seed, **kw)
    from scipy.spatial import cKDTree
    c = p.center.astype(np.float64)
    d, _ = cKDTree(c).query(c, k=2)
    p.radii[:] = np.clip(radius_scale * d[:, 1], 0.02, 2.0)[:, None].astype(np.float32)
    return p


def batch_rooms(n_rooms: int, seed0: int = 1000, planes=(200, 3000), views=(16, 96),
                sizes=((240, 320), (360, 480), (480, 640)), n_rect: int = 2000) -> list:
    """n_rooms independent rooms as large_room, each with its own plane count
    K ~ U{planes}, view count V ~ U{views} and resolution drawn from sizes
    (fx = fy = 500 W / 640).  Returns [(Room, K)]."""
    rng = np.random.default_rng(seed0 - 1)
    out = []
    for s in range(n_rooms):
        K = int(rng.integers(planes[0], planes[1] + 1))
        V = int(rng.integers(views[0], views[1] + 1))
        H, W = sizes[int(rng.integers(0, len(sizes)))]
        room = large_room(seed0 + s, n_rect=n_rect, n_views=V, H=H, W=W, f=500.0 * W / 640.0)
        out.append((room, K))
    return out


def random_planes_in_view(seed: int, K: int, depth_range=(1.0, 4.0), half=(0.1, 0.6),
                          fov=0.6, tilt_deg=40.0) -> Planes:
    """K random rectangles in front of an identity camera (for small tests):
    centers spread inside a cone of half-angle ~fov around +z, normals tilted
    from -z by up to tilt_deg, one-sided radii drawn independently."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(*depth_range, size=K)
    xy = rng.uniform(-fov, fov, size=(K, 2)) * z[:, None]
    c = np.concatenate([xy, z[:, None]], axis=1)
    base = np.tile(np.array([0.0, 1.0, 0.0, 0.0]), (K, 1))   # 180 deg about x: n = -z
    ax = random_unit_vectors(rng, K)
    ang = np.deg2rad(rng.uniform(-tilt_deg, tilt_deg, size=K))
    q = quat_mul(quat_axis_angle(ax, ang), base)
    r = rng.uniform(*half, size=(K, 4))
    return Planes(c.astype(np.float32), q.astype(np.float32), r.astype(np.float32))


def identity_cameras(V: int, H: int, W: int, f: float, seed: int = 0, jitter: float = 0.0) -> Cameras:
    """V cameras at the origin looking down +z, optionally with small random
    rotations (jitter, radians) and translations (jitter metres)."""
    rng = np.random.default_rng(seed)
    w2c, intr = [], []
    for v in range(V):
        Rt = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
        if jitter > 0 and v > 0:
            ax = random_unit_vectors(rng, 1)[0]
            th = rng.normal(0, jitter)
            Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
            R = np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * (Kx @ Kx)   # Rodrigues
            Rt = np.concatenate([R, rng.normal(0, jitter, size=(3, 1))], axis=1)
        w2c.append(Rt)
        intr.append([f, f, W / 2.0, H / 2.0])
    return Cameras(np.asarray(w2c, np.float32), np.asarray(intr, np.float32), H, W)
