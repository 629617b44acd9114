"""Host-side logic that needs no GPU: the autotuner's cache keys and file cache,
and the seeded scene generators' determinism (every input is seeded)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2412_03451_gb300 import autotune as AT
from paper_2412_03451_gb300 import scenes as S


def test_autotune_key_buckets_planes_and_sorts_sizes():
    k = AT._key([(480, 640), (240, 320), (480, 640)], 8, 3000)
    assert k == "240x320,480x640|v8|k11"
    assert AT._key([(480, 640)], 8, 2048) == AT._key([(480, 640)], 8, 4095)
    assert AT._key([(480, 640)], 8, 2047) != AT._key([(480, 640)], 8, 2048)


def test_autotune_answers_from_the_file_cache_without_timing(tmp_path, monkeypatch):
    key = AT._key([(480, 640)], 8, 3000)
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: {"tile": [32, 8], "warps": 2, "ms": {"32x8/w2": 1.0}}}))
    monkeypatch.setenv("PS_AUTOTUNE_CACHE", str(path))
    monkeypatch.setattr(AT, "_cache", {})

    def no_renderer(tile, warps):
        raise AssertionError("a cached key must not be timed")

    tile, warps, ms = AT.pick_launch(no_renderer, None, None, None, 20.0, key)
    assert tile == (32, 8) and warps == 2 and ms == {"32x8/w2": 1.0}


def test_autotune_searches_tiles_and_warps(monkeypatch):
    # every (tile, warps) pair is timed on the caller's renderer and the fastest is kept
    monkeypatch.setattr(AT, "_cache", {})
    monkeypatch.delenv("PS_AUTOTUNE_CACHE", raising=False)
    seen = []
    t = {"now": 0.0}

    class FakeEvent:
        def __init__(self, enable_timing=False):
            self.at = 0.0

        def record(self):
            self.at = t["now"]

        def elapsed_time(self, other):
            return other.at - self.at

    class FakeRenderer:
        def __init__(self, tile, warps):
            self.cost = 1.0 + (tile != (8, 8)) + 0.5 * (warps != 2)
            seen.append((tile, warps))

        def ensure_capacity(self, *a, **k):
            return False

        def project_bin(self, *a):
            t["now"] += self.cost

        def fused(self, *a):
            pass

    monkeypatch.setattr(AT.torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(AT.torch.cuda, "synchronize", lambda: None)
    flat = torch.zeros(11)
    tile, warps, ms = AT.pick_launch(FakeRenderer, flat, None, None, 20.0, "k")
    assert (tile, warps) == ((8, 8), 2)
    assert sorted(seen) == sorted((tl, w) for tl in AT.TILES for w in AT.WARPS)
    assert set(ms) == {"%dx%d/w%d" % (tl[0], tl[1], w) for tl in AT.TILES for w in AT.WARPS}


def test_scene_generators_are_seeded():
    a, b = S.large_room(1003, n_rect=300, n_views=4), S.large_room(1003, n_rect=300, n_views=4)
    assert np.array_equal(a.gt.center, b.gt.center) and np.array_equal(a.gt.quat, b.gt.quat)
    assert np.array_equal(a.cams.w2c, b.cams.w2c)
    c = S.large_room(1004, n_rect=300, n_views=4)
    assert not np.array_equal(a.gt.center, c.gt.center)
    p, q = S.surface_init(a, 200, 5), S.surface_init(a, 200, 5)
    assert np.array_equal(p.center, q.center) and np.array_equal(p.radii, q.radii)


def test_sphere_init_on_bounding_sphere_facing_its_centre():
    # Sec. 4.3 ablation start: planes of radius 0.05 on the scene's bounding sphere
    # (centre of the room box, radius half its diagonal), normals toward the centre
    from scipy.spatial.transform import Rotation
    room = S.large_room(1005, n_rect=300, n_views=4)
    p = S.sphere_init(room, 500, 3)
    size = np.asarray(room.size, np.float64)
    centre = size / 2.0
    R = 0.5 * np.linalg.norm(size)
    off = p.center.astype(np.float64) - centre
    assert np.allclose(np.linalg.norm(off, axis=1), R, rtol=1e-6)
    # third column of the rotation of (w, x, y, z) is the plane normal (Eq. 2-3)
    q = p.quat.astype(np.float64)
    mats = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], axis=1)).as_matrix()
    n = mats[:, :, 2]
    assert np.allclose(n, -off / np.linalg.norm(off, axis=1, keepdims=True), atol=1e-5)
    assert np.all(p.radii == np.float32(0.05))
    # directions cover the sphere (no hemisphere left empty)
    u = off / R
    assert (u[:, 0] > 0.5).any() and (u[:, 0] < -0.5).any() and (u[:, 2] > 0.5).any() and (u[:, 2] < -0.5).any()
    q2 = S.sphere_init(room, 500, 3)
    assert np.array_equal(p.center, q2.center) and np.array_equal(p.quat, q2.quat)
