"""CPU checks of the seeded workload generators' rules: the served rooms (radius
scaling, the camera outside every sphere), the served jobs' statistics grid, and
that the main workload does not move."""
import hashlib
import math

import numpy as np

import mars_workloads as W


def _digest(sc):
    return hashlib.sha1(b"".join(np.ascontiguousarray(getattr(sc, f)).tobytes()
                                 for f in ("quads", "spheres", "materials", "camera"))).hexdigest()


def test_served_rooms_keep_the_camera_outside_every_sphere():
    for seed in range(12):
        for n in (16, 64, 500, 4096):
            sc = W.guided_room_scene(seed, 8, 8, n_spheres=n)
            s = np.asarray(sc.spheres, np.float64)
            cam = np.asarray(sc.camera[:3], np.float64)
            assert (np.linalg.norm(s[:, :3] - cam, axis=1) > s[:, 3]).all(), (seed, n)


def test_dense_rooms_hold_no_more_sphere_volume_than_64_spheres():
    """Beyond 64 spheres the radii shrink by (64 / n)^(1/3): the expected sphere
    volume of the room stays that of 64 spheres (within sampling noise)."""
    vol = {}
    for n in (64, 512, 4096):
        v = []
        for seed in range(8):
            s = np.asarray(W.guided_room_scene(seed, 8, 8, n_spheres=n).spheres, np.float64)
            v.append((4.0 / 3.0 * math.pi * s[:, 3] ** 3).sum())
        vol[n] = np.mean(v)
    assert 0.7 < vol[512] / vol[64] < 1.3 and 0.8 < vol[4096] / vol[64] < 1.2
    s = np.asarray(W.guided_room_scene(3, 8, 8, n_spheres=4096).spheres, np.float64)
    assert s[:, 3].max() <= 0.5 * 0.25 + 1e-6


def test_served_jobs_grid_follows_their_samples():
    reqs = W.serving_requests(64, rate=20.0, seed=11)
    for r in reqs:
        px = r["scene"].width * r["scene"].height
        n = r["grid_n"]
        assert 8 <= n <= 32
        want = min(32, max(8, round((px * r["iterations"] / 64.0) ** (1.0 / 3.0))))
        assert n == want
        if 8 < n < 32:   # about 64 camera samples per cell over the job
            assert 64 / 4 < px * r["iterations"] / n ** 3 < 64 * 4


def test_the_main_workload_is_unchanged_by_the_room_rules():
    """The 64-sphere room of seed 0 has no sphere around the camera, so the
    rules leave it as it was (its scene arrays hash as before)."""
    sc = W.config_guided(512, 512).scene
    assert len(sc.spheres) == 64
    s = np.asarray(sc.spheres, np.float64)
    assert (np.linalg.norm(s[:, :3] - np.asarray(sc.camera[:3]), axis=1) > s[:, 3]).all()
    assert _digest(sc)[:12] == "e454ed1ee3b7"
