"""The seeded synthetic workloads have the shapes their recipes state: sizes,
views per point, outlier share, ranges of the batched problems, distinct
(camera, point) pairs, a shuffled observation order, every point in front
of every camera that observes it, and the same arrays for the same seed."""
import numpy as np
import pytest

import scenegen
from oracle.ba_oracle import _camera_point


def _views(sc):
    return np.bincount(sc.pt_idx, minlength=sc.P)


def _pairs_distinct(sc):
    key = sc.cam_idx.astype(np.int64) * sc.P + sc.pt_idx
    return np.unique(key).shape[0] == sc.O


def _in_front(sc, cams, points, chunk=1 << 20):
    # the camera looks down -z: a point in front has X_cam[2] < 0
    worst = -np.inf
    for a in range(0, sc.O, chunk):
        _, _, _, _, Pc = _camera_point(cams, points, sc.cam_idx[a:a + chunk], sc.pt_idx[a:a + chunk])
        worst = max(worst, float(Pc[:, 2].max()))
    return worst


@pytest.fixture(scope="module")
def ba4000():
    return scenegen.config_scene("ba4000")


def test_ba4000_recipe(ba4000):
    sc = ba4000
    assert (sc.C, sc.P, sc.O) == (4000, 1_200_000, 8_044_313)
    v = _views(sc)
    # 2 + Geom0(1/5.7): mean 6.7, at least two views
    assert v.min() >= 2 and abs(v.mean() - 6.7) < 0.02
    assert _pairs_distinct(sc)
    assert sc.huber_delta == 0.0
    # the observation order is shuffled, so both sorts do real work
    assert np.any(np.diff(sc.cam_idx) < 0) and np.any(np.diff(sc.pt_idx) < 0)
    # 1 px noise per component
    assert abs(sc.noise.std() - 1.0) < 0.01


def test_ba250_recipe():
    sc = scenegen.config_scene("ba250")
    assert (sc.C, sc.P) == (250, 60_000) and 470_000 < sc.O < 490_000
    v = _views(sc)
    assert v.min() >= 2 and abs(v.mean() - 8.0) < 0.05
    assert _pairs_distinct(sc)
    # 2 % outliers of 20 px on top of 1 px noise, Huber delta 1 px
    out = np.linalg.norm(sc.noise, axis=1) > 10.0
    assert abs(out.mean() - 0.02) < 0.002
    assert sc.huber_delta == 1.0
    assert _in_front(sc, sc.cams_gt, sc.points_gt) < 0.0
    assert _in_front(sc, sc.cams_init, sc.points_init) < 0.0


def test_ba16_and_ba64_recipes():
    a = scenegen.config_scene("ba16")
    v = _views(a)
    assert (a.C, a.P) == (16, 1000) and v.min() >= 4 and v.max() <= 12
    assert 7_500 < a.O < 8_500 and _pairs_distinct(a)
    assert _in_front(a, a.cams_gt, a.points_gt) < 0.0
    b = scenegen.config_scene("ba64")
    assert (b.C, b.P) == (64, 10_000) and 75_000 < b.O < 85_000 and _pairs_distinct(b)
    assert _in_front(b, b.cams_gt, b.points_gt) < 0.0


def test_batch512_recipe():
    scenes = scenegen.batch_scenes(512, seed=4)
    assert len(scenes) == 512
    C = np.array([s.C for s in scenes])
    P = np.array([s.P for s in scenes])
    assert C.min() >= 5 and C.max() <= 20 and P.min() >= 200 and P.max() <= 3000
    # log-uniform point counts: the median sits near the geometric mean
    assert abs(np.log(np.median(P)) - 0.5 * (np.log(200) + np.log(3000))) < 0.2
    for s in scenes[:64]:
        v = _views(s)
        assert v.min() >= 4 and v.max() <= min(10, s.C) and _pairs_distinct(s)
    assert 3.3e6 < sum(s.O for s in scenes) < 4.1e6


def test_same_seed_same_scene():
    a = scenegen.ring_scene(30, 500, seed=7, outlier_frac=0.05, huber_delta=1.0)
    b = scenegen.ring_scene(30, 500, seed=7, outlier_frac=0.05, huber_delta=1.0)
    for f in ("cam_idx", "pt_idx", "noise", "cams_init", "points_init", "cams_gt", "points_gt"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    c = scenegen.ring_scene(30, 500, seed=8, outlier_frac=0.05, huber_delta=1.0)
    assert not np.array_equal(a.noise, c.noise)
