"""The training schedule around the rasterizer (Sec. 5.2): camera and target
scaling of the resolution scheduler, the r_max rule (mean per-tile list at
most ~150, factor capped at 4), the coarse-to-fine levels, and the epoch plan
of the scale reset and the entropy term.  CPU tests pin the host logic to
the pinhole model, to block averages and to the oracle's lists; the GPU test
takes r_max from the library's lists and the oracle's and requires the same
factor."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_09277_gb300 import scenes, schedule


def _pinhole(cam, X):
    wtc = np.asarray(cam["world_to_cam"], np.float64)
    t = wtc[:, :3] @ X + wtc[:, 3]
    return np.array([cam["fx"] * t[0] / t[2] + cam["cx"], cam["fy"] * t[1] / t[2] + cam["cy"]])


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_scaled_camera_maps_points_to_the_coarse_pixel_grid(r):
    cam = scenes.orbit_cameras(3, 1237, 822, seed=1)[1]
    c = schedule.scaled_camera(cam, r)
    assert (c["width"], c["height"]) == (1237 // r, 822 // r)
    rng = np.random.default_rng(r)
    for X in rng.uniform(-1, 1, (5, 3)) + np.array([0, 0, 4.0]):
        # a coarse pixel (u, v) covers full pixels [r u, r u + r): positions scale by 1/r
        assert np.allclose(_pinhole(c, X), _pinhole(cam, X) / r, rtol=0, atol=1e-9)


def test_downsample_image_is_the_block_mean():
    rng = np.random.default_rng(0)
    img = rng.random((23, 31, 3))
    for r in (1, 2, 3, 4):
        d = schedule.downsample_image(img, r)
        H, W = 23 // r, 31 // r
        assert d.shape == (H, W, 3)
        for y in range(H):
            for x in range(W):
                assert np.allclose(d[y, x], img[r * y:r * y + r, r * x:r * x + r].mean((0, 1)))


def test_choose_r_max_rule():
    # longer lists at coarser factors; the largest factor <= 4 at or below the threshold
    assert schedule.choose_r_max(lambda r: 40.0 * r) == 3        # 120 at r = 3, 160 at r = 4
    assert schedule.choose_r_max(lambda r: 10.0 * r) == 4        # capped at 4
    assert schedule.choose_r_max(lambda r: 200.0 * r) == 1       # even r = 2 exceeds
    assert schedule.choose_r_max(lambda r: 150.0 if r == 2 else 151.0) == 2  # at the threshold
    assert schedule.choose_r_max(lambda r: 40.0 * r, cap=2) == 2
    calls = []
    schedule.choose_r_max(lambda r: calls.append(r) or 100.0)
    assert calls == [4]  # stops at the first qualifying factor


def test_resolution_levels_coarse_to_fine():
    lv = schedule.resolution_levels(4, 30)
    assert lv[0] == 4 and (np.diff(lv) <= 0).all()
    assert (lv[15:] == 1).all() and (lv[:15] > 1).all()
    counts = [int((lv == k).sum()) for k in (4, 3, 2)]
    assert sum(counts) == 15 and max(counts) - min(counts) <= 1
    assert (schedule.resolution_levels(1, 10) == 1).all()
    assert (schedule.resolution_levels(2, 10)[:5] == 2).all()


def test_epoch_plan_reset_entropy_and_stage_adaptive_values():
    plan = schedule.EpochSchedule(epochs=60, reset_every=20, r_max=3)
    resets = [e for e in range(60) if plan.reset_after(e)]
    assert resets == [19, 39]  # every 20 epochs, not after the last one
    on = [plan.entropy_on(e) for e in range(60)]
    for start in (0, 20, 40):  # every other epoch of each reset period
        assert on[start:start + 20] == [False, True] * 10
    lv = plan.levels()
    for e in range(60):
        g = plan.gamma_at(e)
        assert g == (0.0 if not on[e] else (0.015 if lv[e] == 1 else 0.005))
        assert plan.zeta_at(e) == (0.2 if lv[e] == 1 else 0.5)
    order = plan.image_order(32, seed=1)
    assert order.shape == (60, 200) and order.min() >= 0 and order.max() < 32


def test_coarse_levels_lengthen_the_oracle_lists():
    """The premise of the r_max rule, on the oracle: the mean per-tile list
    length grows with the downsampling factor (the same Gaussians over
    fewer tiles)."""
    scene, cams, _, prm = scenes.config1()
    means = []
    for r in (1, 2, 4):
        cam = schedule.scaled_camera(cams[0], r)
        proj = oracle.preprocess(scene, cam, prm)
        ts, ids = oracle.build_lists(proj, cam)
        means.append(len(ids) / (len(ts) - 1))
    assert means[0] < means[1] < means[2]


@pytest.mark.gpu
def test_r_max_from_gpu_lists_equals_oracle():
    torch = pytest.importorskip("torch")
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device
    scene, cams, _, prm = scenes.config1()
    N = scene["means"].shape[0]
    p = scene_to_device(scene)

    def gpu_mean(r):
        cam = schedule.scaled_camera(cams[0], r)
        rast = Rasterizer([cam], prm, N)
        rast.preprocess(p)
        return rast.bin_sort() / rast.total_tiles

    def ora_mean(r):
        cam = schedule.scaled_camera(cams[0], r)
        ts, ids = oracle.build_lists(oracle.preprocess(scene, cam, prm), cam)
        return len(ids) / (len(ts) - 1)

    for thr in (50.0, 150.0, 400.0, 2000.0):
        assert (schedule.choose_r_max(gpu_mean, threshold=thr)
                == schedule.choose_r_max(ora_mean, threshold=thr))
    for r in (1, 2, 3, 4):
        assert gpu_mean(r) == pytest.approx(ora_mean(r), rel=1e-3)
