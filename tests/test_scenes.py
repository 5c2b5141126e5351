"""The seeded input generators hold the recipe the workloads are built from.

Same seed, same bits; the shapes and the distributions the recipe states
(uniform box, log-normal scales, unit quaternions, DC colour range, cluster
ball, view sizes and orbits, the sweep's scale factor), checked on samples
large enough that a wrong parameter fails.  Inputs only: nothing here
touches the method's arithmetic.
"""
import math

import numpy as np
import pytest

from paper_2603_09277_gb300 import scenes


def _same(a, b):
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert a[k].dtype == b[k].dtype and np.array_equal(a[k], b[k]), k
        else:
            assert a[k] == b[k], k


def test_same_seed_same_bits_other_seed_other_scene():
    a = scenes.box_scene(5000, seed=3)
    _same(a, scenes.box_scene(5000, seed=3))
    c = scenes.box_scene(5000, seed=4)
    assert not np.array_equal(a["means"], c["means"])
    t1 = scenes.noise_targets([scenes.camera(20, 10, 20.0)], seed=9)
    t2 = scenes.noise_targets([scenes.camera(20, 10, 20.0)], seed=9)
    assert np.array_equal(t1[0], t2[0]) and t1[0].shape == (10, 20, 3)


def test_box_scene_distributions():
    n = 200_000
    s = scenes.box_scene(n, seed=1)
    assert s["means"].shape == (n, 3) and s["means"].dtype == np.float32
    lo, hi = s["means"].min(0), s["means"].max(0)
    assert (lo >= [-1, -1, 2]).all() and (hi <= [1, 1, 6]).all()
    assert np.allclose(s["means"].mean(0), [0, 0, 4], atol=0.02)
    ls = s["log_scales"].astype(np.float64)
    assert abs(ls.mean() + 3.5) < 0.01 and abs(ls.std() - 0.5) < 0.01
    q = s["quats"].astype(np.float64)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6)
    op = s["opacity_logits"].astype(np.float64)
    assert abs(op.mean()) < 0.01 and abs(op.std() - 1.0) < 0.01
    # SH degree 0: DC uniform on [-sqrt(pi), sqrt(pi)], higher bands zero
    dc = s["sh"][:, 0, :].astype(np.float64)
    assert s["sh_degree"] == 0 and (s["sh"][:, 1:, :] == 0).all()
    assert dc.min() >= -math.sqrt(math.pi) and dc.max() <= math.sqrt(math.pi)
    assert abs(dc.mean()) < 0.02


def test_cluster_scene_ball_and_sh():
    s = scenes.cluster_scene(100_000, seed=2)
    r = np.linalg.norm(s["means"].astype(np.float64), axis=1)
    assert r.max() <= 10.0 + 1e-4
    assert s["sh_degree"] == 3 and s["sh"].shape == (100_000, 16, 3)
    sh = s["sh"].astype(np.float64)
    assert abs(sh.std() - 0.2) < 0.005
    ls = s["log_scales"].astype(np.float64)
    assert abs(ls.mean() + 4.0) < 0.01 and abs(ls.std() - 0.7) < 0.01


def test_workload_cameras():
    _, cams, targets, prm = scenes.config1(n=100)
    assert [(c["width"], c["height"], c["fx"]) for c in cams] == [(256, 256, 256.0)]
    assert targets[0].shape == (256, 256, 3)
    _, cams, _, prm = scenes.config3(n=100)
    assert [(c["width"], c["height"]) for c in cams] == scenes.CONFIG3_SIZES
    assert all(c["fx"] == c["width"] for c in cams)
    # every camera looks at (0, 0, 4): that point projects to the image centre
    for c in cams:
        w = c["world_to_cam"].astype(np.float64)
        pc = w[:, :3] @ np.array([0.0, 0.0, 4.0]) + w[:, 3]
        u = c["fx"] * pc[0] / pc[2] + c["cx"]
        v = c["fy"] * pc[1] / pc[2] + c["cy"]
        assert abs(u - c["width"] / 2) < 1e-3 and abs(v - c["height"] / 2) < 1e-3
    _, cams, _, prm = scenes.config2(n=100)
    assert (cams[0]["width"], cams[0]["height"]) == (1237, 822) and prm["sh_degree"] == 3


@pytest.mark.parametrize("k", [-2, 0, 3])
def test_sweep_scales_by_powers_of_half(k):
    a, _, _, _ = scenes.config4(k=0)
    b, _, _, _ = scenes.config4(k=k)
    d = b["log_scales"].astype(np.float64) - a["log_scales"].astype(np.float64)
    assert np.allclose(d, k * math.log(0.5), atol=1e-5)
    assert np.array_equal(a["means"], b["means"])


def test_cfg5_view_and_box_and_the_density_matched_cfg3():
    s, cams, targets, prm = scenes.config5(n=50_000)
    assert [(c["width"], c["height"], c["fx"]) for c in cams] == [(1920, 1080, 1920.0)]
    assert targets[0].shape == (1080, 1920, 3) and prm["sh_degree"] == 0
    m = s["means"].astype(np.float64)
    ar = 1080 / 1920
    assert (np.abs(m[:, 0]) <= 1).all() and (np.abs(m[:, 1]) <= ar + 1e-6).all()
    assert m[:, 1].max() > 0.98 * ar and m[:, 1].min() < -0.98 * ar  # the 16:9 extent is filled
    # the labelled density-matched cfg3 variant shifts the log-scale mean by ln((1e4/n)^(1/3))
    a, _, _, _ = scenes.config3(n=20_000)
    b, _, _, _ = scenes.config3(n=20_000, density_matched=True)
    d = b["log_scales"].astype(np.float64) - a["log_scales"].astype(np.float64)
    assert np.allclose(d, math.log((1e4 / 20_000) ** (1.0 / 3.0)), atol=1e-5)


def test_orbit_cameras_look_at_the_centre():
    cams = scenes.orbit_cameras(32, 64, 48, seed=3)
    assert len(cams) == 32
    for c in cams:
        w = c["world_to_cam"].astype(np.float64)
        pc = w[:, :3] @ np.array([0.0, 0.0, 4.0]) + w[:, 3]
        assert abs(pc[0]) < 1e-4 and abs(pc[1]) < 1e-4
        assert abs(pc[2] - math.hypot(4.0, 0.5)) < 1e-4  # radius 4, height offset 0.5
