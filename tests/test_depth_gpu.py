"""The depth sort key on the GPU against the oracle where FP32 rounding is
delicate.

Both sides define the key as the FP32 rounding of the FP64 value
((R20 mx + R21 my) + R22 mz) + t2.  The GPU evaluates it with error-free FP32
transformations and falls back to the FP64 expression only when that
estimate lies within its error bound of an FP32 rounding midpoint.  The means
below put the exact depth on a midpoint, a few FP64 ulps from one, or
(2^-59 below a midpoint) where the FP64 rounding itself lands on the midpoint
and the tie goes to the even neighbour, not to the side of the exact value:
there the fallback is the only way to reach the defined key.  Every key must
match the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2603_09277_gb300 import scenes

pytestmark = pytest.mark.gpu


def _camera(row2, t2):
    wtc = np.zeros((3, 4), np.float32)
    wtc[0, :3] = (0.0, 0.0, 1.0)
    wtc[1, :3] = (0.0, 1.0, 0.0)
    wtc[2, :3] = row2
    wtc[2, 3] = t2
    return {"width": 64, "height": 64, "fx": 64.0, "fy": 64.0, "cx": 32.0, "cy": 32.0,
            "world_to_cam": wtc, "cam_pos": np.zeros(3, np.float32)}


def _gpu_depth(scene, cam, prm):
    import torch
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device
    n = scene["means"].shape[0]
    r = Rasterizer([cam], prm, n, keep_debug=True)
    r.preprocess(scene_to_device(scene))
    torch.cuda.synchronize()
    return r.depth[:n].cpu().numpy()


def _check(scene, cam, prm):
    want = oracle.preprocess(scene, cam, prm)["depth"].astype(np.float32)
    got = _gpu_depth(scene, cam, prm)
    bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
    assert bad.size == 0, (bad[:8], got[bad[:8]], want[bad[:8]])
    return want


def test_depth_key_where_fp64_rounding_decides_the_tie():
    # R20 = 2^-23 (1 + 2^-18), mx = 1 - 2^-18: R20 mx = 2^-23 - 2^-59 exactly,
    # so with my = 2 + j 2^-22 the exact depth lies 2^-59 below the FP32
    # midpoint my + 2^-23; FP64 rounds it onto the midpoint and the FP32
    # rounding then goes to the even one of my and my + 2^-22.
    rng = np.random.default_rng(7)
    n = 8192
    scene = scenes.box_scene(n, seed=3)
    r20 = np.float32(2.0 ** -23 * (1.0 + 2.0 ** -18))
    cam = _camera((r20, 1.0, 0.0), 0.0)
    j = rng.integers(0, 1 << 21, n)
    my = (2.0 + j * 2.0 ** -22).astype(np.float32)
    mx = np.full(n, 1.0 - 2.0 ** -18, np.float32)
    # a quarter of the rows: other mx near 1 and random values (ordinary cases)
    k = n // 4
    mx[:k] = rng.choice(np.array([1.0, 1.0 + 2.0 ** -18, 1.0 - 2.0 ** -17], np.float32), k)
    mx[k:2 * k] = rng.uniform(0.5, 2.0, k).astype(np.float32)
    scene["means"] = np.stack([mx, my, rng.uniform(-1, 1, n).astype(np.float32)], 1)
    want = _check(scene, cam, scenes.params())
    # the crafted rows with odd j are the ones where the defined key is the
    # upper neighbour although the exact depth is below the midpoint
    tie = np.arange(n) >= 2 * k
    odd = tie & (j % 2 == 1)
    assert odd.sum() > 1000
    assert (want[odd] == my[odd] + np.float32(2.0 ** -22)).all()
    assert (want[tie & (j % 2 == 0)] == my[tie & (j % 2 == 0)]).all()


def test_depth_key_on_and_near_midpoints():
    # R2 = (1, 2^-24, 0), t2 = 0: depth = mx + 2^-24 my exactly (FP64 holds
    # it), with mx in [1, 2) (FP32 spacing 2^-23): my = +-1 gives exact ties,
    # my = +-(1 +- k 2^-23) values a few 2^-47 off a midpoint, and random my
    # ordinary values.
    rng = np.random.default_rng(11)
    n = 8192
    scene = scenes.box_scene(n, seed=4)
    cam = _camera((1.0, 2.0 ** -24, 0.0), 0.0)
    mx = rng.uniform(1.0, 2.0, n).astype(np.float32)
    sgn = rng.choice(np.array([-1.0, 1.0]), n)
    kk = rng.integers(-4, 5, n)
    my = (sgn * (1.0 + kk * 2.0 ** -23)).astype(np.float32)
    my[: n // 4] = rng.uniform(-3.0, 3.0, n // 4).astype(np.float32)
    scene["means"] = np.stack([mx, my, np.zeros(n, np.float32)], 1)
    _check(scene, cam, scenes.params())


def test_depth_key_cancellation_zero_and_tiny():
    # terms of size ~1e3 that cancel to small depths, exact zeros and values
    # near the bottom of the normal range (the estimate is not trusted there)
    rng = np.random.default_rng(13)
    n = 4096
    scene = scenes.box_scene(n, seed=5)
    cam = _camera((0.6, 0.8, 0.0), 1.5)
    x = rng.uniform(-1e3, 1e3, n).astype(np.float32)
    y = (-(0.6 / 0.8) * x.astype(np.float64) + rng.normal(0, 1e-3, n)).astype(np.float32)
    means = np.stack([x, y, rng.uniform(-1, 1, n).astype(np.float32)], 1)
    means[:64] = 0.0
    means[64:128, 0] = (rng.uniform(1, 2, 64) * 2.0 ** -120).astype(np.float32)
    means[64:128, 1] = 0.0
    scene["means"] = means
    cam0 = _camera((0.6, 0.8, 0.0), 0.0)
    _check(scene, cam0, scenes.params())
    _check(scene, cam, scenes.params())
