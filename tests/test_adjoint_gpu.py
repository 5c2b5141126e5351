"""The projection adjoint's outputs are fully written on every call.

The adjoint runs over a list of the Gaussians some view sees, after every
gradient is zeroed.  Every gradient buffer is filled with NaN before the
call, so an entry that the call leaves unwritten shows up; the written values
are checked against the oracle elsewhere (test_parity_gpu.py), here only that
unseen Gaussians get exact zeros, that SH coefficients past the degree in use
get exact zeros, that repeated calls give the same gradients, and that the
moment rows are zero when the backward starts whether the forward zeroed
them beside its kernel or the backward zeroes them itself.  The forward's
zeroing of a caller's region (gs_launch.zero_beside) is exact at unaligned
ends and leaves the forward's outputs unchanged.
"""
import numpy as np
import pytest

from paper_2603_09277_gb300 import scenes

pytestmark = pytest.mark.gpu


def _run(scene, cams, prm, sh_stride, reps=2):
    import torch
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device, targets_to_device
    n = scene["means"].shape[0]
    r = Rasterizer(cams, prm, n, sh_stride=sh_stride)
    p = scene_to_device(scene)
    tg = targets_to_device(scenes.noise_targets(cams, 5))
    outs = []
    for _ in range(reps):
        for t in r.grads.values():
            t.fill_(float("nan"))
        r.step(p, tg, scenes.GAMMA)
        torch.cuda.synchronize()
        outs.append({k: v[:n].cpu().numpy().copy() for k, v in r.grads.items()})
    return r, outs


@pytest.mark.parametrize("views", [1, 3])
def test_every_gradient_written_unseen_zero_sh_tail_zero(views):
    rng = np.random.default_rng(21)
    n = 5000
    scene = scenes.box_scene(n, seed=9)
    # a third of the Gaussians behind the camera (no view sees them)
    behind = rng.random(n) < 1.0 / 3.0
    scene["means"][behind, 2] = -3.0
    # SH degree 1 in blocks of 16 coefficients
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, :4, :] = rng.normal(0.0, 0.3, (n, 4, 3))
    sh[:, 0, :] += 0.5
    scene["sh"] = sh
    scene["sh_degree"] = 1
    prm = scenes.params(sh_degree=1)
    cams = scenes.yaw_cameras([(96, 64), (64, 48), (80, 80)][:views], [0.0, 7.0, -5.0][:views])
    r, outs = _run(scene, cams, prm, sh_stride=16)
    g = outs[0]
    for k, v in g.items():
        assert np.isfinite(v).all(), k
    tt = r.tiles_touched.cpu().numpy().reshape(views, n)
    seen = (tt > 0).any(0)
    assert (~seen).sum() > 1000 and seen.sum() > 1000
    for k, v in g.items():
        assert (v[~seen] == 0).all(), k
    assert (g["sh"][:, 4:, :] == 0).all()
    assert np.abs(g["sh"][seen, :4, :]).sum() > 0
    # the same inputs give the same gradients (no stale state between calls)
    for k in g:
        np.testing.assert_allclose(outs[1][k], g[k], rtol=1e-5, atol=1e-7)


def test_grad2d_zeroed_beside_the_forward_or_by_the_backward():
    # grad2d starts as NaN: the forward zeroes it beside its kernel for the
    # first backward; a second backward of the same forward finds the first
    # one's sums there and zeroes them itself
    import torch
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device, targets_to_device
    n = 4000
    scene = scenes.box_scene(n, seed=12)
    prm = scenes.params()
    cams = scenes.yaw_cameras([(96, 64), (80, 80)], [0.0, 6.0])
    r = Rasterizer(cams, prm, n)
    p = scene_to_device(scene)
    tg = targets_to_device(scenes.noise_targets(cams, 6))
    r.preprocess(p)
    r.bin_sort()
    r.grad2d.fill_(float("nan"))
    r.render_fwd()
    r.loss(tg, scenes.GAMMA)
    outs = []
    for _ in range(2):
        g = r.render_bwd(p)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy().copy() for k, v in g.items()})
    for k in outs[0]:
        assert np.isfinite(outs[0][k]).all(), k
        assert np.abs(outs[0][k]).sum() > 0, k
        np.testing.assert_allclose(outs[1][k], outs[0][k], rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("off,size", [(3, 1001), (16, 4096), (5, 7), (0, 100_003)])
def test_forward_zeroes_an_unaligned_region_exactly(off, size):
    # gs_launch.zero_beside: the forward kernel's CTAs zero the region's
    # 16-byte-aligned body and memsets its ragged ends; the bytes around it
    # stay as they were and the forward's outputs do not change
    import torch
    from paper_2603_09277_gb300 import gs
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device
    n = 3000
    scene = scenes.box_scene(n, seed=13)
    cams = scenes.yaw_cameras([(96, 64), (64, 80)], [0.0, 5.0])
    r = Rasterizer(cams, scenes.params(), n)
    r.preprocess(scene_to_device(scene))
    r.bin_sort()
    gs.gs_render_fwd(r.proj_c, r.N, r.cams_c, r.prm_c, r.sorted_vals, r.tile_ranges, r.image,
                     r.final_T, r.last_idx, r.entropy, gs.make_launch())
    ref = (r.image.clone(), r.final_T.clone(), r.last_idx.clone(), r.entropy.clone())
    buf = torch.full((off + size + 64,), 0xAB, dtype=torch.uint8, device="cuda")
    region = buf[off:off + size]
    gs.gs_render_fwd(r.proj_c, r.N, r.cams_c, r.prm_c, r.sorted_vals, r.tile_ranges, r.image,
                     r.final_T, r.last_idx, r.entropy, gs.make_launch(zero_beside=region))
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert (b[off:off + size] == 0).all()
    assert (b[:off] == 0xAB).all() and (b[off + size:] == 0xAB).all()
    for got, want in zip((r.image, r.final_T, r.last_idx, r.entropy), ref):
        assert torch.equal(got, want)
