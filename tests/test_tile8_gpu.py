"""8x8-pixel tiles (the tile side of LiteGS and of the paper's own runs,
Sec. 5 "Effect of tile sizes"): the whole GPU step against the FP64 oracle
run with the same tile side, at the same bars as the 16x16 path: integers
bit-exact, images within 1e-5, gradients within 1e-4 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2603_09277_gb300 import scenes

from parity_util import run_gpu
from test_parity_gpu import check_grads, check_lists, check_pixels, check_projection

pytestmark = pytest.mark.gpu


def _case(scene, cams, targets, prm, **kw):
    L, views, grads, g9 = oracle.step(scene, cams, targets, prm, scenes.GAMMA)
    dC = np.concatenate([v["dL_dC"].reshape(-1, 3) for v in views])
    dH = np.concatenate([v["dL_dH"].reshape(-1) for v in views])
    g = run_gpu(scene, cams, prm, target=targets, dL_dimage=dC, dL_dentropy=dH, **kw)
    return L, views, grads, g


@pytest.fixture(scope="module")
def cfg1_tile8():
    scene, cams, targets, prm = scenes.config1()
    prm["tile"] = 8
    return (scene, cams, targets, prm) + _case(scene, cams, targets, prm)


def test_tile8_projection_and_lists(cfg1_tile8):
    scene, cams, targets, prm, L, views, grads, g = cfg1_tile8
    N = scene["means"].shape[0]
    assert len(g["ranges"]) == 32 * 32  # 256 x 256 px in 8-px tiles
    check_projection(g, views, cams, N)
    assert g["P"] == views[0]["lists"][0][-1] or views[0]["proj"]["boundary"].any()
    check_lists(g, views, cams, N)


def test_tile8_pixels_loss_and_gradients(cfg1_tile8):
    scene, cams, targets, prm, L, views, grads, g = cfg1_tile8
    N = scene["means"].shape[0]
    check_pixels(g, views, cams, N)
    assert g["loss"] == pytest.approx(L, rel=1e-5)
    check_grads(g, grads, views, cams, N, 1)


@pytest.mark.parametrize("ppt,persistent,sh_layout", [(1, 0, 0), (2, 152 * 8, 1)])
def test_tile8_launch_forms_and_uneven_views(ppt, persistent, sh_layout):
    # views whose sizes are not multiples of 8, one pixel per thread or a
    # persistent grid over the list-length queue (with the SH coefficients
    # in layout 1)
    sizes = [(61, 45), (130, 97), (256, 200)]
    cams = scenes.yaw_cameras(sizes, [0.0, 7.0, -9.0])
    scene = scenes.box_scene(4_000, seed=11)
    targets = scenes.noise_targets(cams, 12)
    prm = scenes.params(tile=8)
    L, views, grads, g = _case(scene, cams, targets, prm, ppt=ppt, persistent=persistent,
                               sh_layout=sh_layout)
    N = scene["means"].shape[0]
    check_lists(g, views, cams, N)
    check_pixels(g, views, cams, N)
    check_grads(g, grads, views, cams, N, 1)


def test_tile8_lists_are_the_16px_lists_refined():
    """Every 8-px tile's list is the 16-px list of its parent tile restricted
    to the Gaussians whose 8-px rect covers it (same order)."""
    scene, cams, _, prm = scenes.config1()
    g16 = run_gpu(scene, cams, prm)
    g8 = run_gpu(scene, cams, dict(prm, tile=8))
    rect8 = g8["rect"]
    for ty in range(32):
        for tx in range(32):
            t8, t16 = ty * 32 + tx, (ty // 2) * 16 + tx // 2
            a, b = g8["ranges"][t8]
            c, d = g16["ranges"][t16]
            parent = g16["vals"][c:d]
            r = rect8[parent]
            keep = (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
            assert (g8["vals"][a:b] == parent[keep]).all()
