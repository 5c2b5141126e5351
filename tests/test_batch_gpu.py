"""The 128-entry staging batch of the blending kernels (an autotuner
candidate beside the 256-entry default).

The batch size only changes how many list entries a CTA stages in shared
memory at a time, never which entries a pixel blends or in which order: the
forward outputs equal the 256-entry form's bit for bit, and the whole step
meets the oracle bars (integers bit-exact, images within 1e-5, gradients
within 1e-4 relative).  Lists of up to ~9,000 entries span many batches and
end in ragged tails; 1, 2 and 4 pixels per thread and a persistent grid.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2603_09277_gb300 import scenes

from parity_util import run_gpu
from test_parity_gpu import check_grads, check_lists, check_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def long_lists():
    cams = scenes.yaw_cameras([(61, 45), (130, 97), (256, 200)], [0.0, 7.0, -9.0])
    scene = scenes.box_scene(20_000, seed=13)
    targets = scenes.noise_targets(cams, 14)
    prm = scenes.params()
    L, views, grads, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA)
    dC = np.concatenate([v["dL_dC"].reshape(-1, 3) for v in views])
    dH = np.concatenate([v["dL_dH"].reshape(-1) for v in views])
    return scene, cams, targets, prm, L, views, grads, dC, dH


@pytest.mark.parametrize("ppt,persistent,sh_layout", [(1, 0, 0), (2, 0, 1), (4, 0, 0),
                                                       (2, 152 * 4, 1)])
def test_batch128_matches_batch256_and_the_oracle(long_lists, ppt, persistent, sh_layout):
    scene, cams, targets, prm, L, views, grads, dC, dH = long_lists
    N = scene["means"].shape[0]
    kw = dict(target=targets, dL_dimage=dC, dL_dentropy=dH, ppt=ppt, persistent=persistent,
              sh_layout=sh_layout)
    g = run_gpu(scene, cams, prm, batch=128, **kw)
    ref = run_gpu(scene, cams, prm, batch=256, **kw)
    lengths = np.diff(g["ranges"], axis=1)
    assert (lengths > 1024).any() and ((lengths % 128) != 0).any()
    for k in ("image", "final_T", "last", "entropy"):
        assert np.array_equal(g[k], ref[k]), k
    assert g["loss"] == pytest.approx(ref["loss"], rel=1e-12)
    assert g["loss"] == pytest.approx(L, rel=1e-5)
    check_lists(g, views, cams, N)
    check_pixels(g, views, cams, N)
    check_grads(g, grads, views, cams, N, 1)
