"""The torch.autograd wrappers over the C ABI (rasterize, l1_entropy_loss).

Gradients that flow through the wrappers to the parameter tensors equal the
FP64 oracle's on a small scene, the SH gradient included; an FP32 central
difference of the loss through the same wrappers agrees with the autograd
gradient on well-conditioned coordinates.  Also the invariant of the weights
(Suppl. A): with every colour 1 the image is the sum of the blending weights,
so image + final T = 1 per pixel.
"""
import numpy as np
import pytest

import oracle
from paper_2603_09277_gb300 import scenes

from parity_util import GRAD_TOL, elementwise_violations

pytestmark = pytest.mark.gpu

GAMMA = 0.015


def _scene():
    scene, cams, targets, prm = scenes.tiny_scene(24, seed=5, width=48, height=40, sh_degree=1)
    return scene, cams, targets, prm


def _loss_and_grads(scene, cams, targets, prm, backward=True, sh_layout=0):
    import torch
    from paper_2603_09277_gb300.rasterize import (PARAM_KEYS, Rasterizer, l1_entropy_loss,
                                                  rasterize, scene_to_device, targets_to_device)
    n = scene["means"].shape[0]
    r = Rasterizer(cams, prm, n, sh_stride=scene["sh"].shape[1])
    p = scene_to_device(scene, requires_grad=True, sh_layout=sh_layout)
    img, ent = rasterize(p, r)
    loss = l1_entropy_loss(img, ent, targets_to_device(targets), r, GAMMA)
    if backward:
        loss.backward()
    torch.cuda.synchronize()

    def grad(k):  # the SH gradient back in [N][K][3]
        t = p[k].grad.detach()
        return (t.transpose(0, 1) if k == "sh" and sh_layout == 1 else t).cpu().numpy()
    return float(loss.item()), {k: (grad(k) if backward else None) for k in PARAM_KEYS}, r


@pytest.mark.parametrize("sh_layout", [0, 1])
def test_autograd_gradients_match_the_oracle(sh_layout):
    scene, cams, targets, prm = _scene()
    L, _, ora, _ = oracle.step(scene, cams, targets, prm, GAMMA)
    loss, grads, _ = _loss_and_grads(scene, cams, targets, prm, sh_layout=sh_layout)
    assert loss == pytest.approx(L, rel=1e-5)
    n = scene["means"].shape[0]
    K = (prm["sh_degree"] + 1) ** 2
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        got = grads[k][:n]
        want = np.asarray(ora[k])[:n]
        if k == "sh":
            got, want = got[:, :K], want[:, :K]
        err = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
        assert err <= GRAD_TOL, (k, err)  # (no pixel of this scene lies near a threshold)
        nv, worst = elementwise_violations(got, want)
        assert nv == 0, (k, nv, worst)


def test_autograd_gradient_against_fp32_central_difference():
    scene, cams, targets, prm = _scene()
    _, grads, _ = _loss_and_grads(scene, cams, targets, prm)
    # the Gaussian with the largest opacity-logit gradient, away from thresholds
    g = int(np.argmax(np.abs(grads["opacity_logits"])))
    h = 1e-2
    for key, idx in (("opacity_logits", (g,)), ("means", (g, 0)), ("log_scales", (g, 1))):
        vals = []
        for sgn in (1.0, -1.0):
            s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
            s2[key][idx] += sgn * h
            loss, _, _ = _loss_and_grads(s2, cams, targets, prm, backward=False)
            vals.append(loss)
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = float(grads[key][idx])
        assert abs(fd - ad) <= 0.05 * abs(ad) + 1e-6, (key, fd, ad)


def test_weights_and_final_transmittance_sum_to_one():
    import torch
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device
    scene = scenes.box_scene(3000, seed=8)
    # rgb = Y0 sh0 + 0.5 = 1 in every channel: the image is the sum of the weights
    scene["sh"][:] = 0.0
    scene["sh"][:, 0, :] = 0.5 / 0.28209479177387814
    cams = [scenes.camera(80, 64, 80.0)]
    prm = scenes.params()
    r = Rasterizer(cams, prm, 3000, sh_stride=scene["sh"].shape[1])
    p = scene_to_device(scene)
    r.preprocess(p)
    r.bin_sort()
    r.render_fwd()
    torch.cuda.synchronize()
    img = r.image.cpu().numpy().astype(np.float64)
    T = r.final_T.cpu().numpy().astype(np.float64)
    assert (T < 0.999).mean() > 0.5  # most pixels are covered
    for ch in range(3):
        assert np.abs(img[:, ch] + T - 1.0).max() < 2e-5
