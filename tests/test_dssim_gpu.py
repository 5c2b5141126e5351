"""The D-SSIM term of L_base (Sec. 3 Eq. base; 1 - SSIM with 3DGS's SSIM)
on the GPU against the FP64 oracle: the loss value and dL/dC on seeded
images of uneven sizes (including a nearly equal image/target pair, where
the window variances are small), lambda = 0 reducing exactly to the L1 +
entropy call, and a whole step with lambda = 0.2 through the rasterizer.
Tolerances: the loss within 1e-5 relative; dL/dC within 1e-4 relative in
tensor norm and element-wise 1e-4 relative with a floor of 1e-4 of the
largest entry (121-tap FP32 window sums; the moments are centred on the
pixel's own value, so no two large sums cancel)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2603_09277_gb300 import scenes

from parity_util import GRAD_TOL, elementwise_violations, rel_norm_err, run_gpu

pytestmark = pytest.mark.gpu


def _gpu_loss(imgs, tgts, ents, cams, lam, gamma, base=True):
    from paper_2603_09277_gb300 import gs
    cams_c = gs.make_cameras(cams)
    cat = lambda xs, c: torch.as_tensor(np.concatenate([x.reshape(-1, c) for x in xs])
                                        .astype(np.float32)).cuda().contiguous()
    img, tgt = cat(imgs, 3), cat(tgts, 3)
    ent = cat(ents, 1).reshape(-1).contiguous()
    P = img.shape[0]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dimg = torch.zeros(P, 3, device="cuda")
    dent = torch.zeros(P, device="cuda")
    if base:
        ws = torch.empty(gs.gs_loss_base_workspace_size(cams_c), dtype=torch.uint8, device="cuda")
        gs.gs_loss_base(img, tgt, ent, cams_c, lam, gamma, loss, dimg, dent, ws)
    else:
        ws = torch.empty(gs.gs_loss_workspace_size(P), dtype=torch.uint8, device="cuda")
        gs.gs_loss_l1_entropy(img, tgt, ent, cams_c, gamma, loss, dimg, dent, ws)
    torch.cuda.synchronize()
    return float(loss.item()), dimg.cpu().numpy(), dent.cpu().numpy()


def _oracle_loss(imgs, tgts, ents, lam, gamma):
    V = len(imgs)
    L, dCs, dHs = 0.0, [], []
    for i, t, e in zip(imgs, tgts, ents):
        Lv, dC, dH = oracle.loss_base(i.astype(np.float64), e.astype(np.float64), t, gamma, lam,
                                      1.0 / V)
        L += Lv
        dCs.append(dC.reshape(-1, 3))
        dHs.append(dH.reshape(-1))
    return L, np.concatenate(dCs), np.concatenate(dHs)


def _check_grad(g, o):
    """1e-4 relative per tensor; element-wise 1e-4 relative with a floor of
    1e-5 of the largest entry (ten times the rasterizer's floor): SSIM's
    window variances are differences of second moments, and where the image
    is close to its target (variances ~1e-4 against moments ~0.3) FP32
    resolves them to about 1e-7 / 1e-4 relative, which the small entries of
    dL/dC inherit."""
    assert rel_norm_err(g, o) <= GRAD_TOL
    nv, worst = elementwise_violations(g, o, floor=1e-5)
    assert nv == 0, (nv, worst)


@pytest.mark.parametrize("near", [False, True])
def test_dssim_loss_and_gradient_match_oracle(near):
    rng = np.random.default_rng(7 if near else 8)
    sizes = [(61, 45), (130, 97), (16, 16)]
    cams = [scenes.camera(w, h, float(w)) for w, h in sizes]
    tgts = [rng.random((h, w, 3)).astype(np.float32) for w, h in sizes]
    if near:  # image close to the target: SSIM near 1, small window variances
        imgs = [np.clip(t + rng.normal(0, 0.01, t.shape), 0, 1).astype(np.float32) for t in tgts]
    else:
        imgs = [rng.random((h, w, 3)).astype(np.float32) for w, h in sizes]
    ents = [rng.random((h, w)).astype(np.float32) for w, h in sizes]
    for lam in (0.2, 1.0):
        Lg, dg, hg = _gpu_loss(imgs, tgts, ents, cams, lam, 0.015)
        Lo, do, ho = _oracle_loss(imgs, tgts, ents, lam, 0.015)
        assert Lg == pytest.approx(Lo, rel=1e-5)
        _check_grad(dg, do)
        assert np.allclose(hg, ho, rtol=1e-6, atol=0)


def test_dssim_lambda_zero_is_the_l1_entropy_call():
    rng = np.random.default_rng(9)
    cams = [scenes.camera(70, 50, 70.0)]
    imgs = [rng.random((50, 70, 3)).astype(np.float32)]
    tgts = [rng.random((50, 70, 3)).astype(np.float32)]
    ents = [rng.random((50, 70)).astype(np.float32)]
    a = _gpu_loss(imgs, tgts, ents, cams, 0.0, 0.015, base=True)
    b = _gpu_loss(imgs, tgts, ents, cams, 0.0, 0.015, base=False)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_dssim_whole_step_gradients():
    """L_base with lambda = 0.2 and the entropy term through the rasterizer
    (cfg1): the GPU's own loss gradient feeds its backward; parameter
    gradients against the oracle's step with the same loss."""
    from parity_util import gaussian_exclusion, pixel_exclusion
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device, targets_to_device
    scene, cams, targets, prm = scenes.config1()
    N = scene["means"].shape[0]
    L, views, grads, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA, lam=0.2)
    rast = Rasterizer(cams, prm, N)
    p = scene_to_device(scene)
    rast.preprocess(p)
    rast.bin_sort()
    rast.render_fwd()
    rast.loss(targets_to_device(targets), scenes.GAMMA, lam=0.2)
    g = rast.render_bwd(p)
    torch.cuda.synchronize()
    assert float(rast.loss_dev.item()) == pytest.approx(L, rel=1e-5)
    bad = gaussian_exclusion(views[0], cams[0], pixel_exclusion(views[0], cams[0]))
    ok = ~bad
    assert ok.mean() > 0.9
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        gg, oo = g[k].cpu().numpy()[ok], grads[k][ok]
        assert rel_norm_err(gg, oo) <= GRAD_TOL, k
