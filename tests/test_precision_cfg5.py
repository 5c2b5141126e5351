"""Mixed-precision staging at full size (3,000,000 Gaussians, one 1920x1080
view): render records in FP32, FP16 and BF16 (the 2D mean always FP32;
exponent, transmittance and accumulation FP32), each against the FP64
oracle on sampled pixels and sampled Gaussians.  The FP32 outputs must
meet the parity bar: the forward on the non-excluded pixels, the gradients
of the sampled small Gaussians that are reached and excluded by no
threshold rule (per tensor within 1e-4 relative; element-wise within 1e-4
with the floor on those no near-threshold flip can move).
The 16-bit forms have no bar (their error per output is the measured
quantity) and only sanity bounds.
With GS_REPORT_DIR set the table is written there as precision_cfg5.json."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2603_09277_gb300 import scenes

from parity_util import (GRAD_TOL, IMG_TOL, elementwise_violations, flip_sensitive,
                         gaussian_exclusion, last_ids_gpu, last_ids_oracle, pixel_exclusion,
                         rel_norm_err, run_gpu)

pytestmark = pytest.mark.gpu


def test_cfg5_staging_precision_error_per_output():
    scene, cams, targets, prm = scenes.config5()
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    N = scene["means"].shape[0]
    TX, TY = oracle.tile_grid(cam)
    proj = oracle.preprocess(scene, cam, prm)
    rng = np.random.default_rng(0)
    # candidates: the 48 front-most unflagged Gaussians with rects of at most
    # 6x6 tiles (deeper ones are rarely reached before T < t_min in this dense
    # scene); sampled tiles: their rects plus 48 random tiles
    cand = np.nonzero((proj["tiles"] > 0) & (proj["tiles"] <= 36) & (proj["boundary"] == 0))[0]
    cand = cand[np.argsort(proj["depth"][cand], kind="stable")[:48]]
    tmask = np.zeros((TY, TX), bool)
    for i in cand:
        x0, y0, x1, y1 = proj["rect"][i]
        tmask[y0:y1, x0:x1] = True
    tmask.reshape(-1)[rng.choice(TX * TY, 48, replace=False)] = True
    lists = oracle.build_lists(proj, cam, tile_mask=tmask)
    pmask = tmask[np.arange(H)[:, None] // 16, np.arange(W)[None, :] // 16]
    fwd = oracle.render_fwd(proj, lists, cam, prm, mask=pmask)
    M = W * H
    dC = np.where(fwd["image"] - targets[0] > 0, 1.0, -1.0) / (3 * M)
    dC[~pmask] = 0.0
    dH = np.where(pmask, scenes.GAMMA / M, 0.0)
    # every candidate's rect lies in the sampled tiles, so its gradient from
    # the sampled pixels is complete; check the candidates that are reached
    g9 = oracle.render_bwd(proj, lists, cam, prm, dC, dH, mask=pmask)
    view = {"proj": proj, "lists": lists, "fwd": fwd}
    bad = pixel_exclusion(view, cam) | ~pmask
    ok = ~bad.reshape(-1)
    # the reached candidates whose gradient no FP32 threshold flip can change
    badg = gaussian_exclusion(view, cam, pixel_exclusion(view, cam) & pmask)
    flip = flip_sensitive(view, cam, prm, dC, dH, g9_all=g9)
    pick = cand[(np.abs(g9[cand]).sum(1) > 0) & ~badg[cand]][:32]
    el = ~flip[pick]  # element-wise: the ones no near-threshold flip can move
    gm = np.zeros(N, np.uint8)
    gm[pick] = 1
    og = oracle.preprocess_bwd(scene, cam, prm, g9, gmask=gm)
    use = pick
    report = {"workload": "cfg5: 3M Gaussians, 1920x1080, SH0", "pixels_checked": int(ok.sum()),
              "gaussians_checked": int(len(use)), "gaussians_elementwise": int(el.sum())}
    for attr in ("f32", "f16", "bf16"):
        g = run_gpu(scene, cams, prm, attr=attr, dL_dimage=dC.astype(np.float32),
                    dL_dentropy=dH.astype(np.float32), keys=False)
        row = {}
        for k, o in (("image", fwd["image"].reshape(-1, 3)), ("final_T", fwd["final_T"].reshape(-1)),
                     ("entropy", fwd["entropy"].reshape(-1))):
            d = np.abs(g[k] - o).reshape(M, -1).max(1)[ok]
            row[k] = {"max_abs": float(d.max()), "mean_abs": float(d.mean())}
        row["last_entry_match"] = float(
            (last_ids_gpu(g, cams, 0, N)[ok] == last_ids_oracle(view, cam)[ok]).mean())
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            gg, oo = g["grads"][k][use], og[k][use]
            if k == "sh":
                gg, oo = gg[:, :1], oo[:, :1]
            assert np.linalg.norm(oo) > 0, k  # the sampled Gaussians are reached
            row["grad_" + k] = rel_norm_err(gg, oo)
            row["grad_elementwise_" + k] = elementwise_violations(gg[el], oo[el])[0]
        report[attr] = row
    out = os.environ.get("GS_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_cfg5.json"), "w") as f:
            json.dump(report, f, indent=1)
    print(json.dumps(report))
    f32 = report["f32"]
    # (in this dense scene few small Gaussians are reached before the pixels
    # stop: about 20 of the 48 front-most)
    assert report["pixels_checked"] > 10000 and report["gaussians_checked"] >= 12
    assert report["gaussians_elementwise"] >= 4
    assert f32["image"]["max_abs"] <= IMG_TOL and f32["final_T"]["max_abs"] <= IMG_TOL
    assert f32["entropy"]["max_abs"] <= IMG_TOL and f32["last_entry_match"] == 1.0
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert f32["grad_" + k] <= GRAD_TOL, (k, f32["grad_" + k])
        assert f32["grad_elementwise_" + k] == 0, k
    for attr in ("f16", "bf16"):
        assert report[attr]["image"]["mean_abs"] < 2e-2
        assert report[attr]["grad_means"] < 0.5
