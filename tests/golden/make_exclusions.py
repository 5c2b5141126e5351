"""Writes exclusions.json: the threshold-boundary cases of every workload,
counted and listed (readings c7 and c14), as the FP64 oracle finds them:
per view, the Gaussians whose tile rect an FP32 rounding of an edge or of the
radius could change (ids listed), the tiles such a rect may or may not reach,
the pixels with a threshold test (alpha_min, alpha_max, t_min) within 1e-4
(relative) of its limit, and the pixels the parity checks leave out (the
rule of oracle.exclusions: near a limit, or in a tile whose list may gain or
lose a flagged Gaussian that the pixel's walk meets with alpha >= alpha_min).
Calls only oracle/ (and the seeded scene generators); run from the repository
root:

    python tests/golden/make_exclusions.py

The pixel counts of the large views cover every pixel of the view; for cfg5
(3M Gaussians at 1920x1080, lists of several thousand entries) the pixel
counts are over a band of 8 tile rows through the middle of the view.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import exclusions  # noqa: E402
from paper_2603_09277_gb300 import scenes  # noqa: E402


def view_report(scene, cam, prm, band_rows=0):
    T = int(prm.get("tile", 16))
    W, H = cam["width"], cam["height"]
    TX, TY = (W + T - 1) // T, (H + T - 1) // T
    proj = oracle.preprocess(scene, cam, prm)
    rows = np.arange(H) // T
    if band_rows:
        t0 = TY // 2 - band_rows // 2
        band = (rows >= t0) & (rows < t0 + band_rows)
        tmask = np.zeros((TY, TX), bool)
        tmask[t0:t0 + band_rows] = True
    else:
        band = np.ones(H, bool)
        tmask = None
    lists = oracle.build_lists(proj, cam, tile_mask=tmask)
    mask = np.repeat(band[:, None], W, 1)
    fwd = oracle.render_fwd(proj, lists, cam, prm, mask=mask)
    view = {"proj": proj, "lists": lists, "fwd": fwd}
    s = exclusions.summary(view, cam, mask, prm=prm)
    # tiles that some but not every reachable rect of a flagged Gaussian covers
    amb = np.zeros((TY, TX), bool)
    for i in s["flagged_ids"]:
        hx0, hy0, hx1, hy1 = proj["rect_hi"][i]
        lx0, ly0, lx1, ly1 = proj["rect_lo"][i]
        m = np.zeros((TY, TX), bool)
        m[hy0:hy1, hx0:hx1] = True
        if lx1 > lx0 and ly1 > ly0:
            m[ly0:ly1, lx0:lx1] = False
        amb |= m
    out = {"size": [W, H], "tile": T, "visible_gaussians": int((proj["tiles"] > 0).sum()),
           "ambiguous_tiles": int(amb.sum())}
    out.update(s)
    return out


def report(name, scene, cams, prm, band_rows=0):
    return {"workload": name,
            "views": [view_report(scene, c, prm, band_rows) for c in cams]}


def cases():
    s, c, _, p = scenes.config1()
    yield "cfg1", s, c, p, 0
    p8 = dict(p, tile=8)
    yield "cfg1, 8x8 tiles", s, c, p8, 0
    for k in (-2, 4):
        s, c, _, p = scenes.config4(k=k)
        yield "cfg4 k=%d" % k, s, c, p, 0
    s, c, _, p = scenes.config2()
    yield "cfg2", s, c, p, 0
    s, c, _, p = scenes.config3()
    yield "cfg3 (views 0, 3, 6: one of each size)", s, [c[0], c[3], c[6]], p, 0
    s, c, _, p = scenes.config5()
    yield "cfg5 (8 tile rows)", s, c, p, 8


def main():
    out = [report(*args) for args in cases()]
    path = os.path.join(HERE, "exclusions.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    for r in out:
        for v in r["views"]:
            print(r["workload"], v["size"], "flagged", v["flagged_gaussians"], "ambiguous tiles",
                  v["ambiguous_tiles"], "near-threshold px", v["near_threshold_pixels"],
                  "excluded px", v["excluded_pixels"], "of", v["pixels_counted"])


if __name__ == "__main__":
    main()
