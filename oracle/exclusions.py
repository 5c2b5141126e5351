"""Threshold-boundary exclusions of the parity checks, derived from the FP64
oracle's outputs alone (readings c7 and c14 of the paper's thresholds).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

An FP32 implementation of the method may decide a threshold differently
from the FP64 definition where the decision lies within its rounding:

- a Gaussian whose tile rect a rounding of an edge or of the 3-sigma radius
  changes (the oracle's ``boundary`` flag) may be in or out of the lists of
  the tiles between its intersection and union rects (``rect_lo`` /
  ``rect_hi``).  A pixel of such a tile can only change if the walk of its
  list would meet that Gaussian, i.e. the pixel does not stop before the
  Gaussian's place in the depth order (key: FP32 depth bits, then id), and
  only if the Gaussian's alpha reaches alpha_min there;
- a pixel whose smallest relative distance of any threshold test (alpha_min,
  alpha_max, t_min) is below ``margin`` may take the other branch.

``pixel_exclusion`` marks the pixels of one view left out of the pixel
checks; ``gaussian_exclusion`` the Gaussians whose gradient such a pixel can
change by more than the tolerance.
"""
from __future__ import annotations

import numpy as np

import oracle as _oracle

MARGIN = 1e-4


def _alpha_min32(prm):
    return float(np.float32((prm or {}).get("alpha_min", 1.0 / 255)))


def stop_keys(ora_view, cam):
    """Per pixel (H, W): the depth key (FP32 depth bits, id) of the entry
    whose test stopped the walk, as two arrays; pixels that walked their
    whole list get (2^32, 0) (every Gaussian comes before that)."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    ts, ids = ora_view["lists"]
    T = proj.get("tile", 16)
    W, H = cam["width"], cam["height"]
    TX = (W + T - 1) // T
    yy, xx = np.divmod(np.arange(W * H), W)
    tile = (yy // T) * TX + xx // T
    start, end = ts[tile], ts[tile + 1]
    ne = fwd["neval"].reshape(-1).astype(np.int64)
    stopped = start + ne < end + 0  # a stop leaves entries after it
    stopped &= ne > 0
    # with a stop, the stopping entry is the last evaluated one
    pos = np.where(stopped, start + ne - 1, 0)
    sid = np.where(stopped, ids[np.minimum(pos, max(len(ids) - 1, 0))] if len(ids) else 0, 0)
    dbits = proj["depth"].view(np.uint32).astype(np.int64)
    skey = np.where(stopped, dbits[sid], np.int64(1) << 32)
    sidk = np.where(stopped, sid, 0)
    return skey.reshape(H, W), sidk.reshape(H, W)


def pixel_exclusion(ora_view, cam, margin=MARGIN, prm=None):
    """Boolean [H, W]: pixels of one view left out of the pixel checks."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    W, H = cam["width"], cam["height"]
    T = proj.get("tile", 16)
    TX, TY = (W + T - 1) // T, (H + T - 1) // T
    bad = fwd["margin"] < margin
    amin = _alpha_min32(prm)
    flagged = np.nonzero(proj["boundary"])[0]
    if len(flagged) == 0:
        return bad
    skey, sid = stop_keys(ora_view, cam)
    dbits = proj["depth"].view(np.uint32).astype(np.int64)
    for i in flagged:
        hx0, hy0, hx1, hy1 = proj["rect_hi"][i]
        lx0, ly0, lx1, ly1 = proj["rect_lo"][i]
        if hx1 <= hx0 or hy1 <= hy0:
            continue
        m = np.zeros((TY, TX), bool)
        m[hy0:hy1, hx0:hx1] = True
        if lx1 > lx0 and ly1 > ly0:
            m[ly0:ly1, lx0:lx1] = False
        g = proj["P9"][i]
        ki = dbits[i]
        for ty, tx in zip(*np.nonzero(m)):
            ys = slice(ty * T, min(H, ty * T + T))
            xs = slice(tx * T, min(W, tx * T + T))
            u = np.arange(xs.start, xs.stop) + 0.5 - g[0]
            v = np.arange(ys.start, ys.stop) + 0.5 - g[1]
            du, dv = np.meshgrid(u, v)
            a = g[5] * np.exp(-0.5 * (g[2] * du * du + 2 * g[3] * du * dv + g[4] * dv * dv))
            # the walk meets Gaussian i unless it stops at an entry before it
            meets = (ki < skey[ys, xs]) | ((ki == skey[ys, xs]) & (i <= sid[ys, xs]))
            bad[ys, xs] |= meets & (a >= amin * (1 - margin))
    return bad


def gaussian_exclusion(ora_view, cam, bad_pixels, margin=MARGIN):
    """Boolean [N]: Gaussians whose gradient an FP32 threshold decision may
    change by more than the tolerance: the boundary-flagged ones; at a pixel
    with a near-threshold test, the entry at the first near-threshold list
    position and the next two (a flipped skip or clamp changes that entry's
    own contribution entirely; later entries only through T, by a factor
    within alpha_min of 1, and a flipped stop adds entries of weight below
    t_min); at any other excluded pixel (a tile whose list may gain or lose
    a flagged Gaussian the walk meets), the whole list."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    ts, ids = ora_view["lists"]
    T = proj.get("tile", 16)
    TX = (cam["width"] + T - 1) // T
    bad = proj["boundary"].astype(bool).copy()
    margin_bad = fwd["margin"] < margin
    ys, xs = np.nonzero(bad_pixels)
    for y, x in zip(ys, xs):
        t = (y // T) * TX + x // T
        fn = int(fwd["first_near"][y, x])
        if margin_bad[y, x] and fn >= 0:
            bad[ids[ts[t] + fn:min(ts[t + 1], ts[t] + fn + 3)]] = True
        else:
            bad[ids[ts[t]:ts[t + 1]]] = True
    return bad


def summary(ora_view, cam, mask=None, margin=MARGIN, prm=None):
    """Counts (and ids) of one view's threshold-boundary cases over the
    pixels of `mask` (all pixels if None)."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    W, H = cam["width"], cam["height"]
    mask = np.ones((H, W), bool) if mask is None else mask
    flagged = np.nonzero(proj["boundary"])[0]
    excl = pixel_exclusion(ora_view, cam, margin, prm) & mask
    near = (fwd["margin"] < margin) & mask
    return {"flagged_gaussians": int(len(flagged)), "flagged_ids": [int(i) for i in flagged],
            "near_threshold_pixels": int(near.sum()),
            "excluded_pixels": int(excl.sum()), "pixels_counted": int(mask.sum()),
            "compared_pixels": int((mask & ~excl).sum())}


def flip_sensitive(ora_view, cam, prm, dL_dC, dL_dH, g9_all=None, share=0.02, margin=MARGIN):
    """Boolean [N]: Gaussians whose gradient a threshold flip at a
    near-threshold pixel (smallest relative margin below `margin`) can move
    by a noticeable part.  A flip there changes the pixel's contributions to
    every later entry by a factor within alpha_min of 1 (about 0.4 %), so a
    Gaussian that takes `share` or more of any of its nine 2D-gradient
    components (mean, conic, opacity, colour) from such pixels is marked.
    dL_dC [H,W,3], dL_dH [H,W]: the loss gradients of the view; g9_all: the
    oracle's 2D gradients of the whole view (recomputed if None)."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    N = proj["P9"].shape[0]
    mb = fwd["margin"] < margin
    if not mb.any():
        return np.zeros(N, bool)
    dC = np.array(dL_dC, np.float64, copy=True)
    dC[~mb] = 0.0
    dH = None
    if dL_dH is not None:
        dH = np.array(dL_dH, np.float64, copy=True)
        dH[~mb] = 0.0
    g9b = _oracle.render_bwd(proj, ora_view["lists"], cam, prm, dC, dH, mask=mb)
    if g9_all is None:
        g9_all = _oracle.render_bwd(proj, ora_view["lists"], cam, prm, dL_dC, dL_dH)
    ratio = np.abs(g9b) / np.maximum(np.abs(g9_all), 1e-300)
    return (ratio >= share).any(1) & (np.abs(g9b).sum(1) > 0)
