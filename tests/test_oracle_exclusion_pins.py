"""Pins of the oracle's threshold-boundary outputs, which decide what every
parity test leaves out: the per-Gaussian rect flag and the bounds of the
rects an FP32 rounding can reach (readings c7, c14), and the per-pixel
threshold margin and first near-threshold list position (Sec. 3 thresholds,
reading c2).  Each is checked against a computation of its own: the
reachable rects by brute force over every combination of edge and radius
roundings from the 2D covariance recovered by inverting the oracle's conic;
the margins by a vectorised walk of each pixel's list; and targeted cases
placed at a known distance from a limit.

The bands are the oracle's stated readings: a rect edge within 2e-3 px of a
tile boundary or a 3-sigma radius within 2e-5 (relative) of an integer may
round either way in FP32; a threshold test within 1e-3 (relative) of its
limit marks the first near-threshold list position."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2603_09277_gb300 import scenes

EPS_PX = 2e-3     # pixel band of a rect edge (reading c7)
EPS_R = 2e-5      # relative band of the 3-sigma radius (reading c7)
NEAR_BAND = 1e-3  # relative band of the first near-threshold position


def _rect(l, r, t, b, TX, TY, tile):
    x0 = np.clip(np.floor(l / tile), 0, TX)
    x1 = np.clip(np.floor(r / tile) + 1, 0, TX)
    y0 = np.clip(np.floor(t / tile), 0, TY)
    y1 = np.clip(np.floor(b / tile) + 1, 0, TY)
    return np.stack([x0, y0, x1, y1], 1).astype(np.int64)


def _reachable(P9, W, H, tile):
    """Base rect, flag, intersection and union of every rect reachable by
    rounding each edge by -EPS_PX, 0 or +EPS_PX independently and the radius
    from 3 sqrt(lambda_max) (1 - EPS_R), (1), (1 + EPS_R), where lambda_max is
    the larger eigenvalue of the 2D covariance, the inverse of the conic."""
    a, b, c = P9[:, 2], P9[:, 3], P9[:, 4]
    det_c = a * c - b * b
    # covariance = conic^-1; its larger eigenvalue
    A, B, C = c / det_c, -b / det_c, a / det_c
    lam = np.linalg.eigvalsh(np.stack([np.stack([A, B], 1), np.stack([B, C], 1)], 1))[:, 1]
    rf = 3.0 * np.sqrt(lam)
    mx, my = P9[:, 0], P9[:, 1]
    TX, TY = (W + tile - 1) // tile, (H + tile - 1) // tile
    r0 = np.ceil(rf)
    base = _rect(mx - r0, mx + r0, my - r0, my + r0, TX, TY, tile)
    lo = base.copy()
    hi = base.copy()
    flag = np.zeros(len(P9), bool)
    for rr in (np.ceil(rf * (1 - EPS_R)), r0, np.ceil(rf * (1 + EPS_R))):
        for s in itertools.product((-EPS_PX, 0.0, EPS_PX), repeat=4):
            q = _rect(mx - rr + s[0], mx + rr + s[1], my - rr + s[2], my + rr + s[3], TX, TY, tile)
            flag |= (q != base).any(1)
            lo[:, :2] = np.maximum(lo[:, :2], q[:, :2])
            lo[:, 2:] = np.minimum(lo[:, 2:], q[:, 2:])
            hi[:, :2] = np.minimum(hi[:, :2], q[:, :2])
            hi[:, 2:] = np.maximum(hi[:, 2:], q[:, 2:])
    return r0.astype(np.int64), base, flag, lo, hi


def _near_edge_scene(n, seed, W, H, f, tile):
    """Isotropic Gaussians on an identity camera, each placed so that one
    rect edge lies at a chosen offset from a tile boundary: within the band
    for half of them (offsets in (-EPS_PX, EPS_PX) / 2), outside it for the
    other half (offsets of 3 EPS_PX .. 0.3 px)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(2.0, 4.0, n)
    s0 = rng.uniform(0.004, 0.02, n)
    k = rng.integers(4, (W // tile) - 4, n)
    near = np.arange(n) % 2 == 0
    off = np.where(near, rng.uniform(-0.5, 0.5, n) * EPS_PX,
                   rng.choice([-1, 1], n) * rng.uniform(3 * EPS_PX, 0.3, n))
    my = rng.uniform(tile * 4, H - tile * 4, n)
    y = (my - H / 2) * z / f
    x = np.zeros(n)
    # an isotropic Gaussian at camera-space (x, y, z) has the 2D covariance
    # (f s0 / z)^2 (I + u u^T) + 0.3 I with u = (x, y) / z (dilation 0.3), so
    # lambda_max = (f s0 / z)^2 (1 + |u|^2) + 0.3; the left edge mx - r is put
    # at the tile boundary k tile plus the offset (r depends on x: iterate)
    for _ in range(6):
        lam = (f * s0 / z) ** 2 * (1 + (x / z) ** 2 + (y / z) ** 2) + 0.3
        r = np.ceil(3.0 * np.sqrt(lam))
        mx = k * tile + r + off
        x = (mx - W / 2) * z / f
    scene = {"means": np.stack([x, y, z], 1).astype(np.float32),
             "log_scales": np.repeat(np.log(s0)[:, None], 3, 1).astype(np.float32),
             "quats": np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
             "opacity_logits": rng.normal(0, 1, n).astype(np.float32),
             "sh": np.zeros((n, 16, 3), np.float32), "sh_degree": 0}
    return scene, near


@pytest.mark.parametrize("tile", [16, 8])
def test_boundary_flags_and_reachable_rects_by_brute_force(tile):
    W, H, f = 320, 240, 320.0
    scene, cams, _, prm = scenes.config1(n=40000, seed=3)
    cams = [scenes.camera(W, H, f)]
    prm = dict(prm, tile=tile)
    pr = oracle.preprocess(scene, cams[0], prm)
    vis = pr["tiles"] > 0
    r0, base, flag, lo, hi = _reachable(pr["P9"], W, H, tile)
    assert (r0[vis] == pr["radius"][vis]).all()
    assert (base[vis] == pr["rect"][vis]).all()
    ob = pr["boundary"].astype(bool)
    assert (flag[vis] == ob[vis]).all()
    assert ob[vis].sum() >= 10  # the scene exercises the flag
    fl = vis & ob
    assert (lo[fl] == pr["rect_lo"][fl]).all() and (hi[fl] == pr["rect_hi"][fl]).all()
    # the union holds the rect, the rect holds the intersection
    assert (pr["rect_hi"][fl][:, :2] <= pr["rect"][fl][:, :2]).all()
    assert (pr["rect_hi"][fl][:, 2:] >= pr["rect"][fl][:, 2:]).all()
    assert (pr["rect_lo"][fl][:, :2] >= pr["rect"][fl][:, :2]).all()
    assert (pr["rect_lo"][fl][:, 2:] <= pr["rect"][fl][:, 2:]).all()


def test_boundary_flag_on_edges_placed_near_a_tile_boundary():
    """Left edges placed within half the band of a tile boundary are flagged
    and their union reaches one tile further left; edges 3 bands or more
    away are not flagged (unless their radius or another edge is near)."""
    W, H, f, tile = 640, 480, 640.0, 16
    scene, near = _near_edge_scene(400, 11, W, H, f, tile)
    cam = scenes.camera(W, H, f)
    prm = scenes.params(sh_degree=0, tile=tile)
    pr = oracle.preprocess(scene, cam, prm)
    assert (pr["tiles"] > 0).all()
    ob = pr["boundary"].astype(bool)
    assert ob[near].all()
    # the union's left column is one tile left of the intersection's
    assert (pr["rect_hi"][near, 0] == pr["rect_lo"][near, 0] - 1).all()
    _, _, flag, _, _ = _reachable(pr["P9"], W, H, tile)
    assert (flag == ob).all()
    assert (~ob[~near]).mean() > 0.9


def _walk_brute(P9, ids, px, py, amin, amax, tmin):
    """Margin, first near-threshold position, evaluated entries and the
    last blended position of one pixel from vectorised arrays: every alpha of
    the list at once, the running T as a product over the entries that pass
    the skip test, the stop at the first entry whose T (1 - alpha) < tmin."""
    g = P9[ids]
    dx, dy = px - g[:, 0], py - g[:, 1]
    araw = g[:, 5] * np.exp(-0.5 * (g[:, 2] * dx * dx + 2 * g[:, 3] * dx * dy + g[:, 4] * dy * dy))
    ah = np.minimum(amax, araw)
    keep = ah >= amin
    om = np.where(keep, 1.0 - ah, 1.0)
    T_before = np.concatenate([[1.0], np.cumprod(om)[:-1]])
    testT = T_before * (1.0 - ah)
    stop = np.nonzero(keep & (testT < tmin))[0]
    n_eval = (stop[0] + 1) if len(stop) else len(ids)
    ev = np.arange(len(ids)) < n_eval
    m_alpha = np.minimum(np.abs(araw - amin) / amin, np.abs(araw - amax) / amax)
    m_T = np.where(keep, np.abs(testT - tmin) / tmin, np.inf)
    margin = min(m_alpha[ev].min(initial=np.inf), m_T[ev].min(initial=np.inf))
    near = ev & ((m_alpha < NEAR_BAND) | (m_T < NEAR_BAND))
    first_near = int(np.nonzero(near)[0][0]) if near.any() else -1
    blended = np.nonzero(keep & ev & ~((testT < tmin) & keep))[0]
    last = int(blended[-1] + 1) if len(blended) else 0
    return margin, first_near, int(n_eval), last


@pytest.mark.parametrize("seed", [0, 1])
def test_margin_and_first_near_by_vectorised_walk(seed):
    scene, cams, _, prm = scenes.tiny_scene(40, seed=seed, width=48, height=32)
    cam = cams[0]
    pr = oracle.preprocess(scene, cam, prm)
    ts, ids = oracle.build_lists(pr, cam)
    fwd = oracle.render_fwd(pr, (ts, ids), cam, prm)
    amin, amax, tmin = (float(np.float32(prm[k])) for k in ("alpha_min", "alpha_max", "t_min"))
    TX = (cam["width"] + 15) // 16
    nonempty = 0
    for y in range(cam["height"]):
        for x in range(cam["width"]):
            t = (y // 16) * TX + x // 16
            lst = ids[ts[t]:ts[t + 1]]
            if len(lst) == 0:
                assert fwd["first_near"][y, x] == -1 and math.isinf(fwd["margin"][y, x])
                continue
            nonempty += 1
            m, fn, ne, last = _walk_brute(pr["P9"], lst, x + 0.5, y + 0.5, amin, amax, tmin)
            assert fwd["margin"][y, x] == pytest.approx(m, rel=1e-9, abs=1e-300)
            assert fwd["first_near"][y, x] == fn
            assert fwd["neval"][y, x] == ne
            assert fwd["last"][y, x] == last
    assert nonempty > 1000


@pytest.mark.parametrize("delta", [3e-4, -3e-4, 2e-3])
def test_margin_of_an_alpha_placed_near_alpha_min(delta):
    """One isotropic Gaussian on the axis (dilation 0): its alpha at the pixel
    centre (u + 0.5, v + 0.5) at distance rho from the mean is
    sigma exp(-rho^2 z^2 / (2 f^2 s0^2)); choosing the opacity so that this is
    alpha_min (1 + delta) gives a margin of |delta| there (the other pixels
    are farther from every limit or evaluate this same entry), and a first
    near-threshold position of 0 exactly when |delta| < 1e-3."""
    W = H = 32
    f, z, s0 = 32.0, 3.0, 0.25
    cam = scenes.camera(W, H, f)
    prm = scenes.params(sh_degree=0, dilation=0.0)
    amin = float(np.float32(prm["alpha_min"]))
    px, py = 20.5, 16.5  # pixel (20, 16); the mean projects to (16, 16)
    rho2 = (px - 16.0) ** 2 + (py - 16.0) ** 2
    sig = amin * (1 + delta) / math.exp(-rho2 * z * z / (2 * f * f * s0 * s0))
    scene = {"means": np.array([[0.0, 0.0, z]], np.float32),
             "log_scales": np.full((1, 3), math.log(s0), np.float32),
             "quats": np.array([[1, 0, 0, 0]], np.float32),
             "opacity_logits": np.array([math.log(sig / (1 - sig))], np.float32),
             "sh": np.zeros((1, 16, 3), np.float32), "sh_degree": 0}
    pr = oracle.preprocess(scene, cam, prm)
    # alpha from the stored (FP32) inputs, which move it by a few 1e-8
    sig_st = pr["P9"][0, 5]
    s_st = math.exp(float(scene["log_scales"][0, 0]))
    a_pix = sig_st * math.exp(-rho2 * z * z / (2 * f * f * s_st * s_st))
    fwd = oracle.render_fwd(pr, oracle.build_lists(pr, cam), cam, prm)
    m = fwd["margin"][16, 20]
    assert m == pytest.approx(abs(a_pix - amin) / amin, rel=1e-6)
    assert m == pytest.approx(abs(delta), rel=1e-3)
    assert fwd["first_near"][16, 20] == (0 if abs(delta) < NEAR_BAND else -1)
    # skipped below alpha_min, blended above
    assert fwd["last"][16, 20] == (1 if delta > 0 else 0)


def _composite(P9, ids, px, py, amin, amax, tmin):
    """Colour and final T of one pixel over a list (vectorised walk)."""
    if len(ids) == 0:
        return np.zeros(3), 1.0
    g = P9[ids]
    dx, dy = px - g[:, 0], py - g[:, 1]
    araw = g[:, 5] * np.exp(-0.5 * (g[:, 2] * dx * dx + 2 * g[:, 3] * dx * dy + g[:, 4] * dy * dy))
    ah = np.minimum(amax, araw)
    keep = ah >= amin
    om = np.where(keep, 1.0 - ah, 1.0)
    T_before = np.concatenate([[1.0], np.cumprod(om)[:-1]])
    stop = np.nonzero(keep & (T_before * (1.0 - ah) < tmin))[0]
    n = stop[0] if len(stop) else len(ids)
    w = np.where(keep, ah, 0.0)[:n] * T_before[:n]
    return (w[:, None] * g[:n, 6:9]).sum(0), (T_before[n] if n < len(ids) else
                                               T_before[-1] * om[-1])


@pytest.mark.parametrize("cfg", ["cfg1", "cfg4k-2", "near_edge"])
def test_pixel_exclusion_covers_every_pixel_a_flagged_gaussian_can_change(cfg):
    """Soundness of the exclusion rule: for every flagged Gaussian and every
    pixel of a tile that some but not every reachable rect covers, the pixel
    is composited with the Gaussian inserted in (or removed from) its tile's
    list at its place in the depth order; wherever that changes the colour or
    the final T, the rule excludes the pixel.  And the rule stays narrow."""
    from oracle import exclusions
    if cfg == "cfg1":
        scene, cams, _, prm = scenes.config1()
    elif cfg == "cfg4k-2":
        scene, cams, _, prm = scenes.config4(k=-2)
    else:
        # edges placed at tile boundaries (half of them within the band),
        # nearly opaque, so that the ambiguous tiles' nearest pixels pass
        # alpha_min; colours from the scene's seeded draw
        scene, _ = _near_edge_scene(160, 5, 320, 240, 320.0, 16)
        scene["opacity_logits"][:] = 3.0
        scene["sh"][:, 0, :] = np.random.default_rng(5).uniform(-1.5, 1.5, (160, 3))
        cams = [scenes.camera(320, 240, 320.0)]
        prm = scenes.params(sh_degree=0)
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    pr = oracle.preprocess(scene, cam, prm)
    ts, ids = oracle.build_lists(pr, cam)
    fwd = oracle.render_fwd(pr, (ts, ids), cam, prm)
    view = {"proj": pr, "lists": (ts, ids), "fwd": fwd}
    bad = exclusions.pixel_exclusion(view, cam, prm=prm)
    amin, amax, tmin = (float(np.float32(prm[k])) for k in ("alpha_min", "alpha_max", "t_min"))
    key = pr["depth"].view(np.uint32).astype(np.int64) * (1 << 32) + np.arange(len(pr["depth"]))
    TX = (W + 15) // 16
    flagged = np.nonzero(pr["boundary"])[0]
    assert len(flagged) >= 5
    changed = 0
    for i in flagged:
        hx0, hy0, hx1, hy1 = pr["rect_hi"][i]
        lx0, ly0, lx1, ly1 = pr["rect_lo"][i]
        for ty in range(hy0, hy1):
            for tx in range(hx0, hx1):
                if lx0 <= tx < lx1 and ly0 <= ty < ly1:
                    continue  # in every reachable rect: listed either way
                lst = ids[ts[ty * TX + tx]:ts[ty * TX + tx + 1]]
                without = lst[lst != i]
                pos = np.searchsorted(key[without], key[i])
                with_i = np.insert(without, pos, i)
                for y in range(ty * 16, min(H, ty * 16 + 16)):
                    for x in range(tx * 16, min(W, tx * 16 + 16)):
                        c0, t0 = _composite(pr["P9"], without, x + 0.5, y + 0.5, amin, amax, tmin)
                        c1, t1 = _composite(pr["P9"], with_i, x + 0.5, y + 0.5, amin, amax, tmin)
                        if np.abs(c0 - c1).max() > 1e-12 or abs(t0 - t1) > 1e-12:
                            changed += 1
                            assert bad[y, x], (i, x, y)
    if cfg == "near_edge":
        assert changed > 0  # the scene holds pixels the rule must catch
    assert bad.mean() < 0.05


def test_stored_exclusion_report_matches_the_oracle():
    """tests/golden/exclusions.json (written by make_exclusions.py from the
    oracle alone) still describes the oracle: the small workloads' entries
    are recomputed and must agree exactly; the large ones must be present
    with few excluded pixels."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_exclusions as mk
    stored = {r["workload"]: r for r in json.load(open(os.path.join(here, "exclusions.json")))}
    s, c, _, p = scenes.config1()
    assert mk.report("cfg1", s, c, p) == stored["cfg1"]
    s, c, _, p = scenes.config4(k=4)
    assert mk.report("cfg4 k=4", s, c, p) == stored["cfg4 k=4"]
    for name, r in stored.items():
        for v in r["views"]:
            assert v["excluded_pixels"] <= 0.01 * v["pixels_counted"], (name, v["size"])
            assert len(v["flagged_ids"]) == v["flagged_gaussians"]
