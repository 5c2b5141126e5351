"""Shared helpers of the GPU parity tests: run the libgs path through the
C ABI, run the oracle, and derive the threshold-boundary exclusions.

Exclusion rules (from the oracle only, never from the GPU results):
- a Gaussian whose rect could round differently in FP32 (oracle boundary
  flag) is left out of the bit-exact rect/list checks, and the tiles that
  lie in some but not every rect reachable under the rounding bands are
  left out of the pixel checks (their lists may hold one entry more or less);
- a pixel whose smallest relative distance of any threshold test
  (alpha_min, alpha_max, t_min) is below MARGIN may take the other branch in
  FP32 and is left out of the pixel checks;
- gradients are compared per tensor on the relative norm, and element-wise
  on the Gaussians that no excluded pixel evaluates.
"""
import numpy as np
import torch

import oracle
from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device, targets_to_device

MARGIN = 1e-4       # relative threshold margin below which a pixel is excluded
IMG_TOL = 1e-5      # absolute, images / T / entropy (FP32 vs FP64)
GRAD_TOL = 1e-4     # relative, gradient tensors (norm), FP32 vs FP64


def run_gpu(scene, cams, prm, target=None, gamma=0.015, attr="f32", persistent=0,
            dL_dimage=None, dL_dentropy=None, keys=True, ppt=0, batch=0):
    """Runs preprocess, bin_sort, render_fwd, loss (if target) and
    render_bwd through the C ABI.  dL_dimage / dL_dentropy (numpy, per
    pixel) override the loss gradients.  Returns numpy arrays."""
    N = scene["means"].shape[0]
    rast = Rasterizer(cams, prm, N, attr_dtype=attr, keep_debug=True, persistent=persistent,
                      pixels_per_thread=ppt, batch=batch)
    p = scene_to_device(scene)
    rast.preprocess(p)
    P = rast.bin_sort(keys=keys)
    rast.render_fwd(stats=True)
    out = {"P": P}
    if target is not None:
        tgt = targets_to_device(target)
        rast.loss(tgt, gamma)
        out["loss"] = float(rast.loss_dev.item())
    if dL_dimage is not None:
        dimg = torch.as_tensor(np.ascontiguousarray(dL_dimage, np.float32).reshape(-1, 3)).cuda()
        dent = (None if dL_dentropy is None else
                torch.as_tensor(np.ascontiguousarray(dL_dentropy, np.float32).reshape(-1)).cuda())
        rast.render_bwd(p, dimg, dent)
    elif target is not None:
        rast.render_bwd(p)
    torch.cuda.synchronize()
    n = lambda t: t.detach().cpu().numpy()
    out.update({
        "rast": rast,
        "depth": n(rast.depth), "rect": n(rast.rect), "tiles": n(rast.tiles_touched),
        "radius": n(rast.radius), "mean2d": n(rast.mean2d), "conic_opacity": n(rast.conic_opacity),
        "rgb": n(rast.rgb), "ranges": n(rast.tile_ranges).astype(np.int64),
        "vals": n(rast.sorted_vals)[:P].astype(np.int64) if P else np.zeros(0, np.int64),
        "keys": (n(rast.sorted_keys)[:P].view(np.uint64) if (keys and P) else None),
        "image": n(rast.image), "final_T": n(rast.final_T),
        "last": n(rast.last_idx).astype(np.int64), "entropy": n(rast.entropy),
        "stats": n(rast.stats),
        "grad2d": n(rast.grad2d),
        "grads": {k: n(v) for k, v in rast.grads.items()},
    })
    return out


def view_pixels(cams):
    out, off = [], 0
    for c in cams:
        n = c["width"] * c["height"]
        out.append((off, off + n))
        off += n
    return out


def view_tiles(cams, tile=16):
    out, off = [], 0
    for c in cams:
        tx, ty = oracle.tile_grid(c, {"tile": tile})
        out.append((off, off + tx * ty))
        off += tx * ty
    return out


def pixel_exclusion(ora_view, cam, margin=MARGIN):
    """Boolean [H,W]: pixels left out of the pixel checks of one view."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    W, H = cam["width"], cam["height"]
    T = proj.get("tile", 16)
    TX, TY = oracle.tile_grid(cam, {"tile": T})
    bad_tiles = np.zeros((TY, TX), bool)
    amin = float(np.float32(1.0 / 255))
    for i in np.nonzero(proj["boundary"])[0]:
        # tiles that are in some reachable rect but not in every one ...
        hx0, hy0, hx1, hy1 = proj["rect_hi"][i]
        lx0, ly0, lx1, ly1 = proj["rect_lo"][i]
        m = np.zeros((TY, TX), bool)
        m[hy0:hy1, hx0:hx1] = True
        if lx1 > lx0 and ly1 > ly0:
            m[ly0:ly1, lx0:lx1] = False
        # ... and where the Gaussian's alpha reaches alpha_min at some pixel
        # (elsewhere it is skipped whether or not it is listed)
        g = proj["P9"][i]
        for ty, tx in zip(*np.nonzero(m)):
            u = np.arange(tx * T, min(W, tx * T + T)) + 0.5 - g[0]
            v = np.arange(ty * T, min(H, ty * T + T)) + 0.5 - g[1]
            du, dv = np.meshgrid(u, v)
            a = g[5] * np.exp(-0.5 * (g[2] * du * du + 2 * g[3] * du * dv + g[4] * dv * dv))
            if a.max() >= amin * (1 - margin):
                bad_tiles[ty, tx] = True
    px_tiles = bad_tiles[np.arange(H)[:, None] // T, np.arange(W)[None, :] // T]
    return px_tiles | (fwd["margin"] < margin)


def last_ids_gpu(g, cams, v, N, tile_px=16):
    """Row id of each pixel's last blended entry (-1 if none), GPU side."""
    a, b = view_pixels(cams)[v]
    t0 = view_tiles(cams, tile_px)[v][0]
    cam = cams[v]
    W, H = cam["width"], cam["height"]
    T = tile_px
    TX = (W + T - 1) // T
    yy, xx = np.divmod(np.arange(W * H), W)
    tile = t0 + (yy // T) * TX + xx // T
    last = g["last"][a:b]
    start = g["ranges"][tile, 0]
    out = np.full(W * H, -1, np.int64)
    has = last > 0
    out[has] = g["vals"][start[has] + last[has] - 1] - v * N
    return out


def last_ids_oracle(view, cam):
    """Gaussian id of each pixel's last blended entry (-1 if none), oracle side."""
    ts, ids = view["lists"]
    W, H = cam["width"], cam["height"]
    T = view["proj"].get("tile", 16)
    TX = (W + T - 1) // T
    yy, xx = np.divmod(np.arange(W * H), W)
    tile = (yy // T) * TX + xx // T
    last = view["fwd"]["last"].reshape(-1)
    out = np.full(W * H, -1, np.int64)
    has = last > 0
    out[has] = ids[ts[tile[has]] + last[has] - 1]
    return out


def gaussian_exclusion(ora_view, cam, bad_pixels):
    """Boolean [N]: Gaussians whose gradient an FP32 threshold decision may
    change by more than the tolerance: the boundary-flagged ones; at a pixel
    with a near-threshold test, the entry at the first near-threshold list
    position and the next two (a flipped skip or clamp changes that entry's
    own contribution entirely; later entries only through T, by a factor
    within alpha_min of 1, and a flipped stop adds entries of weight below
    t_min); at a pixel of a tile whose list may gain or lose a flagged
    Gaussian of visible alpha, the whole list."""
    proj, fwd = ora_view["proj"], ora_view["fwd"]
    ts, ids = ora_view["lists"]
    T = proj.get("tile", 16)
    TX, TY = oracle.tile_grid(cam, {"tile": T})
    bad = proj["boundary"].astype(bool).copy()
    margin_bad = fwd["margin"] < MARGIN
    ys, xs = np.nonzero(bad_pixels)
    for y, x in zip(ys, xs):
        t = (y // T) * TX + x // T
        fn = int(fwd["first_near"][y, x])
        if margin_bad[y, x] and fn >= 0:
            bad[ids[ts[t] + fn:min(ts[t + 1], ts[t] + fn + 3)]] = True
        else:
            bad[ids[ts[t]:ts[t + 1]]] = True
    return bad


def rel_norm_err(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
