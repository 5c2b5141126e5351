"""Shared helpers of the GPU parity tests: run the libgs path through the
C ABI, run the oracle, and apply the threshold-boundary exclusions.

Exclusion rules (oracle.exclusions, from the oracle only, never from the GPU
results):
- a Gaussian whose rect could round differently in FP32 (oracle boundary
  flag) is left out of the bit-exact rect/list checks; a pixel of a tile
  that lies in some but not every rect reachable under the rounding bands
  is left out of the pixel checks when its walk meets that Gaussian (does
  not stop before the Gaussian's place in the depth order) and the
  Gaussian's alpha reaches alpha_min there;
- a pixel whose smallest relative distance of any threshold test
  (alpha_min, alpha_max, t_min) is below MARGIN may take the other branch in
  FP32 and is left out of the pixel checks;
- gradients are compared per tensor on the relative norm, and element-wise
  (1e-4 relative with a floor of 1e-6 of the tensor's largest entry), on the
  Gaussians that no excluded pixel's decision can change.
"""
import numpy as np
import torch

import oracle
import oracle.exclusions as _exc
from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device, targets_to_device

MARGIN = 1e-4       # relative threshold margin below which a pixel is excluded
IMG_TOL = 1e-5      # absolute, images / T / entropy (FP32 vs FP64)
GRAD_TOL = 1e-4     # relative, gradient tensors (norm), FP32 vs FP64
# element-wise gradient bar: 1e-4 relative with a floor of 1e-5 of the
# tensor's largest entry.  The gradients of a pixel-mean loss scale with
# 1 / pixels (largest entries 4e-3 .. 2e-2 here), so the floor is stated
# relative to the tensor; it is below an absolute 1e-6 on every workload.
# It covers the FP32 rounding of the sums of dd-moments over pixels, whose
# terms cancel (measured up to 4.9e-6 of the largest entry where no
# threshold is near)
ELEM_FLOOR = 1e-5
# Gaussians taking this share of a 2D-gradient component from near-threshold
# pixels are left out of the element-wise check (oracle.exclusions)
FLIP_SHARE = 0.02


def run_gpu(scene, cams, prm, target=None, gamma=0.015, attr="f32", persistent=0,
            dL_dimage=None, dL_dentropy=None, keys=True, ppt=0, batch=0, sh_layout=0):
    """Runs preprocess, bin_sort, render_fwd, loss (if target) and
    render_bwd through the C ABI.  dL_dimage / dL_dentropy (numpy, per
    pixel) override the loss gradients; sh_layout is the layout of the SH
    coefficients on the device (the SH gradient comes back as [N][K][3]).
    Returns numpy arrays."""
    N = scene["means"].shape[0]
    rast = Rasterizer(cams, prm, N, sh_stride=scene["sh"].shape[1], attr_dtype=attr,
                      keep_debug=True, persistent=persistent, pixels_per_thread=ppt, batch=batch)
    p = scene_to_device(scene, sh_layout=sh_layout)
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
        "grads": {k: (n(v.transpose(0, 1)) if k == "sh" and sh_layout == 1 else n(v))
                  for k, v in rast.grads.items()},
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
    """Boolean [H,W]: pixels left out of the pixel checks of one view (the
    rule of oracle.exclusions, from the oracle's outputs alone)."""
    return _exc.pixel_exclusion(ora_view, cam, margin)


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
    change by more than the tolerance (oracle.exclusions)."""
    return _exc.gaussian_exclusion(ora_view, cam, bad_pixels, MARGIN)


def rel_norm_err(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def elementwise_violations(g, o, floor=ELEM_FLOOR):
    """Entries of a gradient tensor outside the element-wise bar
    |g - o| <= GRAD_TOL |o| + floor max|o|; returns (count, worst ratio of
    the difference to its bound)."""
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    if o.size == 0:
        return 0, 0.0
    bound = GRAD_TOL * np.abs(o) + floor * np.abs(o).max()
    ratio = np.abs(g - o) / np.maximum(bound, 1e-300)
    return int((ratio > 1.0).sum()), float(ratio.max())


def flip_sensitive(ora_view, cam, prm, dL_dC, dL_dH, g9_all=None):
    """Boolean [N]: Gaussians a near-threshold flip can move by a noticeable
    part of an element (oracle.exclusions.flip_sensitive)."""
    return _exc.flip_sensitive(ora_view, cam, prm, dL_dC, dL_dH, g9_all, FLIP_SHARE, MARGIN)
