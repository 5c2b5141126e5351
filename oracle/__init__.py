"""FP64 CPU oracle for the 16x16-tile Gaussian rasterizer with the entropy term
on blending weights (arXiv 2603.09277, Sec. 3-4 and Suppl. A-C).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2603_09277_gb300``); the two meet only in
the seeded input generators (``paper_2603_09277_gb300.scenes``), which hold
none of the method's arithmetic.

The arithmetic lives in ``gs_oracle.c`` (plain C, IEEE double, OpenMP over
pixels and Gaussians); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.

Functions (all inputs are numpy arrays as produced by ``scenes``):

- ``preprocess``: per-Gaussian projection of one view (Sec. 3).
- ``build_lists``: per-tile Gaussian lists sorted by (depth key, id), for
  square tiles of 16 px (3DGS) or 8 px (prm["tile"] = 8: LiteGS and the
  paper's own runs, Sec. 5 "Effect of tile sizes").
- ``render_fwd``: compositing, transmittance and per-pixel entropy (Sec. 3,
  Sec. 4.3), with a per-pixel threshold margin.
- ``render_bwd``: dL/d(2D attributes) from the closed forms (Sec. 4.4,
  Suppl. B, Suppl. C) with inner sums written out.
- ``preprocess_bwd``: dL/d(parameters) by the complex step.
- ``loss``: L1 + gamma * mean entropy (Sec. 3 eq. base with lambda = 0, Sec. 4.3).
- ``dH_dalpha_{direct,closed,alg1}``, ``entropy``: the entropy gradient
  three ways (Suppl. B, Sec. 4.4, Algorithm 1).
- ``scale_reset``: s <- zeta s (Sec. 4.2).
- ``step``: the whole forward + backward over several views.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgs_oracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compiles gs_oracle.c into oracle/_build/libgs_oracle.so (gcc, FP64,
    no fast-math, no FP contraction).  Returns the library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.ora_entropy.restype = ctypes.c_double
            _lib.ora_ssim.restype = ctypes.c_double
            _lib.ora_loss.restype = ctypes.c_double
            _lib.ora_build_lists.restype = ctypes.c_longlong
            _lib.ora_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().ora_num_threads())


def cam_vector(cam) -> np.ndarray:
    """Flattens a camera dict (width, height, fx, fy, cx, cy, world_to_cam
    [3x4 float32], cam_pos [3 float32]) into the oracle's double layout."""
    v = np.zeros(21, np.float64)
    v[0] = cam["width"]
    v[1] = cam["height"]
    v[2:6] = [np.float32(cam["fx"]), np.float32(cam["fy"]),
              np.float32(cam["cx"]), np.float32(cam["cy"])]
    v[6:18] = np.asarray(cam["world_to_cam"], np.float32).reshape(12)
    v[18:21] = np.asarray(cam["cam_pos"], np.float32).reshape(3)
    return v


def prm_vector(prm) -> np.ndarray:
    """Thresholds are FP32 numbers by definition; widen the FP32 values.
    The last entry is the tile side in pixels (16 unless prm says 8)."""
    keys = ["alpha_max", "alpha_min", "t_min", "dilation", "near_z", "fov_clamp"]
    v = [np.float32(prm[k]) for k in keys] + [tile_of(prm)]
    return np.array(v, np.float64)


def tile_of(prm) -> int:
    """Tile side in pixels: 16 (3DGS) or 8 (LiteGS and the paper's runs,
    Sec. 5 "Effect of tile sizes")."""
    t = int(prm.get("tile", TILE)) if prm is not None else TILE
    if t not in (8, 16):
        raise ValueError("tile side must be 8 or 16")
    return t


def tile_grid(cam, prm=None):
    t = tile_of(prm)
    return (cam["width"] + t - 1) // t, (cam["height"] + t - 1) // t


def preprocess(scene, cam, prm):
    """Per-Gaussian projection of one view.  Returns dict with P9 [N,9]
    (mean2d x,y; conic a,b,c; opacity; rgb), depth [N] f32, radius, rect
    [N,4], tiles [N], clamped [N,3], boundary [N] (rect may differ in FP32),
    rect_lo / rect_hi [N,4] (intersection / union of the rects reachable
    under the FP32 rounding bands; set for flagged Gaussians)."""
    lib = _load()
    means, ls, q, op, sh = (_f64(scene["means"]), _f64(scene["log_scales"]),
                            _f64(scene["quats"]), _f64(scene["opacity_logits"]),
                            _f64(scene["sh"]))
    N = means.shape[0]
    Kst = sh.shape[1]
    deg = int(scene["sh_degree"])
    out = {
        "P9": np.zeros((N, 9), np.float64),
        "depth": np.zeros(N, np.float32),
        "radius": np.zeros(N, np.int32),
        "rect": np.zeros((N, 4), np.int32),
        "tiles": np.zeros(N, np.int32),
        "clamped": np.zeros((N, 3), np.int32),
        "boundary": np.zeros(N, np.int32),
        "rect_lo": np.zeros((N, 4), np.int32),
        "rect_hi": np.zeros((N, 4), np.int32),
    }
    out["tile"] = tile_of(prm)
    lib.ora_preprocess(ctypes.c_int(N), _p(means), _p(ls), _p(q), _p(op), _p(sh),
                       ctypes.c_int(Kst), ctypes.c_int(deg), _p(cam_vector(cam)),
                       _p(prm_vector(prm)), _p(out["P9"]), _p(out["depth"]), _p(out["radius"]),
                       _p(out["rect"]), _p(out["tiles"]), _p(out["clamped"]),
                       _p(out["boundary"]), _p(out["rect_lo"]), _p(out["rect_hi"]))
    return out


def build_lists(proj, cam, tile_mask=None):
    """Per-tile lists: tile_start [TX*TY+1] int64 and ids [P] int32, each
    tile's ids sorted by (FP32 depth bits, Gaussian id).  tile_mask
    (optional bool [TX*TY]) keeps only the marked tiles' lists."""
    lib = _load()
    TX, TY = tile_grid(cam, {"tile": proj.get("tile", TILE)})
    rect, tiles, depth = proj["rect"], proj["tiles"], proj["depth"]
    N = rect.shape[0]
    ts = np.zeros(TX * TY + 1, np.int64)
    m = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8).reshape(-1)
    P = lib.ora_build_lists(ctypes.c_int(N), _p(rect), _p(tiles), _p(depth), ctypes.c_int(TX),
                            ctypes.c_int(TY), _p(ts), ctypes.c_void_p(0), _p(m))
    ids = np.zeros(max(P, 1), np.int32)
    lib.ora_build_lists(ctypes.c_int(N), _p(rect), _p(tiles), _p(depth), ctypes.c_int(TX),
                        ctypes.c_int(TY), _p(ts), _p(ids), _p(m))
    return ts, ids[:P]


def render_fwd(proj, lists, cam, prm, mask=None):
    """Compositing of one view.  Returns image [H,W,3], final_T, last (1-based
    list position of the last blended entry, 0 if none), entropy, nblend,
    neval, margin (smallest relative distance of any threshold test) and
    first_near (first list position whose test is within 1e-3 of a
    threshold, -1 if none)."""
    lib = _load()
    W, H = cam["width"], cam["height"]
    ts, ids = lists
    ids = np.ascontiguousarray(ids, np.int32) if len(ids) else np.zeros(1, np.int32)
    o = {
        "image": np.zeros((H, W, 3), np.float64),
        "final_T": np.zeros((H, W), np.float64),
        "last": np.zeros((H, W), np.int32),
        "entropy": np.zeros((H, W), np.float64),
        "nblend": np.zeros((H, W), np.int32),
        "neval": np.zeros((H, W), np.int32),
        "margin": np.full((H, W), np.inf, np.float64),
        "first_near": np.full((H, W), -1, np.int32),
    }
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lib.ora_render_fwd(ctypes.c_int(W), ctypes.c_int(H), _p(ts), _p(ids), _p(proj["P9"]),
                       _p(prm_vector(prm)), _p(m), _p(o["image"]), _p(o["final_T"]),
                       _p(o["last"]), _p(o["entropy"]), _p(o["nblend"]), _p(o["neval"]),
                       _p(o["margin"]), _p(o["first_near"]))
    return o


def render_bwd(proj, lists, cam, prm, dL_dC, dL_dH, mask=None):
    """dL/d(mean2d, conic, opacity, rgb) [N,9] of one view."""
    lib = _load()
    W, H = cam["width"], cam["height"]
    ts, ids = lists
    ids = np.ascontiguousarray(ids, np.int32) if len(ids) else np.zeros(1, np.int32)
    N = proj["P9"].shape[0]
    g = np.zeros((N, 9), np.float64)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lib.ora_render_bwd(ctypes.c_int(W), ctypes.c_int(H), _p(ts), _p(ids), _p(proj["P9"]),
                       _p(prm_vector(prm)), _p(m), _p(_f64(dL_dC)),
                       _p(None if dL_dH is None else _f64(dL_dH)), _p(g))
    return g


def preprocess_bwd(scene, cam, prm, grad9, grads=None, gmask=None):
    """Accumulates dL/d(parameters) of one view into ``grads`` (created if
    None) by the complex step through the projection."""
    lib = _load()
    means, ls, q, op, sh = (_f64(scene["means"]), _f64(scene["log_scales"]),
                            _f64(scene["quats"]), _f64(scene["opacity_logits"]),
                            _f64(scene["sh"]))
    N, Kst = means.shape[0], sh.shape[1]
    if grads is None:
        grads = {
            "means": np.zeros((N, 3)), "log_scales": np.zeros((N, 3)),
            "quats": np.zeros((N, 4)), "opacity_logits": np.zeros(N),
            "sh": np.zeros((N, Kst, 3)),
        }
    m = None if gmask is None else np.ascontiguousarray(gmask, np.uint8)
    lib.ora_preprocess_bwd(ctypes.c_int(N), _p(means), _p(ls), _p(q), _p(op), _p(sh),
                           ctypes.c_int(Kst), ctypes.c_int(int(scene["sh_degree"])),
                           _p(cam_vector(cam)), _p(prm_vector(prm)), _p(_f64(grad9)), _p(m),
                           _p(grads["means"]), _p(grads["log_scales"]), _p(grads["quats"]),
                           _p(grads["opacity_logits"]), _p(grads["sh"]))
    return grads


def loss(image, entropy, target, gamma, view_weight=1.0):
    """L1 + gamma * (1/M) sum H of one view, times view_weight; returns
    (L, dL/dC [H,W,3], dL/dH [H,W])."""
    lib = _load()
    image, entropy = _f64(image), _f64(entropy)
    M = entropy.size
    dC = np.zeros_like(image)
    dH = np.zeros_like(entropy)
    L = lib.ora_loss(ctypes.c_int(M), _p(image), _p(_f32(target)), _p(entropy),
                     ctypes.c_double(gamma), ctypes.c_double(view_weight), _p(dC), _p(dH))
    return float(L), dC, dH


def ssim(image, target, with_grad=False):
    """Mean SSIM of an [H,W,3] image against its target (the D-SSIM term's
    SSIM: 11x11 Gaussian window of sigma 1.5, zero padding, C1 = 0.01^2,
    C2 = 0.03^2); with_grad also returns d SSIM / d image [H,W,3]."""
    lib = _load()
    image = _f64(image)
    H, W = image.shape[:2]
    g = np.zeros_like(image) if with_grad else None
    s = lib.ora_ssim(ctypes.c_int(W), ctypes.c_int(H), _p(image), _p(_f32(target)), _p(g))
    return (float(s), g) if with_grad else float(s)


def loss_base(image, entropy, target, gamma, lam, view_weight=1.0):
    """(1 - lam) L1 + lam (1 - SSIM) + gamma (1/M) sum H of one view (Sec. 3
    Eq. base with D-SSIM = 1 - SSIM, plus the entropy term of Sec. 4.3), times
    view_weight; returns (L, dL/dC, dL/dH)."""
    L1, dC, dH = loss(image, entropy, target, 0.0, view_weight)
    Lh, _, dH = loss(image, entropy, target, gamma, view_weight)
    Lent = Lh - L1
    s, gs = ssim(image, target, with_grad=True)
    L = (1 - lam) * L1 + view_weight * lam * (1 - s) + Lent
    return L, (1 - lam) * dC - view_weight * lam * gs, dH


def entropy(alphas):
    a = _f64(alphas)
    return float(_load().ora_entropy(ctypes.c_int(a.size), _p(a)))


def _dH(fn, alphas):
    a = _f64(alphas)
    out = np.zeros_like(a)
    getattr(_load(), fn)(ctypes.c_int(a.size), _p(a), _p(out))
    return out


def dH_dalpha_direct(alphas):
    return _dH("ora_dH_da_direct", alphas)


def dH_dalpha_closed(alphas):
    return _dH("ora_dH_da_closed", alphas)


def dH_dalpha_alg1(alphas):
    return _dH("ora_dH_da_alg1", alphas)


def sh_basis(deg, dirs):
    d = _f64(dirs).reshape(-1, 3)
    Y = np.zeros((d.shape[0], 16), np.float64)
    _load().ora_sh_basis(ctypes.c_int(deg), _p(d), ctypes.c_int(d.shape[0]), _p(Y))
    return Y


def scale_reset(log_scales, zeta):
    ls = _f32(log_scales)
    out = np.zeros(ls.shape, np.float64)
    _load().ora_scale_reset(ctypes.c_int(ls.size), _p(ls), ctypes.c_double(zeta), _p(out))
    return out


def forward(scene, cams, prm, mask=None):
    """Per view: projection, lists and compositing.  Returns a list of dicts."""
    views = []
    for v, cam in enumerate(cams):
        proj = preprocess(scene, cam, prm)
        lists = build_lists(proj, cam)
        fwd = render_fwd(proj, lists, cam, prm, None if mask is None else mask[v])
        views.append({"proj": proj, "lists": lists, "fwd": fwd})
    return views


def step(scene, cams, targets, prm, gamma, with_grad=True, lam=0.0):
    """One forward + backward of L = (1/V) sum_v (L1_v + gamma L_E,v)
    (reading: per-view pixel averages, then the mean over views); with
    lam > 0 the L1 term is L_base = (1 - lam) L1 + lam D-SSIM.
    Returns (L, views, grads, grad9 per view)."""
    views = forward(scene, cams, prm)
    V = len(cams)
    L = 0.0
    grads = None
    g9s = []
    for v, cam in enumerate(cams):
        f = views[v]["fwd"]
        if lam > 0.0:
            Lv, dC, dH = loss_base(f["image"], f["entropy"], targets[v], gamma, lam, 1.0 / V)
        else:
            Lv, dC, dH = loss(f["image"], f["entropy"], targets[v], gamma, 1.0 / V)
        L += Lv
        views[v]["dL_dC"], views[v]["dL_dH"] = dC, dH
        if with_grad:
            g9 = render_bwd(views[v]["proj"], views[v]["lists"], cam, prm, dC, dH)
            g9s.append(g9)
            grads = preprocess_bwd(scene, cam, prm, g9, grads)
    return L, views, grads, g9s
