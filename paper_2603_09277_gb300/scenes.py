"""Seeded synthetic scenes, cameras and targets (inputs only).

This module holds random draws and camera placement and nothing of the
rasterizer's arithmetic; both the CUDA path and the FP64 oracle read the
arrays it returns, so the two sides see identical bits.  All arrays are
numpy (float32 unless stated), generated on the host with numpy's PCG64.

The scenes stand in for the paper's Mip-NeRF 360 / Tanks & Temples / Deep
Blending captures (Sec. 5.1), which are not available here.  1237x822 is the
quarter-resolution Mip-NeRF 360 outdoor frame size.

Scene dict keys: means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z,
unit length as drawn), opacity_logits [N], sh [N,16,3] (coefficients beyond
the degree in use are zero), sh_degree.
Camera dict keys: width, height, fx, fy, cx, cy, world_to_cam [3,4]
(row-major [R|t], camera looks along +z, x right, y down), cam_pos [3].
"""
from __future__ import annotations

import math

import numpy as np

# Rendering thresholds and projection constants (FP32 numbers by definition).
DEFAULT_PARAMS = {
    "alpha_max": 0.99,       # alpha clamp
    "alpha_min": 1.0 / 255,  # entries below are skipped
    "t_min": 1e-4,           # the walk stops before T would drop below this
    "dilation": 0.3,         # low-pass term added to the 2D covariance diagonal
    "near_z": 0.2,           # near plane
    "fov_clamp": 1.3,        # x/z, y/z clamp for the EWA Jacobian, x half-fov
    "sh_degree": 0,
}

GAMMA = 0.015  # entropy weight (Sec. 5.2)

# sh_0 = (c - 0.5) / Y00 with c ~ U[0,1] and 1 / Y00 = 2 sqrt(pi) gives a DC
# coefficient uniform on [-sqrt(pi), sqrt(pi)].
_DC_HALF_RANGE = math.sqrt(math.pi)


def params(**kw):
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    return p


def camera(width, height, f, R=None, pos=None):
    """Pinhole camera with principal point at the image centre.  R (3x3) maps
    world to camera axes; pos is the camera centre in world space."""
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    pos = np.zeros(3) if pos is None else np.asarray(pos, np.float64)
    R32 = R.astype(np.float32)
    t = -(R32.astype(np.float64) @ pos)
    wtc = np.concatenate([R32, t.astype(np.float32)[:, None]], axis=1)
    # camera centre from the stored FP32 [R|t]: c = -R^T t
    cp = -(wtc[:, :3].astype(np.float64).T @ wtc[:, 3].astype(np.float64))
    return {
        "width": int(width), "height": int(height),
        "fx": float(f), "fy": float(f),
        "cx": width / 2.0, "cy": height / 2.0,
        "world_to_cam": wtc.astype(np.float32),
        "cam_pos": cp.astype(np.float32),
    }


def look_at(pos, target, up=(0.0, -1.0, 0.0)):
    """World->camera rotation whose +z points from pos to target, with y down."""
    pos, target, up = (np.asarray(a, np.float64) for a in (pos, target, up))
    f = target - pos
    f /= np.linalg.norm(f)
    r = np.cross(up, f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return np.stack([r, d, f])


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sh_deg0(rng, n):
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 3))
    return sh


def box_scene(n, seed=0, ls_mean=-3.5, ls_std=0.5, box=((-1, 1), (-1, 1), (2, 6)),
              opacity_mean=0.0):
    """Uniform means in a box (camera space of an identity camera), log-scales
    N(ls_mean, ls_std), unit quaternions, opacity logits N(opacity_mean, 1),
    SH degree 0 with colour U[0,1]."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box], np.float64)
    hi = np.array([b[1] for b in box], np.float64)
    means = (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)
    ls = rng.normal(ls_mean, ls_std, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    op = rng.normal(opacity_mean, 1.0, n).astype(np.float32)
    sh = _sh_deg0(rng, n)
    return {"means": means, "log_scales": ls, "quats": quats, "opacity_logits": op,
            "sh": sh, "sh_degree": 0}


def cluster_scene(n, seed=0, n_clusters=64, radius=10.0, ls_mean=-4.0, ls_std=0.7,
                  sh_degree=3, sh_std=0.2):
    """Means from a mixture of anisotropic 3D Gaussian clusters (centres
    uniform in a ball, axis stds U[0.3, 2], random orientation), points
    outside the ball redrawn; log-scales N(ls_mean, ls_std); SH coefficients
    N(0, sh_std) up to sh_degree; opacity logits N(0, 1)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n_clusters, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    centres = u * radius * rng.random((n_clusters, 1)) ** (1.0 / 3.0)
    stds = rng.uniform(0.3, 2.0, (n_clusters, 3))
    rots = []
    for _ in range(n_clusters):
        qm, rm = np.linalg.qr(rng.standard_normal((3, 3)))
        rots.append(qm * np.sign(np.diag(rm)))
    rots = np.stack(rots)
    means = np.zeros((n, 3), np.float64)
    todo = np.arange(n)
    while todo.size:
        k = rng.integers(0, n_clusters, todo.size)
        z = rng.standard_normal((todo.size, 3)) * stds[k]
        p = centres[k] + np.einsum("nij,nj->ni", rots[k], z)
        ok = np.linalg.norm(p, axis=1) <= radius
        means[todo[ok]] = p[ok]
        todo = todo[~ok]
    ls = rng.normal(ls_mean, ls_std, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    op = rng.normal(0.0, 1.0, n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, :K, :] = rng.normal(0.0, sh_std, (n, K, 3))
    return {"means": means.astype(np.float32), "log_scales": ls, "quats": quats,
            "opacity_logits": op, "sh": sh, "sh_degree": sh_degree}


def noise_targets(cams, seed=1):
    """Per view a target image U[0,1]^3 per pixel, [H,W,3] float32."""
    rng = np.random.default_rng(seed)
    return [rng.random((c["height"], c["width"], 3), dtype=np.float32) for c in cams]


def yaw_cameras(sizes, yaws_deg, centre=(0.0, 0.0, 4.0)):
    """Cameras at the origin rotated by a yaw about the vertical axis through
    `centre`, each looking at `centre`; f = width."""
    cams = []
    c = np.asarray(centre, np.float64)
    for (w, h), yd in zip(sizes, yaws_deg):
        th = math.radians(yd)
        pos = c + np.array([-c[2] * math.sin(th), 0.0, -c[2] * math.cos(th)])
        R = look_at(pos, c)
        cams.append(camera(w, h, w, R, pos))
    return cams


# ----------------------------------------------------------------------------
# The five workload configurations.  Each returns (scene, cams, targets, prm).
# ----------------------------------------------------------------------------

def config1(seed=0, n=10_000):
    """Plain method, one 256x256 view (f = 256, principal point centred),
    10,000 Gaussians uniform in [-1,1]^2 x [2,6] in camera space, log-scales
    N(-3.5, 0.5), SH degree 0, uniform-noise target."""
    scene = box_scene(n, seed)
    cams = [camera(256, 256, 256.0)]
    return scene, cams, noise_targets(cams, seed + 1), params(sh_degree=0)


def config2(seed=0, n=1_000_000):
    """Scene scale: 1,000,000 Gaussians from 64 anisotropic clusters within
    radius 10, log-scales N(-4, 0.7), SH degree 3 ~ N(0, 0.2); one 1237x822
    view (f = 1237) from a radius-4 orbit at height 0.5 looking at the origin."""
    scene = cluster_scene(n, seed)
    rng = np.random.default_rng(seed + 1000)
    th = rng.uniform(0.0, 2.0 * math.pi)
    pos = np.array([4.0 * math.cos(th), 0.5, 4.0 * math.sin(th)])
    cams = [camera(1237, 822, 1237.0, look_at(pos, (0.0, 0.0, 0.0)), pos)]
    return scene, cams, noise_targets(cams, seed + 1), params(sh_degree=3)


CONFIG3_SIZES = [(309, 205)] * 3 + [(618, 411)] * 3 + [(1237, 822)] * 2


def config3(seed=0, n=3_000_000, density_matched=False):
    """Batched: the config-1 distribution with n Gaussians, 8 views of uneven
    resolution (3 x 309x205, 3 x 618x411, 2 x 1237x822; f = width), cameras at
    yaw 0 and 7 seeded yaws within +-15 degrees about (0, 0, 4).
    density_matched scales sizes by (1e4 / n)^(1/3) (labelled variant)."""
    ls_mean = -3.5 + (math.log((1e4 / n) ** (1.0 / 3.0)) if density_matched else 0.0)
    scene = box_scene(n, seed, ls_mean=ls_mean)
    rng = np.random.default_rng(seed + 2000)
    yaws = [0.0] + list(rng.uniform(-15.0, 15.0, 7))
    cams = yaw_cameras(CONFIG3_SIZES, yaws)
    return scene, cams, noise_targets(cams, seed + 1), params(sh_degree=0)


def config4(k=0, opacity_mean=0.0, seed=0, n=10_000):
    """List-length sweep: the config-1 scene with scales times 0.5^k (log-scale
    mean shifted by k ln 0.5) and opacity-logit mean opacity_mean."""
    scene = box_scene(n, seed, ls_mean=-3.5 + k * math.log(0.5), opacity_mean=opacity_mean)
    cams = [camera(256, 256, 256.0)]
    return scene, cams, noise_targets(cams, seed + 1), params(sh_degree=0)


def config5(seed=0, n=3_000_000, width=1920, height=1080):
    """Mixed-precision workload: the config-1 distribution with n Gaussians,
    the box's y extent scaled to the 16:9 field of view, one width x height
    view with f = width."""
    ar = height / width
    scene = box_scene(n, seed, box=((-1, 1), (-ar, ar), (2, 6)))
    cams = [camera(width, height, float(width))]
    return scene, cams, noise_targets(cams, seed + 1), params(sh_degree=0)


def orbit_cameras(n_views, width, height, radius=4.0, centre=(0.0, 0.0, 4.0), height_off=0.5,
                  seed=0):
    """n_views cameras on a circle of `radius` around `centre`, looking at it."""
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, np.float64)
    th0 = rng.uniform(0, 2 * math.pi)
    cams = []
    for i in range(n_views):
        th = th0 + 2 * math.pi * i / n_views
        pos = c + np.array([radius * math.sin(th), height_off, -radius * math.cos(th)])
        cams.append(camera(width, height, float(width), look_at(pos, c), pos))
    return cams


def tiny_scene(n, seed=0, width=32, height=32, ls_mean=-2.5, sh_degree=0):
    """A few Gaussians in front of a small identity camera, for brute force
    and finite-difference checks."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n),
                      rng.uniform(2.0, 4.0, n)], 1).astype(np.float32)
    ls = rng.normal(ls_mean, 0.3, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    op = rng.normal(0.5, 1.0, n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, :K, :] = rng.normal(0.0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 3)) * 0.8
    scene = {"means": means, "log_scales": ls, "quats": quats, "opacity_logits": op,
             "sh": sh, "sh_degree": sh_degree}
    cams = [camera(width, height, float(width))]
    return scene, cams, noise_targets(cams, seed + 1), params(sh_degree=sh_degree)
