"""Training schedule around the rasterizer: the resolution scheduler and the
epoch schedule of the scale reset and the entropy term (Sec. 5.2,
"Implementation Details").

Resolution scheduler (Sec. 5.2, "Resolution Scheduler"): training renders at a
downsampling factor r >= 1, from coarse to full resolution; the largest factor
r_max is chosen so that the mean number of Gaussians per tile stays below a
threshold (about 150 in the paper), and it is capped at 4.  The paper adopts
the rest of the schedule from DashGaussian without stating it; the reading
here is integer levels r_max, r_max - 1, ..., 2 over equal
shares of the first `coarse_fraction` of the epochs, then r = 1.

Epoch schedule (Sec. 5.2, "Scale Reset and Entropy Constraint"): an epoch is a
fixed number of images sampled with replacement (200 in the paper); the scale
reset s <- zeta s runs every `reset_every` epochs (20); within each reset
period the entropy term is on every other epoch (gamma = 0.015); with the
resolution scheduler the regularisation is weaker during the coarse stages
and reaches (zeta, gamma) at full resolution ("stage-adaptive"; the weaker
values are not stated and are parameters here).

This module is host logic only: it chooses factors and switches, and scales
cameras and target images; every rendering runs through ``rasterize``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LIST_THRESHOLD = 150.0  # Gaussians per tile above which coarse levels slow down (Sec. 5.2)
R_CAP = 4  # largest downsampling factor (Sec. 5.2)


def scaled_camera(cam, r: int):
    """The camera of the same view at downsampling factor r: every pixel of
    the coarse image is an r x r block of the full image (floor(W / r) x
    floor(H / r) pixels), so the focal lengths and the principal point scale
    by 1 / r."""
    r = int(r)
    if r < 1:
        raise ValueError("r >= 1")
    if r == 1:
        return dict(cam)
    out = dict(cam)
    out["width"] = cam["width"] // r
    out["height"] = cam["height"] // r
    for k in ("fx", "fy", "cx", "cy"):
        out[k] = cam[k] / r
    return out


def downsample_image(img, r: int):
    """Area (box) average of r x r blocks of an [H, W, C] image (numpy or
    torch), cropped to floor(H / r) x floor(W / r): the target that matches
    scaled_camera(cam, r)."""
    r = int(r)
    if r == 1:
        return img
    H, W = img.shape[0] // r, img.shape[1] // r
    x = img[:H * r, :W * r]
    x = x.reshape(H, r, W, r, -1)
    return x.mean(axis=(1, 3)) if isinstance(x, np.ndarray) else x.mean(dim=(1, 3))


def choose_r_max(mean_list_at, threshold: float = LIST_THRESHOLD, cap: int = R_CAP) -> int:
    """Largest integer factor r in [1, cap] whose mean per-tile list length
    (mean_list_at(r), computed by the caller from the per-tile lists) stays
    at or below `threshold`; 1 if none does.  Coarser levels have longer
    lists (each tile covers more of the scene), so the search runs from the
    cap down and stops at the first factor that qualifies."""
    for r in range(int(cap), 1, -1):
        if mean_list_at(r) <= threshold:
            return r
    return 1


def resolution_levels(r_max: int, epochs: int, coarse_fraction: float = 0.5):
    """Per epoch the downsampling factor: r_max, r_max - 1, ..., 2 over equal
    shares of the first coarse_fraction of the epochs (in that order), then 1."""
    r_max = int(r_max)
    levels = np.ones(int(epochs), np.int64)
    if r_max <= 1 or epochs <= 0:
        return levels
    n_coarse = int(math.floor(coarse_fraction * epochs))
    steps = r_max - 1  # levels r_max .. 2
    for e in range(n_coarse):
        levels[e] = r_max - min(steps - 1, (e * steps) // max(n_coarse, 1))
    return levels


@dataclass
class EpochSchedule:
    """The epoch plan of Sec. 5.2.  images_per_epoch images are sampled with
    replacement per epoch; the scale reset runs after every reset_every-th
    epoch; within each reset period the entropy term is on in every other
    epoch (the second, fourth, ... of the period); coarse stages (r > 1) use
    zeta_coarse / gamma_coarse, full resolution zeta / gamma."""
    epochs: int = 150
    images_per_epoch: int = 200
    reset_every: int = 20
    zeta: float = 0.2
    gamma: float = 0.015
    zeta_coarse: float = 0.5
    gamma_coarse: float = 0.005
    r_max: int = 1
    coarse_fraction: float = 0.5

    def levels(self):
        return resolution_levels(self.r_max, self.epochs, self.coarse_fraction)

    def entropy_on(self, epoch: int) -> bool:
        return (epoch % self.reset_every) % 2 == 1

    def reset_after(self, epoch: int) -> bool:
        return (epoch + 1) % self.reset_every == 0 and epoch + 1 < self.epochs

    def gamma_at(self, epoch: int) -> float:
        if not self.entropy_on(epoch):
            return 0.0
        return self.gamma if self.levels()[epoch] == 1 else self.gamma_coarse

    def zeta_at(self, epoch: int) -> float:
        return self.zeta if self.levels()[epoch] == 1 else self.zeta_coarse

    def image_order(self, n_views: int, seed: int = 0):
        """[epochs, images_per_epoch] view indices, sampled with replacement."""
        rng = np.random.default_rng(seed)
        return rng.integers(0, n_views, (self.epochs, self.images_per_epoch))
