#!/usr/bin/env python
"""Benchmark of the differentiable tile rasterizer with the entropy term:
one step = projection, per-tile list construction (depth sort of the visible
rows, super-tile items, expansion into the tiles' lists), front-to-back
blending with the weight entropy, the L1 + entropy loss, the reverse-order
adjoint back to every Gaussian parameter, and the scale reset, over one batch
of synthetic inputs resident in HBM.

The JSON line carries, besides the contract's keys: the per-phase event times
(eager) and graph replays, the roofline of the dominant kernel (FP32 FLOP
model) and of the other phases (minimal algorithmic bytes against the
measured HBM copy bandwidth), the FP64 oracle on the host cores as the CPU
baseline, the end-to-end time through the C ABI (target images in, loss out;
and the stricter form with every parameter uploaded), the library's own
launch count and the SM clocks sampled during the timed region.  Other modes:
--config cfg1..cfg5, --tile 8, --dssim LAMBDA, --attr f16|bf16, --sweep
(list-length sweep), --train ITERS (training loop), --train-epochs E (epoch
schedule with the resolution scheduler).

Default workload (N=1): the batched configuration, 3,000,000 Gaussians
seen from 8 views of uneven size (3 x 309x205, 3 x 618x411, 2 x 1237x822, a
progressive-resolution mix) in one pipeline.  Metric: blended
Gaussian-pixels per second over the whole forward + backward step (higher is
better), ms per step alongside; the same line carries the plain form (one
single-view FP32 pipeline per view), the FP16/BF16 staging forms and the other
launch forms, each with its ms per step and its error against the FP64 oracle
on view 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica on its own seeded
scene (the path shards by view/scene and needs no data exchange); the
barrier and the max-over-ranks time are timing plumbing only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/iter and blended Gaussian-pixels/s, batched+mixed vs plain at stated err"
UNIT = "blended Gaussian-pixels/s"
L2_BYTES = 129 * 1024 * 1024

# Algorithmic FP32 operation counts per pair (add/mul/min/transcendental = 1,
# fused multiply-add = 2), from the per-pair formulas of the blending and its
# adjoint:
#   forward:  10 per evaluated pair (pixel offset 2, base-2 exponent 8)
#             +14 per blended pair (exp, clamp, 1-alpha, T(1-alpha), w,
#                 colour 3 FMA, log, entropy FMA)
#   backward: 10 per evaluated pair, +56 per blended pair (transmittance
#             recovery 8, colour part of dL/dalpha 14, entropy part 7, colour
#             gradient 3, S and R updates 9, dd and the six moments
#             dd (1, dx, dy, dx^2, dx dy, dy^2) summed 12, colour sums 3; the
#             conic, 1/sigma and the signs are applied once per Gaussian)
FWD_EVAL, FWD_BLEND = 10, 14
BWD_EVAL, BWD_BLEND = 10, 56


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg3", choices=["cfg1", "cfg2", "cfg3", "cfg4", "cfg5"])
    ap.add_argument("--attr", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--n", type=int, default=0,
                    help="override the configuration's Gaussian count (smaller cases for profiling)")
    ap.add_argument("--persistent", type=int, default=0,
                    help="CTAs of the persistent list-length-ordered launch (0 = one CTA per tile)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the comparison of launch forms and staging precisions")
    ap.add_argument("--ppt", type=int, default=0, help="pixels per thread of the blending kernels")
    ap.add_argument("--batch", type=int, default=0, choices=[0, 128, 256],
                    help="list entries per shared-memory batch of the blending kernels (0 = 256)")
    ap.add_argument("--dssim", type=float, default=0.0,
                    help="lambda of the D-SSIM term of L_base (0: L1 + entropy, the workloads' "
                         "stated loss; 3DGS uses 0.2)")
    ap.add_argument("--tile", type=int, default=16, choices=[16, 8],
                    help="tile side in pixels (16: 3DGS; 8: LiteGS and the paper's runs)")
    ap.add_argument("--no-phase-graphs", action="store_true",
                    help="skip the per-phase graph replays (launch-list captures)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --ppt/--batch/--persistent as given instead of the autotuned form")
    ap.add_argument("--sweep", action="store_true",
                    help="list-length sweep (cfg4): one JSON line per scale/opacity point")
    ap.add_argument("--train", type=int, default=0,
                    help="run the synthetic training loop (cfg5 form) for this many iterations")
    ap.add_argument("--train-size", default="960x540", help="training view size WxH")
    ap.add_argument("--train-n", type=int, default=3_000_000, help="Gaussians in the training scene")
    ap.add_argument("--train-epochs", type=int, default=0,
                    help="run the epoch schedule (resolution scheduler, scale reset every "
                         "--reset-every epochs, entropy on every other epoch) for N epochs")
    ap.add_argument("--images-per-epoch", type=int, default=200)
    ap.add_argument("--reset-every", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-band-rows", type=int, default=0,
                    help="tile rows of view 0 the CPU oracle sample renders (0 = the whole view)")
    ap.add_argument("--ref-band-rows", type=int, default=2,
                    help="tile rows per step of the reference (oracle) arm")
    return ap.parse_args()


def workload(name, seed, n=0):
    from paper_2603_09277_gb300 import scenes
    kw = {"n": n} if n else {}
    tag = " (N overridden: %d)" % n if n else ""
    if name == "cfg1":
        return scenes.config1(seed=seed, **kw), "cfg1: 10k Gaussians, 256x256, SH0, fwd+bwd L1+entropy" + tag
    if name == "cfg2":
        return scenes.config2(seed=seed, **kw), ("cfg2: 1M Gaussians (64 clusters, r=10), SH3, "
                                                 "one 1237x822 view, fwd+bwd L1+entropy" + tag)
    if name == "cfg3":
        return scenes.config3(seed=seed, **kw), ("cfg3: 3M Gaussians, 8 views {3x309x205, "
                                                 "3x618x411, 2x1237x822}, fwd+bwd L1+entropy" + tag)
    if name == "cfg4":
        return scenes.config4(seed=seed, **kw), "cfg4: 10k Gaussians, 256x256, k=0" + tag
    return scenes.config5(seed=seed, **kw), ("cfg5: 3M Gaussians, 1920x1080, SH0, fwd+bwd "
                                             "L1+entropy" + tag)


# ---------------------------------------------------------------------------
# Clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            out = summarise_clock_rows(f.read().splitlines())
        os.unlink(self.path)
        return out


def summarise_clock_rows(lines):
    """The `clocks` object of the JSON line from nvidia-smi CSV rows (the
    ClockSampler.FIELDS columns, no header, no units): the median SM clock,
    the largest maximum clock, and every throttle reason seen Active.  Rows
    that do not parse (a header, "[N/A]") are skipped; None without rows."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i] == "Active"})
    return {"sm_mhz": float(np.median([r[0] for r in rows])),
            "sm_max_mhz": float(max(r[1] for r in rows)), "reasons": reasons,
            "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample(scene, cams, targets, prm, gamma, band_rows, keep=False):
    """Runs the FP64 oracle's whole pipeline on a band of `band_rows` tile
    rows through the middle of view 0: projection of every Gaussian, the tile
    lists of the band's tiles, forward and backward on the band's pixels, and
    the projection adjoint of every Gaussian that received a gradient.
    Returns (blended pairs, seconds, description[, reference]); with keep,
    the reference holds the band mask, the oracle's image, final T and
    entropy of view 0 and the pixels whose FP32 result may take the other
    branch of a threshold test (excluded from the error statement)."""
    import oracle
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    T = int(prm.get("tile", 16))
    TX, TY = (W + T - 1) // T, (H + T - 1) // T
    if band_rows <= 0 or band_rows > TY:
        band_rows = TY
    t_start = max(0, TY // 2 - band_rows // 2)
    rows = np.arange(H) // T
    band = (rows >= t_start) & (rows < t_start + band_rows)
    mask = np.repeat(band[:, None], W, axis=1)
    tmask = np.zeros((TY, TX), bool)
    tmask[t_start:t_start + band_rows] = True
    t0 = time.perf_counter()
    proj = oracle.preprocess(scene, cam, prm)
    lists = oracle.build_lists(proj, cam, tile_mask=None if band_rows == TY else tmask)
    fwd = oracle.render_fwd(proj, lists, cam, prm, mask=mask)
    M = W * H
    dC = np.where(fwd["image"] - targets[0] > 0, 1.0, -1.0) / (3 * M)
    dC[~mask] = 0
    dH = np.where(mask, gamma / M, 0.0)
    g9 = oracle.render_bwd(proj, lists, cam, prm, dC, dH, mask=mask)
    touched = (np.abs(g9).sum(1) > 0).astype(np.uint8)
    oracle.preprocess_bwd(scene, cam, prm, g9, gmask=touched)
    dt = time.perf_counter() - t0
    nb = int(fwd["nblend"][mask].sum())
    desc = ("FP64 oracle, %d tile rows (%d of %d pixels) of view 0 (%dx%d): projection of all "
            "%d Gaussians, the band's lists, fwd+bwd on the band, projection adjoint of the %d "
            "Gaussians with a gradient" % (band_rows, int(mask.sum()), M, W, H,
                                           scene["means"].shape[0], int(touched.sum())))
    if not keep:
        return nb, dt, desc
    # threshold-boundary exclusions (from the oracle alone): pixels with a
    # threshold test within 1e-4 (relative) of its limit, and pixels whose
    # walk meets a Gaussian that an FP32 rounding may add to or drop from
    # their tile's list
    from oracle import exclusions
    view = {"proj": proj, "lists": lists, "fwd": fwd}
    excl = exclusions.pixel_exclusion(view, cam, prm=prm) & mask
    summ = exclusions.summary(view, cam, mask, prm=prm)
    summ["flagged_ids"] = summ["flagged_ids"][:32]
    ref = {"mask": mask, "image": fwd["image"], "final_T": fwd["final_T"],
           "entropy": fwd["entropy"], "excluded": excl,
           "exclusions": dict(summ, view=0)}
    return nb, dt, desc, ref


def view0_error(ref, image, final_T, entropy):
    """Largest absolute difference from the FP64 oracle over the compared
    pixels of view 0 (device tensors of the whole pipeline; view 0 comes
    first), per output."""
    H, W = ref["mask"].shape
    n = W * H
    ok = ref["mask"] & ~ref["excluded"]
    img = image[:n].detach().cpu().numpy().astype(np.float64).reshape(H, W, 3)
    t = final_T[:n].detach().cpu().numpy().astype(np.float64).reshape(H, W)
    h = entropy[:n].detach().cpu().numpy().astype(np.float64).reshape(H, W)
    return {"image": float(np.abs(img - ref["image"])[ok].max()),
            "final_T": float(np.abs(t - ref["final_T"])[ok].max()),
            "entropy": float(np.abs(h - ref["entropy"])[ok].max())}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    (scene, cams, targets, prm), wl = workload(args.config, 0, args.n)
    prm["tile"] = args.tile
    from paper_2603_09277_gb300 import scenes
    for _ in range(args.warmup):
        oracle_sample(scene, cams, targets, prm, scenes.GAMMA, args.ref_band_rows)
    nbs, dts = [], []
    desc = ""
    for _ in range(args.steps):
        nb, dt, desc = oracle_sample(scene, cams, targets, prm, scenes.GAMMA, args.ref_band_rows)
        nbs.append(nb)
        dts.append(dt)
    value = sum(nbs) / sum(dts)
    cores = oracle.num_threads()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * np.mean(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl,
                       "sample": "%d tile rows of view 0 per step" % args.ref_band_rows},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def traffic_from_profiles(kernel, config):
    """DRAM bytes per launch of `kernel` on workload `config` from the
    committed ncu summary (profiles/traffic.json: a list of entries, one per
    kernel and workload), if that entry was captured from the current source
    of the kernel's file (csrc/<source>)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        data = json.load(open(path))
    except ValueError:
        return None
    entries = data.get("entries", []) if isinstance(data, dict) else []
    for ent in entries:
        if ent.get("kernel") != kernel or ent.get("config") != config:
            continue
        src = os.path.join(ROOT, "paper_2603_09277_gb300", "csrc", ent.get("source", ""))
        if not ent.get("source") or not os.path.exists(src):
            return None
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return ent.get("bytes_per_launch") if ent.get("source_sha256_16") == h else None
    return None


def run_sweep(args, dev):
    """cfg4: the 10k-Gaussian 256x256 scene with scales x 0.5^k and the
    opacity-logit mean varied; per point the pair count, the mean list
    length per tile, evaluated and blended entries per pixel, and the fwd+bwd
    time and throughput (CUDA graph replay, L2 flushed)."""
    import torch
    from paper_2603_09277_gb300 import scenes
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device, targets_to_device
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    for k in range(-2, 5):
        for om in (-2.0, 0.0, 2.0, 4.0):
            scene, cams, targets, prm = scenes.config4(k=k, opacity_mean=om)
            N = scene["means"].shape[0]
            p = scene_to_device(scene, dev)
            tgt = targets_to_device(targets, dev)
            r = Rasterizer(cams, prm, N, device=dev)
            for _ in range(2):
                r.step(p, tgt, scenes.GAMMA, sync=True)
                r.render_fwd(stats=True)
            torch.cuda.synchronize()
            nb, ne = int(r.stats[0].item()), int(r.stats[1].item())
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream()
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                with torch.cuda.graph(g, stream=cs):
                    r.step(p, tgt, scenes.GAMMA, sync=False)
            torch.cuda.current_stream().wait_stream(cs)
            g.replay()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for i in range(args.steps):
                flush.fill_(float(i))
                a.record()
                g.replay()
                b.record()
                b.synchronize()
                ms.append(a.elapsed_time(b))
            pix = cams[0]["width"] * cams[0]["height"]
            m = float(np.mean(ms))
            print(json.dumps({"sweep": "cfg4", "scale_exp_k": k, "opacity_logit_mean": om,
                              "pairs": r.num_pairs, "mean_list_per_tile": r.num_pairs / r.total_tiles,
                              "evaluated_per_pixel": ne / pix, "blended_per_pixel": nb / pix,
                              "ms_per_step": m, "blended_per_s": nb / (m / 1000.0)}), flush=True)
            del r, g
            torch.cuda.empty_cache()


def run_train(args, dev):
    """cfg5 training form: a seeded ground-truth Gaussian set renders targets
    over 32 orbit views; a perturbed copy is fitted with torch Adam through the
    rasterizer's autograd functions (L1 + gamma entropy, gamma = 0.015), with
    the scale reset (zeta = 0.2) every 500 iterations.  Logs loss, PSNR and the
    mean per-tile list length."""
    import torch
    from paper_2603_09277_gb300 import gs, scenes
    from paper_2603_09277_gb300.rasterize import (Rasterizer, l1_entropy_loss, rasterize,
                                                  scene_to_device)
    W, H = (int(x) for x in args.train_size.split("x"))
    n = args.train_n
    gt_scene, _, _, prm = scenes.config5(seed=2, n=n, width=W, height=H)
    cams = scenes.orbit_cameras(32, W, H, seed=3)
    gt = scene_to_device(gt_scene, dev)
    # targets rendered from the ground-truth set
    targets = []
    for c in cams:
        rr = Rasterizer([c], prm, n, device=dev)
        rr.preprocess(gt)
        rr.bin_sort()
        rr.render_fwd()
        targets.append(rr.image.clone())
        del rr
    torch.cuda.empty_cache()
    rng = np.random.default_rng(4)
    init = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in gt_scene.items()}
    init["means"] = (init["means"] + rng.normal(0, 0.01, init["means"].shape)).astype(np.float32)
    init["log_scales"] = (init["log_scales"] + rng.normal(0, 0.1, init["log_scales"].shape)).astype(np.float32)
    init["opacity_logits"] = (init["opacity_logits"] + rng.normal(0, 0.5, n)).astype(np.float32)
    init["sh"][:, 0] = (init["sh"][:, 0] + rng.normal(0, 0.05, (n, 3))).astype(np.float32)
    p = scene_to_device(init, dev, requires_grad=True)
    params = [p[k] for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    opt = torch.optim.Adam([
        {"params": [p["means"]], "lr": 1.6e-4},
        {"params": [p["log_scales"]], "lr": 5e-3},
        {"params": [p["quats"]], "lr": 1e-3},
        {"params": [p["opacity_logits"]], "lr": 5e-2},
        {"params": [p["sh"]], "lr": 2.5e-3},
    ], eps=1e-15)
    rasts = [Rasterizer([c], prm, n, device=dev) for c in cams[:1]]
    r = rasts[0]
    t0 = time.perf_counter()
    order = np.random.default_rng(5).integers(0, len(cams), args.train)
    for it in range(1, args.train + 1):
        v = int(order[it - 1])
        r.cams = [cams[v]]
        r.cams_c = gs.make_cameras([cams[v]])
        img, ent = rasterize(p, r)
        loss = l1_entropy_loss(img, ent, targets[v], r, scenes.GAMMA)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        with torch.no_grad():
            p["quats"].div_(p["quats"].norm(dim=1, keepdim=True).clamp_min(1e-8))
        if it % 500 == 0:
            gs.gs_scale_reset(p["log_scales"].data, 0.2)
        if it % 100 == 0 or it == 1:
            with torch.no_grad():
                mse = float(((img - targets[v]) ** 2).mean().item())
            print(json.dumps({"train_iter": it, "loss": float(loss.item()),
                              "psnr": -10.0 * math.log10(max(mse, 1e-12)),
                              "pairs": r.num_pairs, "mean_list_per_tile": r.num_pairs / r.total_tiles,
                              "seconds": time.perf_counter() - t0}), flush=True)


def run_train_schedule(args, dev):
    """The training schedule of Sec. 5.2 on the cfg5 training scene: epochs of
    --images-per-epoch images sampled with replacement from 32 orbit views,
    the resolution scheduler (r_max: the largest factor <= 4 whose mean
    per-tile list stays <= 150, measured on the lists themselves; levels
    r_max .. 2 over the first half of the epochs, then full resolution), the
    scale reset every --reset-every epochs and the entropy term on every other
    epoch, with weaker zeta / gamma during the coarse stages.  One JSON line per
    epoch: level, gamma, zeta applied, loss, PSNR at the level, mean list per
    tile, milliseconds per iteration."""
    import torch
    from paper_2603_09277_gb300 import gs, scenes, schedule
    from paper_2603_09277_gb300.rasterize import (Rasterizer, l1_entropy_loss, rasterize,
                                                  scene_to_device)
    W, H = (int(x) for x in args.train_size.split("x"))
    n = args.train_n
    gt_scene, _, _, prm = scenes.config5(seed=2, n=n, width=W, height=H)
    prm["tile"] = args.tile
    cams = scenes.orbit_cameras(32, W, H, seed=3)
    gt = scene_to_device(gt_scene, dev)
    targets = []
    for c in cams:
        rr = Rasterizer([c], prm, n, device=dev)
        rr.preprocess(gt)
        rr.bin_sort()
        rr.render_fwd()
        targets.append(rr.image.reshape(H, W, 3).clone())
        del rr
    torch.cuda.empty_cache()
    rng = np.random.default_rng(4)
    init = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v
            for k, v in gt_scene.items()}
    init["means"] = (init["means"] + rng.normal(0, 0.01, init["means"].shape)).astype(np.float32)
    init["log_scales"] = (init["log_scales"]
                          + rng.normal(0, 0.1, init["log_scales"].shape)).astype(np.float32)
    init["opacity_logits"] = (init["opacity_logits"] + rng.normal(0, 0.5, n)).astype(np.float32)
    init["sh"][:, 0] = (init["sh"][:, 0] + rng.normal(0, 0.05, (n, 3))).astype(np.float32)
    p = scene_to_device(init, dev, requires_grad=True)
    opt = torch.optim.Adam([
        {"params": [p["means"]], "lr": 1.6e-4},
        {"params": [p["log_scales"]], "lr": 5e-3},
        {"params": [p["quats"]], "lr": 1e-3},
        {"params": [p["opacity_logits"]], "lr": 5e-2},
        {"params": [p["sh"]], "lr": 2.5e-3},
    ], eps=1e-15)

    def mean_list(r):
        # mean per-tile list length of the initial scene at factor r, over 4 views
        tot = 0.0
        for v in range(0, 32, 8):
            rr = Rasterizer([schedule.scaled_camera(cams[v], r)], prm, n, device=dev)
            rr.preprocess(p)
            P = rr.bin_sort()
            tot += P / rr.total_tiles
            del rr
        return tot / 4

    probes = {}
    r_max = schedule.choose_r_max(lambda r: probes.setdefault(r, mean_list(r)))
    plan = schedule.EpochSchedule(epochs=args.train_epochs, images_per_epoch=args.images_per_epoch,
                                  reset_every=args.reset_every, r_max=r_max)
    print(json.dumps({"r_max": r_max, "mean_list_probes": probes,
                      "threshold": schedule.LIST_THRESHOLD}), flush=True)
    levels = plan.levels()
    order = plan.image_order(len(cams), seed=5)
    rasts, tcache = {}, {}
    t0 = time.perf_counter()
    for e in range(plan.epochs):
        lv = int(levels[e])
        if lv not in rasts:
            rasts[lv] = Rasterizer([schedule.scaled_camera(cams[0], lv)], prm, n, device=dev)
        r = rasts[lv]
        gamma = plan.gamma_at(e)
        te = time.perf_counter()
        lsum, msum = 0.0, 0.0
        for it in range(plan.images_per_epoch):
            v = int(order[e, it])
            cam = schedule.scaled_camera(cams[v], lv)
            r.cams = [cam]
            r.cams_c = gs.make_cameras([cam])
            key = (v, lv)
            if key not in tcache:
                tcache[key] = schedule.downsample_image(targets[v], lv).reshape(-1, 3).contiguous()
            tgt = tcache[key]
            img, ent = rasterize(p, r)
            loss = l1_entropy_loss(img, ent, tgt, r, gamma)
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            with torch.no_grad():
                p["quats"].div_(p["quats"].norm(dim=1, keepdim=True).clamp_min(1e-8))
                if it == plan.images_per_epoch - 1:
                    lsum = float(loss.item())
                    msum = float(((img - tgt) ** 2).mean().item())
        torch.cuda.synchronize()
        ms_it = 1000.0 * (time.perf_counter() - te) / plan.images_per_epoch
        zeta = None
        if plan.reset_after(e):
            zeta = plan.zeta_at(e)
            gs.gs_scale_reset(p["log_scales"].data, zeta)
        print(json.dumps({"epoch": e, "r": lv, "gamma": gamma, "scale_reset": zeta,
                          "loss": lsum, "psnr": -10.0 * math.log10(max(msum, 1e-12)),
                          "mean_list_per_tile": r.num_pairs / r.total_tiles,
                          "ms_per_iter": ms_it, "seconds": time.perf_counter() - t0}),
              flush=True)


def time_variant(make, p, tgt, gamma, flush, steps, warmup=2):
    """Mean ms per fwd+bwd step (projection .. adjoint) of the rasterizers
    `make()` returns (run back to back: one per view for the per-view form),
    each step captured once in a CUDA graph and replayed (the headline's
    timed form), L2 flushed before every replay.  Returns (ms, the first
    rasterizer, which holds view 0's forward outputs of the last step)."""
    import torch
    rs = make()

    def one(sync):
        for r in rs:
            r.preprocess(p)
            r.bin_sort(sync=sync)
            r.render_fwd()
            r.loss(tgt[r], gamma) if isinstance(tgt, dict) else r.loss(tgt, gamma)
            r.render_bwd(p)

    for _ in range(warmup):
        one(True)  # sizes the pair buffers
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            one(False)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    if any(int(r.status_dev.item()) != 0 for r in rs):
        raise RuntimeError("pair capacity overflow in a variant")
    out = float(np.mean(ms))
    del g
    return out, rs


def super_tile_items(r, cams, tile):
    """Items (visible row x 8x8-tile super-tile its rect meets) of the list
    construction, from the projection's rects on the device."""
    import torch
    if r.rect is None:  # the 8-bit packed rects x0 | y0 << 8 | x1 << 16 | y1 << 24
        p8 = r.rect8[:r.rows].long() & 0xFFFFFFFF
        rect = torch.stack([(p8 >> s) & 255 for s in (0, 8, 16, 24)], 1).view(r.V, r.N, 4)
    else:
        rect = r.rect[:r.rows].long().view(r.V, r.N, 4)
    tot = 0
    for v, c in enumerate(cams):
        TX = (c["width"] + tile - 1) // tile
        TY = (c["height"] + tile - 1) // tile
        rr = rect[v]
        x0, y0 = rr[:, 0].clamp(min=0), rr[:, 1].clamp(min=0)
        x1, y1 = rr[:, 2].clamp(max=TX), rr[:, 3].clamp(max=TY)
        ok = (x1 > x0) & (y1 > y0) & (r.tiles_touched[v * r.N:(v + 1) * r.N] > 0)
        q = ((torch.div(x1 - 1, 8, rounding_mode="floor") - torch.div(x0, 8, rounding_mode="floor")
              + 1) * (torch.div(y1 - 1, 8, rounding_mode="floor")
                      - torch.div(y0, 8, rounding_mode="floor") + 1))
        tot += int(torch.where(ok, q, torch.zeros_like(q)).sum().item())
    return tot


def sm_count(dev):
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def fp32_peak_tflops(dev, clocks):
    """FP32 peak of the device: SMs x 128 FP32 lanes x 2 flop x the largest
    SM clock seen (the sampled maximum, else the measured peaks file's, else
    2070 MHz).  Returns (TFLOP/s, description)."""
    mhz = None
    if clocks and clocks.get("sm_max_mhz"):
        mhz, src = float(clocks["sm_max_mhz"]), "sampled max SM clock"
    else:
        try:
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
            src = "measured peaks file's max SM clock"
        except (OSError, ValueError, KeyError):
            mhz, src = 2070.0, "2070 MHz (nominal max SM clock)"
    sms = sm_count(dev)
    return (sms * 128 * 2 * mhz * 1e6 / 1e12,
            "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s)" % (sms, mhz, src))


def rank_totals(t_local, units_local, world, dev):
    """Whole-job figures of a replicated run: the time is the slowest rank's
    (max over ranks) and the work the sum over ranks; with one rank, the
    local values.  Returns (seconds, units)."""
    if world <= 1:
        return float(t_local), float(units_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units_local)], device=dev, dtype=torch.float64)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def measured_hbm_peak():
    """(GB/s, source) of the measured STREAM-style copy on the GB300s,
    else the stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def phase_graph_ms(fns, flush, reps=20):
    """Median time of each phase replayed alone from its own CUDA graph (L2
    flushed before every replay): without the eager launch gaps."""
    import torch
    out = {}
    s = torch.cuda.Stream()
    for name, fn in fns.items():
        g = torch.cuda.CUDAGraph()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
            with torch.cuda.graph(g, stream=s):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for k in range(reps):
            flush.fill_(float(k))
            a.record()
            g.replay()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = float(np.median(ts))
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2603_09277_gb300 import gs, scenes
    from paper_2603_09277_gb300.rasterize import (Rasterizer, capture_step, scene_to_device,
                                                   sh_layout_for, sh_to_layout, targets_to_device)

    if args.sweep:
        run_sweep(args, dev)
        return
    if args.train:
        run_train(args, dev)
        return
    if args.train_epochs:
        run_train_schedule(args, dev)
        return

    (scene, cams, targets, prm), wl = workload(args.config, rank, args.n)
    prm["tile"] = args.tile
    if args.tile != 16:
        wl += ", %dx%d tiles" % (args.tile, args.tile)
    if args.dssim > 0:
        wl += ", L_base with D-SSIM (lambda %.2f)" % args.dssim
    N = scene["means"].shape[0]
    # the SH layout for the degree in use: each coefficient of all Gaussians
    # together where the degree reads fewer coefficients than are stored
    sh_layout = sh_layout_for(scene["sh_degree"], scene["sh"].shape[1])
    p = scene_to_device(scene, dev, sh_layout=sh_layout)
    tgt = targets_to_device(targets, dev)
    form = {"pixels_per_thread": args.ppt, "persistent": args.persistent, "batch": args.batch}
    tuned = None
    if not args.no_autotune:
        from paper_2603_09277_gb300 import autotune
        form, tuned = autotune.tune(cams, prm, p, tgt, scenes.GAMMA, attr_dtype=args.attr)
    r = Rasterizer(cams, prm, N, attr_dtype=args.attr, device=dev, **form)
    ls_work = p["log_scales"].clone()  # the scale reset writes a working copy
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    gamma = scenes.GAMMA

    def step(sync, ev=None):
        e = ev if ev is not None else [None] * 8
        if e[0] is not None:
            e[0].record()
        r.preprocess(p)
        if e[1] is not None:
            e[1].record()
        r.bin_sort(sync=sync)
        if e[2] is not None:
            e[2].record()
        r.render_fwd(stats=True, events=(e[5], e[6]) if e[5] is not None else None)
        r.loss(tgt, gamma, lam=args.dssim)
        if e[3] is not None:
            e[3].record()
        r.render_bwd(p, events=(e[7], e[4]) if e[7] is not None else None)
        gs.gs_scale_reset(ls_work, 0.2)

    # warm-up with host-synchronised pair counting (sizes the pair buffers)
    for _ in range(max(args.warmup, 3)):
        step(True)
    torch.cuda.synchronize()
    # workload statistics (outside the timed region)
    P = r.num_pairs
    nb_step = int(r.stats[0].item())
    ne_step = int(r.stats[1].item())
    bwd_eval = int(r.last_idx.sum().item())

    K = args.steps
    # (1) eager steps with CUDA events between the phases: the per-phase
    # breakdown and the live per-kernel durations of the blending kernels
    KE = min(K, 20)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(16)] for _ in range(KE)]
    for e in evs:  # materialise the event handles
        for x in e:
            x.record()
    torch.cuda.synchronize()
    for k in range(KE):
        flush.fill_(float(k))  # L2 flush between timed steps (outside the step events)
        e = evs[k]
        # live events around the kernels of the stages without a launch argument
        gs.gs_stage_events(gs.GS_STAGE_PROJECTION, e[10], e[11])
        gs.gs_stage_events(gs.GS_STAGE_EXPANSION, e[12], e[13])
        gs.gs_stage_events(gs.GS_STAGE_ADJOINT, e[14], e[15])
        e[0].record()
        r.preprocess(p)
        e[1].record()
        r.bin_sort(sync=False)
        e[2].record()
        r.render_fwd(stats=False, events=(e[5], e[6]))
        r.loss(tgt, gamma, lam=args.dssim)
        e[3].record()
        r.render_bwd(p, events=(e[7], e[8]))
        gs.gs_scale_reset(ls_work, 0.2)
        e[4].record()
    for st_ in (gs.GS_STAGE_PROJECTION, gs.GS_STAGE_EXPANSION, gs.GS_STAGE_ADJOINT):
        gs.gs_stage_events(st_, None, None)
    torch.cuda.synchronize()
    eager_ms = float(np.mean([e[0].elapsed_time(e[4]) for e in evs]))
    kernel_ms = {
        "render_fwd_kernel": float(np.mean([e[5].elapsed_time(e[6]) for e in evs])),
        "render_bwd_kernel": float(np.mean([e[7].elapsed_time(e[8]) for e in evs])),
        "preprocess_kernel": float(np.mean([e[10].elapsed_time(e[11]) for e in evs])),
        "st_emit_kernel": float(np.mean([e[12].elapsed_time(e[13]) for e in evs])),
        "preprocess_bwd_kernel": float(np.mean([e[14].elapsed_time(e[15]) for e in evs])),
    }
    phase = {
        "preprocess": float(np.mean([e[0].elapsed_time(e[1]) for e in evs])),
        "bin_sort": float(np.mean([e[1].elapsed_time(e[2]) for e in evs])),
        "render_fwd_kernel": float(np.mean([e[5].elapsed_time(e[6]) for e in evs])),
        "render_fwd+loss": float(np.mean([e[2].elapsed_time(e[3]) for e in evs])),
        "render_bwd_kernel": float(np.mean([e[7].elapsed_time(e[8]) for e in evs])),
        "render_bwd+preprocess_bwd+reset": float(np.mean([e[3].elapsed_time(e[4]) for e in evs])),
    }

    # (2) the timed region: the whole step captured once in a CUDA graph (no
    # host synchronisation inside a step: the pair count stays on the device
    # and overflow is checked after the run) and replayed K times
    graph = torch.cuda.CUDAGraph()
    cap_stream = torch.cuda.Stream()
    cap_stream.wait_stream(torch.cuda.current_stream())
    launches_c0 = gs.gs_kernel_launches()
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream):
            r.preprocess(p)
            r.bin_sort(sync=False)
            r.render_fwd()
            r.loss(tgt, gamma, lam=args.dssim)
            r.render_bwd(p)
            gs.gs_scale_reset(ls_work, 0.2)
    torch.cuda.current_stream().wait_stream(cap_stream)
    kernels_per_step = gs.gs_kernel_launches() - launches_c0
    graph.replay()
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(float(k))  # L2 flush between timed steps (outside the step events)
        gev[k][0].record()
        graph.replay()
        gev[k][1].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = kernels_per_step * K
    status = int(r.status_dev.item())
    if status != 0:
        raise RuntimeError("pair capacity overflow in the timed region (status %d)" % status)
    # view-0 outputs of the timed form, for its error against the oracle
    n0 = cams[0]["width"] * cams[0]["height"]
    main_out = (r.image[:n0].clone(), r.final_T[:n0].clone(), r.entropy[:n0].clone())
    step_ms = [a.elapsed_time(b) for a, b in gev]
    t_total, nb_all = rank_totals(sum(step_ms) / 1000.0, nb_step, world, dev)
    value = nb_all * K / t_total
    ms = 1000.0 * t_total / K

    # roofline of the dominant kernel: of the kernels timed live, the one with
    # the longest launch; the blending kernels against the FP32 peak with the
    # FLOP model, the HBM-bound ones against the measured copy bandwidth with
    # their algorithmic bytes per launch
    peak, peak_src = fp32_peak_tflops(dev, clocks)
    hbm, hbm_src = measured_hbm_peak()
    vis_rows = (r.tiles_touched[:r.rows] > 0)
    n_rows_vis = int(vis_rows.sum().item())
    n_gauss_vis = int(vis_rows.view(r.V, r.N).any(0).sum().item())
    Kc = (int(prm.get("sh_degree", 0)) + 1) ** 2
    n_g = int(scene["means"].shape[0])
    rec_b = gs.gs_record_bytes(r.prm_c.attr_dtype)
    Q = super_tile_items(r, cams, args.tile)
    # the rect bytes of a row: the int4 rect of every row when it is written,
    # the 8-bit packed rect of every visible row when the views fit it
    r8 = all(-(-c["width"] // args.tile) <= 255 and -(-c["height"] // args.tile) <= 255
             for c in cams)
    rect_w = (r.rows * 16 if r.rect is not None else 0) + (n_rows_vis * 4 if r8 else 0)
    rect_r = n_rows_vis * 4 if r8 else r.rows * 16
    algo = {
        "render_fwd_kernel": ("alu", FWD_EVAL * ne_step + FWD_BLEND * nb_step),
        "render_bwd_kernel": ("alu", BWD_EVAL * bwd_eval + BWD_BLEND * nb_step),
        # every Gaussian's geometry and opacity, the SH in use of the seen
        # ones; depth and count of every row, its rects, the record of every
        # visible row
        "preprocess_kernel": ("hbm", n_g * 44 + n_gauss_vis * 12 * Kc + r.rows * 8 + rect_w +
                              n_rows_vis * rec_b),
        # the super-tile items (packed key, row) read, every pair written once
        "st_emit_kernel": ("hbm", Q * 8 + P * 4),
        # the moment row of every visible row; parameters read and gradients
        # written of every seen Gaussian
        "preprocess_bwd_kernel": ("hbm", n_rows_vis * 48 + n_gauss_vis * (44 + 12 * Kc) * 2),
    }
    kname = max(kernel_ms, key=kernel_ms.get)
    kms = kernel_ms[kname]
    bound, work = algo[kname]
    if bound == "alu":
        achieved = work / (kms / 1000.0) / 1e12
        roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": (traffic_from_profiles(kname, args.config)
                                if not args.n and args.tile == 16 and args.attr == "f32" else None),
                    "peak_source": peak_src, "flops_per_launch": work, "ms": kms}
    else:
        achieved = work / (kms / 1000.0) / 1e9
        roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm,
                    "traffic": (traffic_from_profiles(kname, args.config)
                                if not args.n and args.tile == 16 and args.attr == "f32" else None),
                    "peak_source": hbm_src, "bytes_per_launch": int(work), "ms": kms}
    kernels = {}
    for kn, kt in kernel_ms.items():
        bd, wk = algo[kn]
        if bd == "alu":
            ach = wk / (kt / 1000.0) / 1e12
            kernels[kn] = {"ms": kt, "bound": "alu", "achieved_tflops": ach, "frac": ach / peak}
        else:
            ach = wk / (kt / 1000.0) / 1e9
            kernels[kn] = {"ms": kt, "bound": "hbm", "achieved_gbs": ach, "frac": ach / hbm,
                           "bytes": int(wk)}
        kernels[kn]["traffic"] = (traffic_from_profiles(kn, args.config)
                                  if not args.n and args.tile == 16 and args.attr == "f32"
                                  else None)

    # per-phase times replayed alone from graphs, and the rooflines of the
    # phases other than the dominant kernel: HBM phases against the measured
    # copy bandwidth with their minimal algorithmic bytes (what the step must
    # move: the projection reads every Gaussian's geometry, the SH in use of
    # the visible rows, writes depth, rect and count of every row and the
    # record of every visible row; the lists read those per-row outputs and
    # write the pair values and ranges; the loss reads colour, target and
    # entropy and writes both gradients), the forward blending against the
    # FP32 peak with its FLOP model
    pg = {} if args.no_phase_graphs else phase_graph_ms({
        "preprocess": lambda: r.preprocess(p),
        "bin_sort": lambda: r.bin_sort(sync=False),
        "render_fwd": lambda: r.render_fwd(),
        "loss": lambda: r.loss(tgt, gamma, lam=args.dssim),
        "render_bwd+preprocess_bwd": lambda: r.render_bwd(p),
    }, flush)
    if not pg:  # fall back on the eager phase events
        pg = {"preprocess": phase["preprocess"], "bin_sort": phase["bin_sort"],
              "render_fwd": phase["render_fwd_kernel"],
              "loss": phase["render_fwd+loss"] - phase["render_fwd_kernel"]}
    n_pix = int(r.image.shape[0])
    bytes_pre = (n_g * 44 + n_gauss_vis * 12 * Kc + r.rows * 8 + rect_w +
                 n_rows_vis * gs.gs_record_bytes(r.prm_c.attr_dtype))
    bytes_bin = r.rows * 8 + rect_r + P * 4 + r.total_tiles * 8
    bytes_loss = n_pix * 44

    def hbm_line(nbytes, ms_):
        gbs = nbytes / (ms_ / 1000.0) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "peak_source": hbm_src, "bytes": int(nbytes), "ms": ms_}

    fwd_tf = (FWD_EVAL * ne_step + FWD_BLEND * nb_step) / (pg["render_fwd"] / 1000.0) / 1e12
    phase_roofline = {
        "preprocess": hbm_line(bytes_pre, pg["preprocess"]),
        "bin_sort": hbm_line(bytes_bin, pg["bin_sort"]),
        "render_fwd": {"bound": "alu", "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s",
                       "frac": fwd_tf / peak, "ms": pg["render_fwd"]},
        # with D-SSIM: the L1/entropy pass, then the SSIM forward (colour and
        # target in, five maps per channel out) and backward (maps, colour
        # and target in, dL/dC read and written)
        "loss": hbm_line(bytes_loss if args.dssim == 0 else n_pix * (44 + 84 + 108),
                         pg["loss"]),
    }

    # end to end through the C ABI with host buffers.  Per step the step's
    # inputs, the target images of its views, come in from pinned host
    # memory and the loss goes out; the Gaussian parameters are model state
    # and stay resident on the device, as in training.  A second, stricter
    # measurement also uploads every parameter each step.
    e2e = None
    e2e_full = None
    e2e_eager = None
    if not args.no_e2e:
        host = {k: torch.as_tensor(np.ascontiguousarray(
                    sh_to_layout(scene[k], p["sh_layout"]) if k == "sh" else scene[k]),
                    dtype=torch.float32).contiguous().pin_memory()
                for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        host_tgt = torch.cat([torch.as_tensor(t).reshape(-1, 3) for t in targets]).pin_memory()
        out_loss = torch.empty(1, dtype=torch.float64).pin_memory()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the parameter upload runs on three copy streams (the SH block in two
        # halves, the rest), joined before the step
        copy_streams = [torch.cuda.Stream(device=dev) for _ in range(3)]
        geo = [(p[kk], host[kk]) for kk in ("means", "log_scales", "quats", "opacity_logits")]
        k_used = (int(scene["sh_degree"]) + 1) ** 2
        late_plan = []
        if p["sh_layout"] == 1 and k_used < host["sh"].shape[0]:
            # coefficient-major SH: the step reads only the coefficients of
            # the degree in use; the others are copied beside the step (on
            # their own stream, joined before the step ends)
            copy_plan = [[(p["sh"][:k_used], host["sh"][:k_used])], geo, []]
            late_plan = [(p["sh"][k_used:], host["sh"][k_used:])]
        else:
            nh = host["sh"].shape[0] // 2
            copy_plan = [[(p["sh"][:nh], host["sh"][:nh])], [(p["sh"][nh:], host["sh"][nh:])], geo]
        late_stream = torch.cuda.Stream(device=dev)

        def e2e_body(upload_params):
            cur = torch.cuda.current_stream()
            if upload_params:
                if late_plan:
                    late_stream.wait_stream(cur)
                    with torch.cuda.stream(late_stream):
                        for dst, src in late_plan:
                            dst.copy_(src, non_blocking=True)
                for cs, plan in zip(copy_streams, copy_plan):
                    cs.wait_stream(cur)
                    with torch.cuda.stream(cs):
                        for dst, src in plan:
                            dst.copy_(src, non_blocking=True)
                for cs in copy_streams:
                    cur.wait_stream(cs)
            # the targets are first read by the loss: their copy runs on a
            # copy stream beside the projection and the list construction
            r.upload_target_async(host_tgt, tgt)
            r.preprocess(p)
            r.bin_sort(sync=False)
            r.render_fwd()
            r.loss(tgt, gamma, lam=args.dssim)
            r.render_bwd(p)
            gs.gs_scale_reset(ls_work, 0.2)
            out_loss.copy_(r.loss_dev, non_blocking=True)
            if upload_params and late_plan:
                cur.wait_stream(late_stream)

        def run_e2e(upload_params, graph=True):
            """Every step: the copies in from pinned host memory, the step and
            the loss read back; with graph, all of it captured once in a CUDA
            graph (copies included) and replayed per step, as a training loop
            on this library runs it; otherwise the calls issued eagerly."""
            step = lambda: e2e_body(upload_params)
            gr = None
            if graph:
                gr = capture_step(step, dev)
                step = gr.replay
            ms = []
            for k in range(K + 1):
                flush.fill_(float(k))
                a.record()
                step()
                b.record()
                b.synchronize()
                if k > 0:
                    ms.append(a.elapsed_time(b))
            if int(r.status_dev.item()) != 0:
                raise RuntimeError("pair capacity overflow in the end-to-end step")
            del gr
            t, _ = rank_totals(sum(ms) / 1000.0, 0, world, dev)
            h2d = host_tgt.numel() * 4 + (sum(v.numel() * 4 for v in host.values())
                                          if upload_params else 0)
            return {"value": nb_all * K / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(out_loss.numel() * 8), "ms_per_step": 1000.0 * t / K,
                    "form": "CUDA graph replay" if graph else "eager calls"}

        e2e = run_e2e(False)
        e2e_full = run_e2e(True)
        e2e_eager = run_e2e(False, graph=False)

    # the FP64 oracle on view 0 (the CPU baseline); its view-0 outputs are
    # also the reference for the error each form below states
    cpu, ref = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        nb_c, dt_c, desc, ref = oracle_sample(scene, cams, targets, prm, gamma,
                                              args.cpu_band_rows, keep=True)
        cpu = {"value": nb_c / dt_c, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle", "sample": desc, "seconds": dt_c}
    main_err = view0_error(ref, *main_out) if ref is not None else None

    # launch forms and staging precisions on the same workload ("batched +
    # mixed vs plain"): fwd+bwd ms per step (graph replay, no scale reset, L2
    # flushed), each with its error against the FP64 oracle on view 0
    variants = None
    if world == 1 and not args.no_variants:
        KV = max(5, min(20, K))
        variants = {}
        V = len(cams)
        pers = 8 * sm_count(dev)
        forms = []
        if V > 1:
            # the plain, unbatched form: one single-view FP32 pipeline per
            # view, back to back (each call of the per-view adjoint overwrites
            # the gradients; a training step would add them up)
            offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])

            def per_view():
                return [Rasterizer([c], prm, N, device=dev) for c in cams]
            forms.append(("per_view_f32", per_view, "views"))
        # the one-pipeline forms (all views in each launch: batched when V > 1)
        pre = "batched" if V > 1 else "plain"
        forms += [(pre + "_f32", dict(form), None),
                  (pre + "_f16", dict(form, attr_dtype="f16"), None),
                  (pre + "_bf16", dict(form, attr_dtype="bf16"), None),
                  ("persistent_f32", dict(form, persistent=pers), None),
                  ("ordered_f32", dict(form, persistent=0, ordered=True), None),
                  ("persistent_bf16", dict(form, persistent=pers, attr_dtype="bf16"), None),
                  (pre + "_f32_1px", dict(form, pixels_per_thread=1), None)]
        if args.tile == 16:
            forms += [(pre + "_f32_4px", dict(form, pixels_per_thread=4), None)]
            if form.get("batch", 256) != 128:
                forms += [(pre + "_f32_batch128", dict(form, batch=128), None)]
        for name, kw, kind in forms:
            if kind == "views":
                rs_probe = kw()
                tg = {rr: tgt[offs[v]:offs[v + 1]] for v, rr in enumerate(rs_probe)}
                ms_v, rs = time_variant(lambda: rs_probe, p, tg, gamma, flush, KV)
            else:
                if kw.get("attr_dtype", "f32") != "f32" and kw.get("batch") == 128:
                    kw = dict(kw, batch=256)  # the 128-entry batch exists for F32 records
                ms_v, rs = time_variant(
                    lambda kw=kw: [Rasterizer(cams, prm, N, device=dev, pair_capacity=r.capacity,
                                              **kw)], p, tgt, gamma, flush, KV)
            ent = {"ms_per_step": ms_v, "value": nb_all / (ms_v / 1000.0)}
            if ref is not None:
                ent["err_vs_oracle_view0"] = view0_error(ref, rs[0].image, rs[0].final_T,
                                                         rs[0].entropy)
            variants[name] = ent
            del rs
            torch.cuda.empty_cache()

    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.attr, "data": "synthetic",
            "config": {"workload": wl, "N": N, "views": len(cams), "pairs": P,
                       "blended_pairs": nb_step, "evaluated_pairs": ne_step,
                       "bwd_evaluated_pairs": bwd_eval, "attr_dtype": args.attr,
                       "sh_layout": ("[stride][N][3] (each coefficient of all Gaussians together)"
                                     if sh_layout else "[N][stride][3]"),
                       "tile": args.tile,
                       "launch": ("persistent %d CTAs over the list-length queue"
                                  % form["persistent"] if form["persistent"]
                                  else "one CTA per %dx%d tile" % (args.tile, args.tile)
                                  + (", longest list first" if form.get("ordered") else ""))
                       + ", %d px/thread, %d-entry batches" % (form["pixels_per_thread"] or 2,
                                                               form.get("batch") or 256),
                       "autotune_ms": tuned,
                       "l2": "flushed (256 MB write) before every timed step",
                       "timed_form": "whole step captured in one CUDA graph, replayed",
                       "eager_ms_per_step": eager_ms,
                       "kernels_per_step": kernels_per_step,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "phases_ms": phase,
            "phases_graph_ms": pg,
            "phase_roofline": phase_roofline,
            "error_vs_oracle_view0": main_err,
            "exclusions_view0": ref["exclusions"] if ref is not None else None,
            "variants": variants,
            "roofline": roofline,
            "kernels": kernels,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_params_uploaded": e2e_full,
            "e2e_eager": e2e_eager,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
