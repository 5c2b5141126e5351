"""Launch-form autotuner for the blending kernels.

Times the candidate launch forms (pixels per thread 1/2/4, list entries per
shared-memory batch 128/256, one CTA per tile in tile order or longest list
first, or a persistent grid of 4 or 8 CTAs per SM over the list-length-ordered
tile queue) on the caller's
actual workload (a few whole fwd+bwd steps each, L2 flushed between steps),
and caches the fastest form per workload signature (views and their sizes,
Gaussian count, staging dtype, device name) in a JSON file under
paper_2603_09277_gb300/_build/.
"""
from __future__ import annotations

import json
import os
import time

import torch

from .rasterize import Rasterizer

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
# per-tile forms; the persistent forms are added with grids of 8 and 4 CTAs
# per SM of the device in use
BASE_CANDIDATES = [
    {"pixels_per_thread": 1, "persistent": 0, "batch": 256},
    {"pixels_per_thread": 2, "persistent": 0, "batch": 256},
    {"pixels_per_thread": 4, "persistent": 0, "batch": 256},
    {"pixels_per_thread": 2, "persistent": 0, "batch": 128},
    {"pixels_per_thread": 4, "persistent": 0, "batch": 128},
    {"pixels_per_thread": 2, "persistent": 0, "batch": 256, "ordered": True},
]
PERSISTENT_PER_SM = [(2, 8), (4, 8), (2, 4)]  # (pixels per thread, CTAs per SM)


def sm_count():
    """Streaming multiprocessors of the current CUDA device (read at run time;
    152 on a GB300), the unit of the persistent grid sizes.  Without a device
    (host-side tests) the GB300 count."""
    if torch.cuda.is_available():
        return int(torch.cuda.get_device_properties(torch.cuda.current_device())
                   .multi_processor_count)
    return 152


def signature(cams, N, attr_dtype, tile=16):
    """Cache key: the views and their sizes, N, staging dtype, tile side, the
    candidate set and the device."""
    views = ",".join("%dx%d" % (c["width"], c["height"]) for c in cams)
    forms = ";".join(form_name(f) for f in candidates(tile, attr_dtype))
    return "%s|N=%d|%s|tile=%d|%s|%s" % (views, N, attr_dtype, tile, forms,
                                         torch.cuda.get_device_name())


def candidates(tile=16, attr_dtype="f32"):
    """Launch forms to try; 8-pixel tiles take 1 or 2 pixels per thread (a
    CTA of one tile must hold at least one full warp); the 128-entry batch
    exists for F32 records on 16-pixel tiles."""
    sms = sm_count()
    pool = BASE_CANDIDATES + [{"pixels_per_thread": ppt, "persistent": sms * k, "batch": 256}
                              for ppt, k in PERSISTENT_PER_SM]
    return [f for f in pool
            if (tile == 16 or f["pixels_per_thread"] <= 2)
            and (f["batch"] == 256 or (tile == 16 and attr_dtype == "f32"))]


def form_name(form):
    """e.g. "ppt2_b256_per_tile", "ppt2_b256_per_tile_ordered", "ppt4_b256_persistent1216"."""
    where = ("persistent%d" % form["persistent"] if form["persistent"] else
             "per_tile_ordered" if form.get("ordered") else "per_tile")
    return "ppt%d_b%d_%s" % (form["pixels_per_thread"], form.get("batch", 256), where)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, CACHE)


def time_form(cams, prm, params, target, gamma, form, attr_dtype="f32", steps=5, warmup=2):
    """Mean ms of a whole eager fwd+bwd step with the given launch form."""
    N = params["means"].shape[0]
    r = Rasterizer(cams, prm, N, attr_dtype=attr_dtype, **form)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=r.device)
    for _ in range(warmup):
        r.step(params, target, gamma, sync=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        a.record()
        r.step(params, target, gamma, sync=False)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    if int(r.status_dev.item()) != 0:
        raise RuntimeError("pair capacity overflow while tuning")
    return sum(ms) / len(ms)


def tune(cams, prm, params, target, gamma, attr_dtype="f32", force=False, steps=5):
    """Returns (best form dict, {form: ms}) and caches the choice."""
    tile = int(prm.get("tile", 16))
    key = signature(cams, params["means"].shape[0], attr_dtype, tile)
    db = _load()
    if not force and key in db:
        return db[key]["best"], db[key]["ms"]
    times = {}
    cands = candidates(tile, attr_dtype)
    for form in cands:
        times[form_name(form)] = time_form(cams, prm, params, target, gamma, form, attr_dtype,
                                           steps)
        torch.cuda.empty_cache()
    best = min(cands, key=lambda f: times[form_name(f)])
    db[key] = {"best": best, "ms": times, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    _store(db)
    return best, times
