"""Device-memory owner and autograd wrappers over the libgs C ABI.

``Rasterizer`` allocates every buffer the hot path needs (torch tensors used
as device memory) and calls the C entry points in order; each step of the
computation runs in libgs kernels.  ``rasterize`` / ``l1_entropy_loss`` are
torch.autograd.Function wrappers for training loops.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gs

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def sh_to_layout(sh, sh_layout):
    """[N][K][3] SH coefficients in the library's layout sh_layout: 0 keeps
    them, 1 gives [K][N][3] (each coefficient of all Gaussians together)."""
    return sh if sh_layout == 0 else sh.transpose(1, 0, 2) if isinstance(sh, np.ndarray) \
        else sh.transpose(0, 1)


def sh_layout_for(sh_degree, sh_stride):
    """The faster SH layout for a degree in use: 1 (each coefficient of all
    Gaussians together) when it reads fewer coefficients than are stored, so
    that its loads stay contiguous instead of picking a few floats out of
    every Gaussian's block; 0 when it reads them all (16-byte loads of each
    Gaussian's block)."""
    return 1 if (int(sh_degree) + 1) ** 2 < int(sh_stride) else 0


def scene_to_device(scene, device="cuda", requires_grad=False, sh_layout=0):
    """numpy scene dict -> dict of contiguous float32 CUDA tensors; the SH
    coefficients in layout sh_layout (recorded as "sh_layout")."""
    out = {}
    for k in PARAM_KEYS:
        a = sh_to_layout(scene[k], sh_layout) if k == "sh" else scene[k]
        t = torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).contiguous().to(device)
        out[k] = t.requires_grad_(requires_grad) if requires_grad else t
    out["sh_degree"] = int(scene["sh_degree"])
    out["sh_layout"] = int(sh_layout)
    return out


def targets_to_device(targets, device="cuda"):
    """List of [H,W,3] arrays -> one flat [sum HW, 3] float32 tensor."""
    return torch.cat([torch.as_tensor(t, dtype=torch.float32).reshape(-1, 3) for t in targets]).to(
        device).contiguous()


def capture_step(fn, device="cuda"):
    """Captures fn() -- a whole step of Rasterizer calls, copies from pinned
    host memory and the loss read-back included -- in a CUDA graph on a side
    stream and returns the graph; graph.replay() reruns the step with the
    buffers' current contents.  Run the step once eagerly first (the pair
    buffers are sized there, and the library's second stream is created
    outside a capture); list construction inside the graph keeps the pair
    count on the device (bin_sort(sync=False)): after a replay, a nonzero
    status_dev means the pair buffers overflowed."""
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(device=device)
    s.wait_stream(torch.cuda.current_stream(device))
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn()
    torch.cuda.current_stream(device).wait_stream(s)
    return g


class Rasterizer:
    """Buffers and calls for one fixed set of views and Gaussian count.

    cams: list of camera dicts; prm: threshold dict (see scenes.params);
    N: Gaussian count; attr_dtype: "f32" | "f16" | "bf16" record staging;
    persistent: 0 (one CTA per tile) or the CTA count of a persistent launch
    claiming tiles from a list-length-ordered queue (the batched form);
    ordered: with one CTA per tile, launch the tiles longest list first (the
    same queue as the block order);
    pixels_per_thread: 1, 2 or 4 (0 = the library default, 2);
    batch: list entries staged per shared-memory batch, 128 or 256 (0 = 256).
    """

    def __init__(self, cams, prm, N, sh_stride=16, attr_dtype="f32", device="cuda",
                 pair_capacity=None, persistent=0, keep_debug=False, pixels_per_thread=0,
                 batch=0, ordered=False):
        self.device = torch.device(device)
        self.cams = cams
        self.cams_c = gs.make_cameras(cams)
        self.prm = dict(prm)
        self.prm_c = gs.make_params(prm, sh_stride, attr_dtype)
        self.N = int(N)
        self.V = len(cams)
        self.sh_stride = sh_stride
        self.rows = self.N * self.V
        self.tile = int(prm.get("tile", 16))
        self.total_tiles = gs.gs_total_tiles(self.cams_c, self.tile)
        self.total_pixels = gs.gs_total_pixels(self.cams_c)
        if self.total_tiles < 0:
            raise ValueError("invalid cameras")
        dev = self.device
        i32 = dict(dtype=torch.int32, device=dev)
        f32 = dict(dtype=torch.float32, device=dev)
        rb = gs.gs_record_bytes(self.prm_c.attr_dtype)
        R = max(self.rows, 1)
        self.records = torch.empty(R * rb, dtype=torch.uint8, device=dev)
        self.depth = torch.empty(R, **f32)
        self.tiles_touched = torch.empty(R, **i32)
        self.rect8 = torch.empty(R, **i32)  # rects packed in 8-bit fields (small views)
        # with every view at most 255 tiles per side the packed rects carry
        # the list construction and the int4 rects are left out (16 bytes of
        # projection writes per row), unless the debug outputs are kept
        self.rect8_only = not keep_debug and all(
            -(-c["width"] // self.tile) <= 255 and -(-c["height"] // self.tile) <= 255
            for c in cams)
        self.rect = None if self.rect8_only else torch.empty(R, 4, **i32)
        self.keep_debug = keep_debug
        if keep_debug:
            self.radius = torch.empty(R, **i32)
            self.mean2d = torch.empty(R, 2, **f32)
            self.conic_opacity = torch.empty(R, 4, **f32)
            self.rgb = torch.empty(R, 3, **f32)
            self.proj_c = gs.make_proj(self.records, self.depth, self.rect, self.tiles_touched,
                                       self.radius, self.mean2d, self.conic_opacity, self.rgb,
                                       self.rect8)
        else:
            self.proj_c = gs.make_proj(self.records, self.depth, self.rect, self.tiles_touched,
                                       rect8=self.rect8)
        self.tile_ranges = torch.zeros(max(self.total_tiles, 1), 2, **i32)
        self.num_pairs_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status_dev = torch.zeros(1, **i32)
        self.capacity = 0
        self._alloc_pairs(pair_capacity if pair_capacity is not None else max(1 << 20, 8 * self.rows))
        P = max(self.total_pixels, 1)
        self.image = torch.empty(P, 3, **f32)
        self.final_T = torch.empty(P, **f32)
        self.last_idx = torch.empty(P, **i32)
        self.entropy = torch.empty(P, **f32)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        self.dL_dimage = torch.empty(P, 3, **f32)
        self.dL_dentropy = torch.empty(P, **f32)
        self.loss_ws = torch.empty(gs.gs_loss_workspace_size(P), dtype=torch.uint8, device=dev)
        self.grad2d = torch.empty(R, 12, **f32)
        self._grad2d_zero = False  # grad2d zeroed by the latest forward, not yet used
        self.grads = {
            "means": torch.empty(max(self.N, 1), 3, **f32),
            "log_scales": torch.empty(max(self.N, 1), 3, **f32),
            "quats": torch.empty(max(self.N, 1), 4, **f32),
            "opacity_logits": torch.empty(max(self.N, 1), **f32),
            "sh": torch.empty(max(self.N, 1), sh_stride, 3, **f32),
        }
        self._gsh = self.grads["sh"]  # its storage, viewed in the parameters' SH layout
        self.stats = torch.zeros(2, dtype=torch.int64, device=dev)
        self.persistent = int(persistent)
        self.ppt = int(pixels_per_thread)
        self.batch = int(batch)
        self.tile_order = None
        self.ordered = bool(ordered) and not self.persistent
        if self.persistent or self.ordered:
            self.tile_order = torch.empty(max(self.total_tiles, 1), **i32)
            self.work_counter = torch.zeros(1, **i32)
            self.queue_ws = torch.empty(gs.gs_tile_queue_workspace_size(self.total_tiles),
                                        dtype=torch.uint8, device=dev)
        self.num_pairs = None
        self.forward_count = 0  # forwards run through rasterize(); see _Rasterize

    def _launch(self, stats=False, events=None, zero_beside=None, grad2d_zeroed=False):
        ev = events if events is not None else (None, None)
        if self.persistent:
            return gs.make_launch(self.tile_order, self.work_counter, self.persistent,
                                  self.stats if stats else None, ev[0], ev[1], self.ppt,
                                  self.batch, zero_beside, grad2d_zeroed)
        return gs.make_launch(self.tile_order if self.ordered else None, None, 0,
                              self.stats if stats else None, ev[0], ev[1], self.ppt, self.batch,
                              zero_beside, grad2d_zeroed)

    def _alloc_pairs(self, cap):
        cap = int(min(max(cap, 1), (1 << 32) - 1))
        self.capacity = cap
        dev = self.device
        self.sorted_vals = torch.empty(cap, dtype=torch.int32, device=dev)
        ws = gs.gs_bin_sort_workspace_size(self.rows, cap, self.total_tiles)
        self.bin_ws = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.sorted_keys = None

    # -- steps -------------------------------------------------------------
    def _sh_layout(self, p):
        """Takes the SH layout of the parameters p (their "sh_layout", 0 when
        absent) for the calls and the SH gradient."""
        lay = int(p.get("sh_layout", 0)) if isinstance(p, dict) else 0
        if lay != self.prm_c.sh_layout:
            self.prm_c.sh_layout = lay
            self.grads["sh"] = (self._gsh if lay == 0 else
                                self._gsh.view(self.sh_stride, max(self.N, 1), 3))

    def preprocess(self, p, stream=None):
        self._sh_layout(p)
        gs.gs_preprocess(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                         self.N, self.cams_c, self.prm_c, self.proj_c, stream)

    def bin_sort(self, sync=True, keys=False, stream=None):
        """Builds the per-tile lists.  With sync, regrows the pair buffers on
        overflow and returns the pair count; without, returns None (graph form)."""
        if keys and (self.sorted_keys is None or self.sorted_keys.numel() < self.capacity):
            self.sorted_keys = torch.empty(self.capacity, dtype=torch.int64, device=self.device)
        while True:
            st, P = gs.gs_bin_sort(self.proj_c, self.N, self.cams_c, self.bin_ws, self.capacity,
                                   self.sorted_vals, self.sorted_keys if keys else None,
                                   self.tile_ranges, self.num_pairs_dev, self.status_dev,
                                   sync_count=sync, stream=stream, tile_size=self.tile)
            if st == gs.GS_OK:
                break
            self._alloc_pairs(int(P * 1.25) + 1024)
            if keys:
                self.sorted_keys = torch.empty(self.capacity, dtype=torch.int64, device=self.device)
        if P is not None:
            self.num_pairs = P
        if self.persistent or self.ordered:
            gs.gs_tile_queue(self.tile_ranges, self.total_tiles, self.tile_order, self.queue_ws,
                             stream)
        return P

    def render_fwd(self, stats=False, stream=None, events=None):
        """events: optional (begin, end) recorded torch.cuda.Events placed
        around the blending kernel."""
        if stats:
            self.stats.zero_()
        # the backward's grad2d is zeroed beside the forward kernel
        gs.gs_render_fwd(self.proj_c, self.N, self.cams_c, self.prm_c, self.sorted_vals,
                         self.tile_ranges, self.image, self.final_T, self.last_idx, self.entropy,
                         self._launch(stats, events, zero_beside=self.grad2d), stream)
        self._grad2d_zero = True

    def _base_ws(self):
        need = gs.gs_loss_base_workspace_size(self.cams_c)
        if getattr(self, "loss_base_ws", None) is None or self.loss_base_ws.numel() < need:
            self.loss_base_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self.loss_base_ws

    def upload_target_async(self, host_target, target, stream=None):
        """Starts the copy of a step's target images from pinned host memory
        into the device tensor `target` on a copy stream, ordered after the
        work already on `stream` (default: the current stream); the next
        loss() on that target waits for it.  The copy then runs beside the
        projection and the list construction, which do not read it."""
        cur = stream if stream is not None else torch.cuda.current_stream(self.device)
        if getattr(self, "_copy_stream", None) is None:
            self._copy_stream = torch.cuda.Stream(device=self.device)
            self._copy_done = torch.cuda.Event()
        self._copy_stream.wait_stream(cur)
        with torch.cuda.stream(self._copy_stream):
            target.copy_(host_target, non_blocking=True)
            self._copy_done.record(self._copy_stream)
        self._copy_pending = target

    def loss(self, target, gamma, stream=None, lam=0.0):
        """L1 + gamma * entropy, or with lam > 0 the full L_base
        (1 - lam) L1 + lam D-SSIM + gamma * entropy."""
        if getattr(self, "_copy_pending", None) is target:
            cur = stream if stream is not None else torch.cuda.current_stream(self.device)
            cur.wait_event(self._copy_done)
            self._copy_pending = None
        if lam > 0.0:
            gs.gs_loss_base(self.image, target, self.entropy, self.cams_c, lam, gamma,
                            self.loss_dev, self.dL_dimage, self.dL_dentropy, self._base_ws(),
                            stream)
        else:
            gs.gs_loss_l1_entropy(self.image, target, self.entropy, self.cams_c, gamma,
                                  self.loss_dev, self.dL_dimage, self.dL_dentropy, self.loss_ws,
                                  stream)
        return self.loss_dev

    def render_bwd(self, p, dL_dimage=None, dL_dentropy="auto", stream=None, events=None):
        dimg = self.dL_dimage if dL_dimage is None else dL_dimage
        dent = self.dL_dentropy if isinstance(dL_dentropy, str) else dL_dentropy
        self._sh_layout(p)
        g = self.grads
        gs.gs_render_bwd(self.proj_c, self.N, self.cams_c, self.prm_c, self.sorted_vals,
                         self.tile_ranges, self.final_T, self.last_idx, dimg, dent, p["means"],
                         p["log_scales"], p["quats"], p["opacity_logits"], p["sh"], self.grad2d,
                         g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"],
                         self._launch(False, events, grad2d_zeroed=self._grad2d_zero), stream)
        self._grad2d_zero = False  # a second backward of one forward zeroes it itself
        return g

    def grad2d_attributes(self, stream=None):
        """Per (view, Gaussian) row the 2D gradients of the latest backward:
        dL/d(mean2d x, y), dL/d(conic a, b, c), dL/dsigma, dL/d(r, g, b)
        [V*N, 9] (gs_grad2d_attributes)."""
        out = torch.empty(max(self.rows, 1), 9, dtype=torch.float32, device=self.device)
        gs.gs_grad2d_attributes(self.proj_c, self.N, self.V, self.prm_c, self.grad2d, out, stream)
        return out

    def step(self, p, target, gamma, sync=True, stream=None):
        """One forward + backward of L1 + gamma * entropy; returns the device loss."""
        self.preprocess(p, stream)
        self.bin_sort(sync=sync, stream=stream)
        self.render_fwd(stream=stream)
        self.loss(target, gamma, stream)
        self.render_bwd(p, stream=stream)
        return self.loss_dev

    # -- views of per-pixel outputs ------------------------------------------
    def view_slices(self):
        out, off = [], 0
        for c in self.cams:
            n = c["width"] * c["height"]
            out.append((off, off + n, c["height"], c["width"]))
            off += n
        return out

    def image_of(self, v):
        a, b, H, W = self.view_slices()[v]
        return self.image[a:b].reshape(H, W, 3)


class _Rasterize(torch.autograd.Function):
    """The backward reads the lists, final transmittances and last indices
    that the Rasterizer holds from its latest forward, so one Rasterizer
    serves one live graph at a time: a backward after a newer forward through
    the same Rasterizer raises instead of using the newer forward's state."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, rast, sh_layout):
        p = {"means": means.contiguous(), "log_scales": log_scales.contiguous(),
             "quats": quats.contiguous(), "opacity_logits": opacity_logits.contiguous(),
             "sh": sh.contiguous(), "sh_layout": sh_layout}
        rast.preprocess(p)
        rast.bin_sort()
        rast.render_fwd()
        rast.forward_count += 1
        ctx.rast = rast
        ctx.forward_id = rast.forward_count
        ctx.sh_layout = sh_layout
        ctx.save_for_backward(*[p[k] for k in PARAM_KEYS])
        return rast.image.clone(), rast.entropy.clone()

    @staticmethod
    def backward(ctx, g_image, g_entropy):
        rast = ctx.rast
        if rast.forward_count != ctx.forward_id:
            raise RuntimeError("rasterize: this Rasterizer ran another forward after the one being "
                               "differentiated; its saved lists belong to the newer call (use one "
                               "Rasterizer per live graph)")
        p = dict(zip(PARAM_KEYS, ctx.saved_tensors))
        p["sh_layout"] = ctx.sh_layout
        g_image = g_image.contiguous() if g_image is not None else torch.zeros_like(rast.image)
        g_entropy = g_entropy.contiguous() if g_entropy is not None else None
        g = rast.render_bwd(p, g_image, g_entropy)
        return (g["means"].clone(), g["log_scales"].clone(), g["quats"].clone(),
                g["opacity_logits"].clone(), g["sh"].clone(), None, None)


def rasterize(params, rast):
    """Differentiable render: returns (image [sum HW, 3], entropy [sum HW]).
    The SH coefficients are in params["sh_layout"] (0 when absent), their
    gradient in the same layout."""
    return _Rasterize.apply(params["means"], params["log_scales"], params["quats"],
                            params["opacity_logits"], params["sh"], rast,
                            int(params.get("sh_layout", 0)))


class _L1Entropy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, entropy, target, rast, gamma, lam):
        if lam > 0.0:
            gs.gs_loss_base(image.contiguous(), target, entropy.contiguous(), rast.cams_c, lam,
                            gamma, rast.loss_dev, rast.dL_dimage, rast.dL_dentropy,
                            rast._base_ws())
        else:
            gs.gs_loss_l1_entropy(image.contiguous(), target, entropy.contiguous(), rast.cams_c,
                                  gamma, rast.loss_dev, rast.dL_dimage, rast.dL_dentropy,
                                  rast.loss_ws)
        ctx.save_for_backward(rast.dL_dimage.clone(), rast.dL_dentropy.clone())
        return rast.loss_dev.clone().to(torch.float32).reshape(())

    @staticmethod
    def backward(ctx, g):
        di, de = ctx.saved_tensors
        return di * g, de * g, None, None, None, None


def l1_entropy_loss(image, entropy, target, rast, gamma, lam=0.0):
    """L = (1/V) sum_v [(1 - lam) mean L1_v + lam D-SSIM_v + gamma mean H_v],
    computed by libgs (lam = 0: L1 + entropy)."""
    return _L1Entropy.apply(image, entropy, target, rast, gamma, float(lam))
