"""ctypes binding of libgs (include/gs.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name, passing device pointers of torch tensors and the current
CUDA stream.  There is no Python or CPU implementation of any step; if
libgs.so has not been built this module raises on import.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CUDA = -2
GS_ERR_CAPACITY = -3
GS_ERR_TIMEOUT = -4
GS_ERR_UNSUPPORTED = -5

GS_ATTR_F32, GS_ATTR_F16, GS_ATTR_BF16 = 0, 1, 2
ATTR_DTYPES = {"f32": GS_ATTR_F32, "f16": GS_ATTR_F16, "bf16": GS_ATTR_BF16}
TILE = 16
MAX_VIEWS = 64


class GsCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("world_to_cam", ctypes.c_float * 12), ("cam_pos", ctypes.c_float * 3)]


class GsParams(ctypes.Structure):
    _fields_ = [("alpha_max", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("t_min", ctypes.c_float), ("dilation", ctypes.c_float),
                ("near_z", ctypes.c_float), ("fov_clamp", ctypes.c_float),
                ("sh_degree", ctypes.c_int), ("sh_stride", ctypes.c_int),
                ("attr_dtype", ctypes.c_int), ("tile_size", ctypes.c_int),
                ("sh_layout", ctypes.c_int)]


class GsProj(ctypes.Structure):
    _fields_ = [("records", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("rect", ctypes.c_void_p), ("tiles_touched", ctypes.c_void_p),
                ("radius", ctypes.c_void_p), ("mean2d", ctypes.c_void_p),
                ("conic_opacity", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("rect8", ctypes.c_void_p)]


class GsLaunch(ctypes.Structure):
    _fields_ = [("tile_order", ctypes.c_void_p), ("work_counter", ctypes.c_void_p),
                ("ctas", ctypes.c_int), ("stats", ctypes.c_void_p),
                ("ev_begin", ctypes.c_void_p), ("ev_end", ctypes.c_void_p),
                ("pixels_per_thread", ctypes.c_int), ("batch", ctypes.c_int),
                ("zero_beside", ctypes.c_void_p), ("zero_bytes", ctypes.c_ulonglong),
                ("grad2d_zeroed", ctypes.c_int)]


class GsError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        msg = "%s failed: %s (%d) %s" % (fn, _lib.gs_status_string(status).decode(), status,
                                         _lib.gs_last_error_string().decode())
        super().__init__(msg)


def _load():
    # GS_LIBRARY selects another build of the library (the bounds-checked one)
    path = os.environ.get("GS_LIBRARY") or _build.LIB
    if not os.path.exists(path):
        raise ImportError("libgs.so is not built (%s); run paper_2603_09277_gb300.build.build() "
                          "or __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i, ll, sz, f, d = (ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t,
                           ctypes.c_float, ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "gs_record_bytes": (i, [i]),
        "gs_total_tiles": (ll, [P(GsCamera), i, i]),
        "gs_total_pixels": (ll, [P(GsCamera), i]),
        "gs_bin_sort_workspace_size": (sz, [ll, ll, ll]),
        "gs_loss_workspace_size": (sz, [ll]),
        "gs_tile_queue_workspace_size": (sz, [ll]),
        "gs_status_string": (ctypes.c_char_p, [i]),
        "gs_last_error_string": (ctypes.c_char_p, []),
        "gs_version": (ctypes.c_char_p, []),
        "gs_kernel_launches": (ctypes.c_ulonglong, []),
        "gs_stage_events": (i, [i, vp, vp]),
        "gs_debug_bounds_status": (i, [P(ctypes.c_uint), i]),
        "gs_preprocess": (i, [vp, vp, vp, vp, vp, i, P(GsCamera), i, P(GsParams), P(GsProj), vp]),
        "gs_bin_sort": (i, [P(GsProj), i, P(GsCamera), i, i, vp, sz, ll, vp, vp, vp, vp, vp, vp,
                            vp]),
        "gs_render_fwd": (i, [P(GsProj), i, P(GsCamera), i, P(GsParams), vp, vp, vp, vp, vp, vp,
                              P(GsLaunch), vp]),
        "gs_loss_l1_entropy": (i, [vp, vp, vp, P(GsCamera), i, f, vp, vp, vp, vp, sz, vp]),
        "gs_loss_base_workspace_size": (sz, [P(GsCamera), i]),
        "gs_loss_base": (i, [vp, vp, vp, P(GsCamera), i, f, f, vp, vp, vp, vp, sz, vp]),
        "gs_render_bwd": (i, [P(GsProj), i, P(GsCamera), i, P(GsParams), vp, vp, vp, vp, vp, vp,
                              vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, P(GsLaunch), vp]),
        "gs_grad2d_attributes": (i, [P(GsProj), i, i, P(GsParams), vp, vp, vp]),
        "gs_scale_reset": (i, [vp, ll, f, vp]),
        "gs_tile_queue": (i, [vp, ll, vp, vp, sz, vp]),
        "gs_tile_queue_static": (i, [vp, ll, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ["gs_record_bytes", "gs_total_tiles", "gs_total_pixels", "gs_bin_sort_workspace_size",
            "gs_loss_workspace_size", "gs_tile_queue_workspace_size", "gs_status_string",
            "gs_last_error_string", "gs_version", "gs_kernel_launches", "gs_stage_events",
            "gs_debug_bounds_status",
            "gs_preprocess", "gs_bin_sort", "gs_render_fwd",
            "gs_loss_l1_entropy", "gs_loss_base_workspace_size", "gs_loss_base",
            "gs_render_bwd", "gs_grad2d_attributes", "gs_scale_reset", "gs_tile_queue",
            "gs_tile_queue_static"]


def library_path() -> str:
    return _build.LIB


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(fn, status):
    if status != GS_OK:
        raise GsError(fn, status)
    return status


# ---------------------------------------------------------------------------
# Host structs
# ---------------------------------------------------------------------------

def make_cameras(cams):
    """cams: list of dicts (width, height, fx, fy, cx, cy, world_to_cam [3,4],
    cam_pos [3]) -> ctypes array of GsCamera."""
    arr = (GsCamera * len(cams))()
    for k, c in enumerate(cams):
        g = arr[k]
        g.width, g.height = int(c["width"]), int(c["height"])
        g.fx, g.fy, g.cx, g.cy = float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"])
        w = [float(x) for x in __import__("numpy").asarray(c["world_to_cam"]).reshape(12)]
        for j in range(12):
            g.world_to_cam[j] = w[j]
        p = [float(x) for x in __import__("numpy").asarray(c["cam_pos"]).reshape(3)]
        for j in range(3):
            g.cam_pos[j] = p[j]
    return arr


def make_params(prm, sh_stride=16, attr_dtype="f32", sh_layout=0):
    p = GsParams()
    p.alpha_max, p.alpha_min, p.t_min = prm["alpha_max"], prm["alpha_min"], prm["t_min"]
    p.dilation, p.near_z, p.fov_clamp = prm["dilation"], prm["near_z"], prm["fov_clamp"]
    p.sh_degree = int(prm.get("sh_degree", 0))
    p.sh_stride = int(sh_stride)
    p.attr_dtype = ATTR_DTYPES[attr_dtype] if isinstance(attr_dtype, str) else int(attr_dtype)
    p.tile_size = int(prm.get("tile", 16))
    p.sh_layout = int(sh_layout)
    return p


def make_proj(records, depth, rect, tiles_touched, radius=None, mean2d=None, conic_opacity=None,
              rgb=None, rect8=None):
    return GsProj(_ptr(records), _ptr(depth), _ptr(rect), _ptr(tiles_touched), _ptr(radius),
                  _ptr(mean2d), _ptr(conic_opacity), _ptr(rgb), _ptr(rect8))


def make_launch(tile_order=None, work_counter=None, ctas=0, stats=None, ev_begin=None,
                ev_end=None, pixels_per_thread=0, batch=0, zero_beside=None, grad2d_zeroed=False):
    """ev_begin / ev_end: recorded torch.cuda.Event objects (or None);
    zero_beside: a device tensor the forward zeroes beside its kernel."""
    zb = 0 if zero_beside is None else zero_beside.numel() * zero_beside.element_size()
    return GsLaunch(_ptr(tile_order), _ptr(work_counter), int(ctas), _ptr(stats),
                    ev_begin.cuda_event if ev_begin is not None else None,
                    ev_end.cuda_event if ev_end is not None else None, int(pixels_per_thread),
                    int(batch), _ptr(zero_beside), zb, 1 if grad2d_zeroed else 0)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def gs_record_bytes(attr_dtype):
    return _lib.gs_record_bytes(attr_dtype)


def gs_total_tiles(cams_c, tile_size=16):
    return _lib.gs_total_tiles(cams_c, len(cams_c), int(tile_size))


def gs_total_pixels(cams_c):
    return _lib.gs_total_pixels(cams_c, len(cams_c))


def gs_bin_sort_workspace_size(n_rows, pair_capacity, total_tiles):
    return _lib.gs_bin_sort_workspace_size(n_rows, pair_capacity, total_tiles)


def gs_loss_workspace_size(total_pixels):
    return _lib.gs_loss_workspace_size(total_pixels)


def gs_tile_queue_workspace_size(total_tiles):
    return _lib.gs_tile_queue_workspace_size(total_tiles)


def gs_version():
    return _lib.gs_version().decode()


def gs_kernel_launches():
    return int(_lib.gs_kernel_launches())


def gs_status_string(status):
    return _lib.gs_status_string(status).decode()


def gs_last_error_string():
    return _lib.gs_last_error_string().decode()


def gs_preprocess(means, log_scales, quats, opacity_logits, sh, N, cams_c, prm_c, proj_c,
                  stream=None):
    return _check("gs_preprocess", _lib.gs_preprocess(
        _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh), N, cams_c,
        len(cams_c), ctypes.byref(prm_c), ctypes.byref(proj_c), _stream(stream)))


def gs_bin_sort(proj_c, N, cams_c, workspace, pair_capacity, sorted_vals, sorted_keys, tile_ranges,
                num_pairs_dev, status_dev, sync_count=True, stream=None, tile_size=16):
    """Returns (status, P) with P the host pair count when sync_count, else None.
    GS_ERR_CAPACITY is returned, not raised."""
    nh = ctypes.c_longlong(0)
    st = _lib.gs_bin_sort(ctypes.byref(proj_c), N, cams_c, len(cams_c), int(tile_size),
                          _ptr(workspace),
                          workspace.numel() * workspace.element_size(), pair_capacity,
                          _ptr(sorted_vals), _ptr(sorted_keys), _ptr(tile_ranges),
                          _ptr(num_pairs_dev), ctypes.byref(nh) if sync_count else None,
                          _ptr(status_dev), _stream(stream))
    if st not in (GS_OK, GS_ERR_CAPACITY):
        raise GsError("gs_bin_sort", st)
    return st, (nh.value if sync_count else None)


def gs_render_fwd(proj_c, N, cams_c, prm_c, sorted_vals, tile_ranges, image, final_T, last_idx,
                  entropy, launch_c=None, stream=None):
    return _check("gs_render_fwd", _lib.gs_render_fwd(
        ctypes.byref(proj_c), N, cams_c, len(cams_c), ctypes.byref(prm_c), _ptr(sorted_vals),
        _ptr(tile_ranges), _ptr(image), _ptr(final_T), _ptr(last_idx), _ptr(entropy),
        ctypes.byref(launch_c) if launch_c is not None else None, _stream(stream)))


def gs_loss_l1_entropy(image, target, entropy, cams_c, gamma, loss_dev, dL_dimage, dL_dentropy,
                       workspace, stream=None):
    return _check("gs_loss_l1_entropy", _lib.gs_loss_l1_entropy(
        _ptr(image), _ptr(target), _ptr(entropy), cams_c, len(cams_c), float(gamma),
        _ptr(loss_dev), _ptr(dL_dimage), _ptr(dL_dentropy), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream)))


def gs_loss_base_workspace_size(cams_c):
    return _lib.gs_loss_base_workspace_size(cams_c, len(cams_c))


def gs_loss_base(image, target, entropy, cams_c, lam, gamma, loss_dev, dL_dimage, dL_dentropy,
                 workspace, stream=None):
    return _check("gs_loss_base", _lib.gs_loss_base(
        _ptr(image), _ptr(target), _ptr(entropy), cams_c, len(cams_c), float(lam), float(gamma),
        _ptr(loss_dev), _ptr(dL_dimage), _ptr(dL_dentropy), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream)))


def gs_render_bwd(proj_c, N, cams_c, prm_c, sorted_vals, tile_ranges, final_T, last_idx, dL_dimage,
                  dL_dentropy, means, log_scales, quats, opacity_logits, sh, grad2d, g_means,
                  g_log_scales, g_quats, g_opacity_logits, g_sh, launch_c=None, stream=None):
    return _check("gs_render_bwd", _lib.gs_render_bwd(
        ctypes.byref(proj_c), N, cams_c, len(cams_c), ctypes.byref(prm_c), _ptr(sorted_vals),
        _ptr(tile_ranges), _ptr(final_T), _ptr(last_idx), _ptr(dL_dimage), _ptr(dL_dentropy),
        _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh), _ptr(grad2d),
        _ptr(g_means), _ptr(g_log_scales), _ptr(g_quats), _ptr(g_opacity_logits), _ptr(g_sh),
        ctypes.byref(launch_c) if launch_c is not None else None, _stream(stream)))


GS_STAGE_EXPANSION, GS_STAGE_PROJECTION, GS_STAGE_ADJOINT = 1, 2, 3


def gs_stage_events(stage, ev_begin=None, ev_end=None):
    """Records the torch.cuda.Events (or None to stop) around a stage's
    kernel in this thread's later calls."""
    h = lambda e: ctypes.c_void_p(e.cuda_event) if e is not None else None
    return _check("gs_stage_events", _lib.gs_stage_events(stage, h(ev_begin), h(ev_end)))


def gs_debug_bounds_status(clear=True):
    """(status, first failed check id) of the bounds-checked debug build;
    status is GS_ERR_UNSUPPORTED in the normal build."""
    v = ctypes.c_uint(0)
    st = _lib.gs_debug_bounds_status(ctypes.byref(v), 1 if clear else 0)
    return st, int(v.value)


def gs_grad2d_attributes(proj_c, N, V, prm_c, grad2d, out, stream=None):
    """dL/d(mean2d, conic a b c, sigma, rgb) [V*N, 9] from grad2d's moment rows."""
    return _check("gs_grad2d_attributes", _lib.gs_grad2d_attributes(
        ctypes.byref(proj_c), N, V, ctypes.byref(prm_c), _ptr(grad2d), _ptr(out),
        _stream(stream)))


def gs_scale_reset(log_scales, zeta, stream=None):
    return _check("gs_scale_reset", _lib.gs_scale_reset(_ptr(log_scales), log_scales.numel(),
                                                        float(zeta), _stream(stream)))


def gs_tile_queue(tile_ranges, total_tiles, tile_order, workspace, stream=None):
    return _check("gs_tile_queue", _lib.gs_tile_queue(
        _ptr(tile_ranges), total_tiles, _ptr(tile_order), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream)))


def gs_tile_queue_static(tile_ranges, total_tiles, tile_order, stream=None):
    """Tile queue in the library's fixed scratch array (no allocation);
    returns the status instead of raising on GS_ERR_INVALID_ARG."""
    st = _lib.gs_tile_queue_static(_ptr(tile_ranges), total_tiles, _ptr(tile_order),
                                   _stream(stream))
    if st not in (GS_OK, GS_ERR_INVALID_ARG):
        raise GsError("gs_tile_queue_static", st)
    return st

