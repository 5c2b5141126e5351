"""The C-ABI library builds for sm_103a and exports every entry point that
include/gs.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(gs_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2603_09277_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("gs_preprocess", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_scale_reset"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (gs_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_wraps_every_symbol(lib_path):
    from paper_2603_09277_gb300 import gs
    assert set(declared_functions()) == set(gs.EXPORTED)
    for n in gs.EXPORTED:
        assert hasattr(gs, n)


def test_host_side_argument_checks(lib_path):
    """Calls that fail validation on the host return before touching a GPU."""
    from paper_2603_09277_gb300 import gs, scenes
    lib = gs._lib
    cams = gs.make_cameras([scenes.camera(64, 48, 64.0), scenes.camera(33, 17, 40.0)])
    assert lib.gs_total_tiles(cams, 2, 16) == 4 * 3 + 3 * 2
    assert lib.gs_total_tiles(cams, 2, 0) == 4 * 3 + 3 * 2
    assert lib.gs_total_tiles(cams, 2, 8) == 8 * 6 + 5 * 3  # 8-pixel tiles
    assert lib.gs_total_tiles(cams, 2, 12) == -1
    assert lib.gs_total_pixels(cams, 2) == 64 * 48 + 33 * 17
    assert lib.gs_record_bytes(gs.GS_ATTR_F32) == 48
    assert lib.gs_record_bytes(gs.GS_ATTR_F16) == 32
    assert lib.gs_record_bytes(7) == -1
    assert lib.gs_scale_reset(None, 10, ctypes.c_float(0.2), None) == gs.GS_ERR_INVALID_ARG
    assert lib.gs_scale_reset(None, 0, ctypes.c_float(1.5), None) == gs.GS_ERR_INVALID_ARG
    prm = gs.make_params(scenes.params(), 16)
    prm.sh_degree = 4
    proj = gs.make_proj(None, None, None, None)
    assert lib.gs_preprocess(None, None, None, None, None, 0, cams, 2, ctypes.byref(prm),
                             ctypes.byref(proj), None) == gs.GS_ERR_INVALID_ARG
    assert b"invalid argument" in lib.gs_last_error_string()
    prm.sh_degree = 0
    prm.tile_size = 12  # only 16 and 8 pixel tiles exist
    assert lib.gs_preprocess(None, None, None, None, None, 0, cams, 2, ctypes.byref(prm),
                             ctypes.byref(proj), None) == gs.GS_ERR_INVALID_ARG
    ws = ctypes.c_void_p(256)  # never dereferenced: the tile side is rejected first
    assert lib.gs_bin_sort(ctypes.byref(proj), 0, cams, 2, 12, ws, 0, 0, None, None, None, None,
                           None, None, None) == gs.GS_ERR_INVALID_ARG
    assert b"tile_size" in lib.gs_last_error_string()
    assert lib.gs_bin_sort_workspace_size(1000, 5000, 64) > 0
    assert b"sm_103a" in lib.gs_version()
