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


def test_render_launch_options_checked_on_the_host(lib_path):
    """Launch controls that no kernel exists for are rejected by both render
    calls before any launch (the pointers below are never dereferenced)."""
    from paper_2603_09277_gb300 import gs, scenes
    lib = gs._lib
    cams = gs.make_cameras([scenes.camera(64, 48, 64.0)])
    fake = 4096  # 16-byte aligned, never touched: every call fails validation
    proj = gs.GsProj(fake, fake, fake, fake, None, None, None, None)

    def calls(prm, opt):
        fwd = lib.gs_render_fwd(ctypes.byref(proj), 10, cams, 1, ctypes.byref(prm), fake, fake,
                                fake, fake, fake, fake, ctypes.byref(opt), None)
        bwd = lib.gs_render_bwd(ctypes.byref(proj), 10, cams, 1, ctypes.byref(prm), fake, fake,
                                fake, fake, fake, fake, fake, fake, fake, fake, fake, fake, fake,
                                fake, fake, fake, fake, ctypes.byref(opt), None)
        return fwd, bwd

    bad = [(16, "f32", dict(pixels_per_thread=3), b"pixels_per_thread"),
           (8, "f32", dict(pixels_per_thread=4), b"16-pixel tiles"),
           (16, "f32", dict(batch=64), b"batch"),
           (16, "bf16", dict(batch=128), b"F32 records"),
           (8, "f32", dict(batch=128), b"F32 records"),
           (16, "f32", dict(ctas=-1), b"ctas"),
           (16, "f32", dict(ctas=152), b"work_counter")]
    for tile, attr, kw, why in bad:
        prm = gs.make_params(scenes.params(tile=tile), 16, attr)
        for status in calls(prm, gs.make_launch(**kw)):
            assert status == gs.GS_ERR_INVALID_ARG, (tile, attr, kw)
            assert why in lib.gs_last_error_string(), (kw, lib.gs_last_error_string())


def test_autotune_candidates_exist_for_the_workload():
    """Every form the autotuner may pick is one the render calls accept: no
    4-pixel form on 8-pixel tiles, the 128-entry batch only for F32 records
    on 16-pixel tiles; forms have distinct names (the timing table's keys)."""
    from paper_2603_09277_gb300 import autotune
    for tile in (16, 8):
        for attr in ("f32", "f16", "bf16"):
            c = autotune.candidates(tile, attr)
            names = [autotune.form_name(f) for f in c]
            assert len(set(names)) == len(names) >= 3
            for f in c:
                assert f["pixels_per_thread"] in (1, 2, 4) and f["batch"] in (128, 256)
                assert tile == 16 or f["pixels_per_thread"] <= 2
                assert f["batch"] == 256 or (tile == 16 and attr == "f32")
                assert f["persistent"] % autotune.sm_count() == 0
    c = autotune.candidates(16, "f32")
    assert {f["batch"] for f in c} == {128, 256}
    assert len({f["persistent"] for f in c if f["persistent"]}) >= 2


def test_debug_bounds_status_needs_the_debug_build():
    """The normal build carries no index checks: the status call says so
    (GS_ERR_UNSUPPORTED) and reports no failed check."""
    from paper_2603_09277_gb300 import gs
    if os.environ.get("GS_LIBRARY"):
        pytest.skip("another build of the library is loaded")
    st, first = gs.gs_debug_bounds_status(clear=True)
    assert st == gs.GS_ERR_UNSUPPORTED and first == 0
