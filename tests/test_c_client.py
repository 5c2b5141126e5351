"""The boundary is a plain C ABI. A C11 program that includes include/gs.h
(no C++ and no CUDA headers), takes the address of every declared entry
point, links against libgs.so and calls the host-only functions and the
host-side argument checks; another prints the C compiler's layout of the
header's structs, which the binding's ctypes structs must match.  Nothing
here reaches a GPU: every compute call below fails validation before it
enqueues anything."""
import ctypes
import os
import shutil
import subprocess

import pytest

from test_abi import HEADER, declared_functions, lib_path  # noqa: F401  (fixture)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include "gs.h"

static void camera(gs_camera* c, int w, int h, float f) {
  memset(c, 0, sizeof *c);
  c->width = w; c->height = h; c->fx = c->fy = f;
  c->cx = 0.5f * (float)w; c->cy = 0.5f * (float)h;
  c->world_to_cam[0] = c->world_to_cam[5] = c->world_to_cam[10] = 1.f;
}

int main(void) {
  uintptr_t table[] = { %(table)s };
  size_t resolved = 0;
  for (size_t i = 0; i < sizeof table / sizeof table[0]; ++i) resolved += table[i] != 0;
  printf("resolved %%zu of %%zu\n", resolved, sizeof table / sizeof table[0]);

  gs_camera c[2];
  camera(&c[0], 64, 48, 64.f);
  camera(&c[1], 33, 17, 40.f);
  printf("tiles %%lld %%lld %%lld\n", gs_total_tiles(c, 2, 16), gs_total_tiles(c, 2, 8),
         gs_total_tiles(c, 2, 12));
  printf("pixels %%lld\n", gs_total_pixels(c, 2));
  printf("record %%d %%d %%d\n", gs_record_bytes(GS_ATTR_F32), gs_record_bytes(GS_ATTR_BF16),
         gs_record_bytes(9));

  int st = gs_scale_reset(NULL, 10, 0.2f, NULL);
  printf("reset %%d %%s\n", st, gs_status_string(st));

  gs_params prm;
  memset(&prm, 0, sizeof prm);
  prm.alpha_max = 0.99f; prm.alpha_min = 1.f / 255.f; prm.t_min = 1e-4f;
  prm.dilation = 0.3f; prm.near_z = 0.2f; prm.fov_clamp = 1.3f;
  prm.sh_degree = 0; prm.sh_stride = 16; prm.attr_dtype = GS_ATTR_F32; prm.tile_size = 16;
  void* fake = (void*)(uintptr_t)4096;  /* never dereferenced */
  gs_proj proj;
  memset(&proj, 0, sizeof proj);
  proj.records = fake; proj.depth = (float*)fake; proj.rect = (int*)fake;
  proj.tiles_touched = (unsigned*)fake;
  gs_launch opt;
  memset(&opt, 0, sizeof opt);
  opt.pixels_per_thread = 3;
  st = gs_render_fwd(&proj, 10, c, 2, &prm, (const unsigned*)fake, (const unsigned*)fake,
                     (float*)fake, (float*)fake, (unsigned*)fake, (float*)fake, &opt, NULL);
  printf("fwd %%d %%s\n", st, gs_last_error_string());
  opt.pixels_per_thread = 2;
  opt.batch = 128;
  prm.attr_dtype = GS_ATTR_BF16;
  st = gs_render_fwd(&proj, 10, c, 2, &prm, (const unsigned*)fake, (const unsigned*)fake,
                     (float*)fake, (float*)fake, (unsigned*)fake, (float*)fake, &opt, NULL);
  printf("fwd %%d %%s\n", st, gs_last_error_string());
  printf("version %%s\n", gs_version());

  /* the int4 rects may be left out only where the packed rects carry them */
  const float* ff = (const float*)fake;
  prm.attr_dtype = GS_ATTR_F32;
  proj.rect = NULL;
  proj.rect8 = NULL;
  st = gs_preprocess(ff, ff, ff, ff, ff, 10, c, 2, &prm, &proj, NULL);
  printf("norect %%d %%s\n", st, gs_last_error_string());
  gs_camera wide;
  camera(&wide, 16 * 300, 48, 1000.f);  /* 300 tiles wide */
  proj.rect8 = (unsigned*)fake;
  st = gs_preprocess(ff, ff, ff, ff, ff, 10, &wide, 1, &prm, &proj, NULL);
  printf("norect %%d %%s\n", st, gs_last_error_string());
  long long np = 0;
  int status = 0;
  st = gs_bin_sort(&proj, 10, &wide, 1, 16, fake, 1u << 30, 100, (unsigned*)fake, NULL,
                   (unsigned*)fake, &np, NULL, &status, NULL);
  printf("norect %%d %%s\n", st, gs_last_error_string());
  return 0;
}
"""


def test_c11_program_links_and_calls_the_abi(lib_path, tmp_path):  # noqa: F811
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = PROGRAM % {"table": ", ".join("(uintptr_t)&%s" % n for n in names)}
    (tmp_path / "client.c").write_text(src)
    libdir = os.path.dirname(lib_path)
    exe = str(tmp_path / "client")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.dirname(HEADER), str(tmp_path / "client.c"),
                        "-L", libdir, "-lgs", "-Wl,-rpath," + libdir, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    out = r.stdout.splitlines()
    assert out[0] == "resolved %d of %d" % (len(names), len(names))
    assert out[1] == "tiles %d %d -1" % (4 * 3 + 3 * 2, 8 * 6 + 5 * 3)
    assert out[2] == "pixels %d" % (64 * 48 + 33 * 17)
    assert out[3] == "record 48 32 -1"
    assert out[4].startswith("reset -1 ")
    assert out[5].startswith("fwd -1 ") and "pixels_per_thread" in out[5]
    assert out[6].startswith("fwd -1 ") and "F32 records" in out[6]
    assert out[7].startswith("version ") and "sm_103a" in out[7]
    assert out[8].startswith("norect -1 ") and "projection buffers" in out[8]
    assert out[9].startswith("norect -1 ") and "255 tiles" in out[9]
    assert out[10].startswith("norect -1 ") and "255 tiles" in out[10]


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structs of the binding have the C compiler's layout of the
    header's structs: the same size and every field at the same offset."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2603_09277_gb300 import gs
    structs = {"gs_camera": gs.GsCamera, "gs_params": gs.GsParams, "gs_proj": gs.GsProj,
               "gs_launch": gs.GsLaunch}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (cname, field, cname, field))
    lines += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                        str(tmp_path / "layout.c"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got["%s size" % cname]) == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert int(got["%s %s" % (cname, field)]) == getattr(py, field).offset, (cname, field)
