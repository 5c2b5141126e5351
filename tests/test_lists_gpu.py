"""Per-tile lists (ranges, list contents and their (depth, id) order) against
the oracle's plain definition on layouts that exercise the list
construction's corners: a view with more than 256 super-tiles of 8x8 tiles
(the super-tile sort then takes two radix passes), views whose tile grids
end inside a super-tile (1x1, 9x9, 2x19, 63x2 tiles), Gaussians whose rects
span many super-tiles, the largest view count (64 views), more than
4 M (view, Gaussian) rows (the row scans then take 4,096-row blocks), and
views of 255 and 263 tiles per side (the rects travel 8-bit packed up to
255 tiles, in 16-bit fields beyond)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2603_09277_gb300 import scenes

from parity_util import run_gpu, view_tiles

pytestmark = pytest.mark.gpu


def _compare_lists(scene, cams, prm):
    N = scene["means"].shape[0]
    g = run_gpu(scene, cams, prm, keys=True)
    vt = view_tiles(cams)
    total = 0
    for v, cam in enumerate(cams):
        proj = oracle.preprocess(scene, cam, prm)
        ts, ids = oracle.build_lists(proj, cam)
        flagged = proj["boundary"].astype(bool)
        t0, t1 = vt[v]
        rng = g["ranges"][t0:t1]
        lens = rng[:, 1] - rng[:, 0]
        if not flagged.any():
            # ranges bit-exact: starts are the running sum of the lengths over
            # all tiles of all views; empty lists are (0, 0)
            assert (lens == np.diff(ts)).all()
        for t in range(t1 - t0):
            a, b = rng[t]
            glist = g["vals"][a:b] - v * N
            olist = ids[ts[t]:ts[t + 1]]
            if flagged.any():
                glist = glist[~flagged[glist]]
                olist = olist[~flagged[olist]]
            assert len(glist) == len(olist) and (glist == olist).all(), (v, t)
        total += len(ids)
    ranges = g["ranges"]
    nz = ranges[:, 1] > ranges[:, 0]
    # non-empty lists tile sorted_vals in global tile order without gaps
    starts, ends = ranges[nz, 0], ranges[nz, 1]
    assert starts[0] == 0 and (starts[1:] == ends[:-1]).all() and ends[-1] == g["P"]
    assert (ranges[~nz] == 0).all()
    # 64-bit keys (tile << 32 | depth bits): the tile of every slot, and
    # non-decreasing overall (tile first, then depth within a tile)
    keys = g["keys"].view(np.int64)
    assert ((keys >> 32) == np.repeat(np.nonzero(nz)[0], ends - starts)).all()
    assert (np.diff(keys) >= 0).all()
    assert ((keys & 0xffffffff).astype(np.uint32) == g["depth"][g["vals"]].view(np.uint32)).all()
    any_flagged = any(oracle.preprocess(scene, c, prm)["boundary"].any() for c in cams)
    return g["P"], total, any_flagged


def test_lists_view_with_two_pass_super_tile_sort():
    # 2600 x 2100 px: 163 x 132 tiles -> 21 x 17 = 357 super-tiles (9 bits, two passes)
    scene = scenes.box_scene(20_000, seed=5, ls_mean=-4.0, ls_std=0.8)
    cams = [scenes.camera(2600, 2100, 2600.0)]
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 100_000 and (flagged or P == total)


def test_lists_ragged_super_tile_borders_and_wide_rects():
    # tile grids of 1x1, 9x9, 2x19 and 63x2; large Gaussians whose rects span
    # several super-tiles
    sizes = [(16, 16), (129, 135), (20, 300), (1000, 31)]
    cams = [scenes.camera(w, h, float(w)) for w, h in sizes]
    scene = scenes.box_scene(3_000, seed=6, ls_mean=-2.0, ls_std=1.0)
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 10_000 and (flagged or P == total)


def test_lists_sixty_four_views():
    rng = np.random.default_rng(7)
    yaws = list(rng.uniform(-20.0, 20.0, 64))
    sizes = [(int(w), int(h)) for w, h in zip(rng.integers(24, 200, 64), rng.integers(24, 160, 64))]
    cams = scenes.yaw_cameras(sizes, yaws)
    scene = scenes.box_scene(2_000, seed=8)
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 10_000 and (flagged or P == total)


def test_lists_more_than_four_million_rows():
    # 70,000 Gaussians x 64 views = 4.48 M rows: the depth-ordered gather and
    # the expansion run on 4,096-row blocks (1,024 up to 4 M rows)
    rng = np.random.default_rng(9)
    yaws = list(rng.uniform(-20.0, 20.0, 64))
    sizes = [(int(w), int(h)) for w, h in zip(rng.integers(24, 200, 64), rng.integers(24, 160, 64))]
    cams = scenes.yaw_cameras(sizes, yaws)
    scene = scenes.box_scene(70_000, seed=10)
    assert 70_000 * 64 > (4 << 20)
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 10_000_000 and (flagged or P == total)


@pytest.mark.parametrize("width", [4080, 4200])
def test_lists_rect_packing_limits(width):
    # 4080 px: 255 tiles, the widest grid of the 8-bit rect packing;
    # 4200 px: 263 tiles, the 16-bit fields; Gaussians reach both edges
    scene = scenes.box_scene(6_000, seed=11, ls_mean=-3.0, ls_std=0.8)
    cams = [scenes.camera(width, 48, float(width) / 2.0)]
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 5_000 and (flagged or P == total)


@pytest.mark.parametrize("sizes", [[(4080, 48)], [(309, 205), (618, 411), (1237, 822)],
                                   [(4200, 48)]])
def test_lists_and_images_from_the_packed_rects_alone(sizes):
    # with every view at most 255 tiles per side the projection leaves the
    # int4 rects out (rect NULL) and the lists come from the packed rects
    # alone: lists, ranges and the forward's outputs equal those of the
    # call that writes both, bit for bit; a wider view keeps the int4 rects
    from paper_2603_09277_gb300.rasterize import Rasterizer, scene_to_device
    scene = scenes.box_scene(8_000, seed=12, ls_mean=-3.0, ls_std=0.8)
    cams = [scenes.camera(w, h, float(w)) for w, h in sizes]
    fits = all(-(-w // 16) <= 255 and -(-h // 16) <= 255 for w, h in sizes)
    p = scene_to_device(scene)
    out = []
    for debug in (False, True):
        r = Rasterizer(cams, scenes.params(), scene["means"].shape[0], keep_debug=debug)
        assert r.rect8_only == (fits and not debug) and (r.rect is None) == r.rect8_only
        r.preprocess(p)
        P = r.bin_sort(keys=True)
        r.render_fwd()
        torch.cuda.synchronize()
        out.append({"P": P, "vals": r.sorted_vals[:P].cpu(), "keys": r.sorted_keys[:P].cpu(),
                    "ranges": r.tile_ranges.cpu(), "image": r.image.cpu(),
                    "T": r.final_T.cpu(), "last": r.last_idx.cpu(), "H": r.entropy.cpu()})
    a, b = out
    assert a["P"] == b["P"] > 1_000
    for k in ("vals", "keys", "ranges", "image", "T", "last", "H"):
        assert torch.equal(a[k], b[k]), k


def test_lists_all_depths_equal():
    # every Gaussian at the same depth: the depth range has no significant
    # bits, the sort is its first pass alone, and every list is in Gaussian
    # id order (the ties of the (tile, depth, id) order)
    scene = scenes.box_scene(5_000, seed=13, ls_mean=-3.0, ls_std=0.6)
    scene["means"][:, 2] = np.float32(4.0)
    cams = [scenes.camera(256, 256, 256.0), scenes.camera(200, 120, 180.0)]
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 5_000 and (flagged or P == total)


@pytest.mark.parametrize("span", [0xFF10, 0xFFFF10])
def test_lists_depth_range_across_digit_boundaries(span):
    # depth bits from m to m + span with m's low byte 0xF0: rounding the
    # range's minimum down to a multiple of 256 for the later passes adds a
    # significant bit (17 instead of 16, 25 instead of 24), so one more pass
    # runs; the lists still follow (tile, depth, id)
    rng = np.random.default_rng(14)
    scene = scenes.box_scene(6_000, seed=14, ls_mean=-3.0, ls_std=0.6)
    m = np.uint32(0x40800000 + 0xF0)  # just above 4.0
    bits = (m + rng.integers(0, span + 1, 6_000, dtype=np.uint64).astype(np.uint32))
    bits[0], bits[1] = m, m + np.uint32(span)
    scene["means"][:, 2] = bits.view(np.float32)
    cams = [scenes.camera(256, 256, 256.0)]
    P, total, flagged = _compare_lists(scene, cams, scenes.params())
    assert P > 5_000 and (flagged or P == total)
