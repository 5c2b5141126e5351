"""Pins of the FP64 oracle to facts outside itself: hand-computed values, the
paper's invariant (Suppl. A), its three equivalent forms of the entropy
gradient (Suppl. B, Sec. 4.4, Algorithm 1), closed forms, library routines
(scipy rotations, Gauss-Legendre quadrature), brute force, and central finite
differences.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_09277_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Entropy on the weights (Sec. 4.3) and its gradient (Sec. 4.4, Suppl. B)
# --------------------------------------------------------------------------

def test_golden_two_half():
    rows = np.loadtxt(os.path.join(GOLDEN, "entropy_two_half.txt"))
    a = rows[:2]
    H, d1, d2 = rows[2], rows[3], rows[4]
    assert oracle.entropy(a) == pytest.approx(H, abs=1e-15)
    for fn in (oracle.dH_dalpha_direct, oracle.dH_dalpha_closed, oracle.dH_dalpha_alg1):
        g = fn(a)
        assert g[0] == pytest.approx(d1, abs=1e-15)
        assert g[1] == pytest.approx(d2, abs=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 30, 120])
def test_entropy_grad_three_ways_and_fd(n):
    rng = np.random.default_rng(n)
    a = rng.uniform(1.0 / 255, 0.99, n)
    # keep T above t_min like the renderer does
    a = np.minimum(a, 0.5) if n > 10 else a
    d = oracle.dH_dalpha_direct(a)
    c = oracle.dH_dalpha_closed(a)
    g = oracle.dH_dalpha_alg1(a)
    scale = np.abs(d).max()
    assert np.abs(d - c).max() <= 1e-12 * scale
    assert np.abs(d - g).max() <= 1e-12 * scale
    for i in range(n):
        h = 1e-6
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        fd = (oracle.entropy(ap) - oracle.entropy(am)) / (2 * h)
        assert fd == pytest.approx(d[i], rel=1e-6, abs=1e-8)


def test_entropy_uniform_maximum():
    # weights all equal to 1/(n+1): alpha_i = 1/(n+2-i) gives w_i = 1/(n+1)
    n = 9
    a = np.array([1.0 / (n + 1 - i) for i in range(n)])
    assert oracle.entropy(a) == pytest.approx(math.log(n + 1), rel=1e-14)


# --------------------------------------------------------------------------
# Compositing invariants on a full config-1 view
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg1():
    scene, cams, targets, prm = scenes.config1()
    proj = oracle.preprocess(scene, cams[0], prm)
    lists = oracle.build_lists(proj, cams[0])
    fwd = oracle.render_fwd(proj, lists, cams[0], prm)
    return scene, cams, targets, prm, proj, lists, fwd


def test_weights_sum_to_unity(cfg1):
    """Suppl. A: sum_{i<=N} w_i + T_{N+1} = 1 at every pixel.  With every
    colour set to 1 the composite equals sum w."""
    scene, cams, targets, prm, proj, lists, fwd = cfg1
    p1 = dict(proj)
    p1["P9"] = proj["P9"].copy()
    p1["P9"][:, 6:9] = 1.0
    f1 = oracle.render_fwd(p1, lists, cams[0], prm)
    s = f1["image"][..., 0] + f1["final_T"]
    assert np.abs(s - 1.0).max() < 1e-12
    assert (f1["final_T"] >= np.float32(prm["t_min"])).all()


def test_entropy_bounds(cfg1):
    *_, fwd = cfg1
    H, nb = fwd["entropy"], fwd["nblend"]
    assert (H >= -1e-15).all()
    assert (H <= np.log(nb + 1.0) + 1e-12).all()
    assert (H[nb == 0] == pytest.approx(0.0, abs=1e-15))


def test_list_lengths_match_tiles_touched(cfg1):
    scene, cams, targets, prm, proj, lists, fwd = cfg1
    ts, ids = lists
    assert ts[-1] == proj["tiles"].sum()
    # every Gaussian appears in exactly tiles_touched lists
    counts = np.bincount(ids, minlength=proj["tiles"].size)
    assert (counts == proj["tiles"]).all()
    # each list is sorted by (depth bits, id)
    dk = proj["depth"].view(np.uint32)
    for t in range(len(ts) - 1):
        seg = ids[ts[t]:ts[t + 1]]
        key = (dk[seg].astype(np.uint64) << np.uint64(32)) | seg.astype(np.uint64)
        assert (key[1:] > key[:-1]).all()  # exact 64-bit comparison, strictly increasing


# --------------------------------------------------------------------------
# Projection (Sec. 3): closed forms and library routines
# --------------------------------------------------------------------------

def _one(mu, ls, q, op, sh0=(0.0, 0.0, 0.0)):
    sh = np.zeros((1, 16, 3), np.float32)
    sh[0, 0] = sh0
    return {"means": np.array([mu], np.float32), "log_scales": np.array([ls], np.float32),
            "quats": np.array([q], np.float32), "opacity_logits": np.array([op], np.float32),
            "sh": sh, "sh_degree": 0}


def test_isotropic_on_axis_closed_form():
    """A single isotropic Gaussian (scale s0, identity rotation) on the optical
    axis at depth z, dilation 0: Sigma' = (f s0 / z)^2 I, conic = (z/(f s0))^2 I,
    r = ceil(3 f s0 / z); C(p) = c min(0.99, sigma exp(-|p - mu'|^2 z^2 / (2 f^2 s0^2)))
    where that is >= 1/255 inside the rect, H = -w log w - (1 - w) log(1 - w)."""
    W = H = 64
    f, z, s0 = 64.0, 3.0, 0.09375  # f s0 / z = 2 px exactly
    op = 1.5
    prm = scenes.params(dilation=0.0)
    cam = scenes.camera(W, H, f)
    scene = _one((0.0, 0.0, z), [math.log(s0)] * 3, (1.0, 0.0, 0.0, 0.0), op,
                 sh0=(0.5 * 2 * math.sqrt(math.pi),) * 3)
    proj = oracle.preprocess(scene, cam, prm)
    s0 = math.exp(float(scene["log_scales"][0, 0]))  # the stored FP32 log-scale
    sig_px = f * s0 / z
    P9 = proj["P9"][0]
    assert P9[0] == pytest.approx(W / 2, abs=1e-12) and P9[1] == pytest.approx(H / 2, abs=1e-12)
    assert P9[2] == pytest.approx(1 / sig_px ** 2, rel=1e-12)
    assert P9[3] == pytest.approx(0.0, abs=1e-14)
    assert P9[4] == pytest.approx(1 / sig_px ** 2, rel=1e-12)
    sigma = 1 / (1 + math.exp(-float(np.float32(op))))
    assert P9[5] == pytest.approx(sigma, rel=1e-14)
    col = float(scene["sh"][0, 0, 0]) / (2 * math.sqrt(math.pi)) + 0.5  # Y00 sh0 + 0.5 ~ 1
    assert P9[6:9] == pytest.approx([col] * 3, rel=1e-14)
    r = math.ceil(3 * sig_px)
    assert proj["radius"][0] == r
    lists = oracle.build_lists(proj, cam)
    fwd = oracle.render_fwd(proj, lists, cam, prm)
    TX = W // 16
    x0, y0, x1, y1 = proj["rect"][0]
    amin, amax = float(np.float32(1 / 255)), float(np.float32(0.99))
    side = oracle.tile_of(prm)
    for v in range(H):
        for u in range(W):
            tx, ty = u // side, v // side
            inside = x0 <= tx < x1 and y0 <= ty < y1
            d2 = (u + 0.5 - W / 2) ** 2 + (v + 0.5 - H / 2) ** 2
            a = min(amax, sigma * math.exp(-d2 / (2 * sig_px ** 2)))
            w = a if (inside and a >= amin) else 0.0
            assert fwd["image"][v, u, 0] == pytest.approx(w * col, abs=1e-14)
            Hc = 0.0 if w == 0.0 else -w * math.log(w) - (1 - w) * math.log(1 - w)
            assert fwd["entropy"][v, u] == pytest.approx(Hc, abs=1e-14)
    assert TX == 4


def _rot_scipy(q_wxyz):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q_wxyz
    return Rotation.from_quat([x, y, z, w]).as_matrix()  # scalar-last in scipy


def _pinhole(cam, X):
    wtc = cam["world_to_cam"].astype(np.float64)
    t = wtc[:, :3] @ X + wtc[:, 3]
    return np.array([cam["fx"] * t[0] / t[2] + cam["cx"], cam["fy"] * t[1] / t[2] + cam["cy"]])


def test_projection_matches_library_linearisation():
    """EWA (Sec. 3): Sigma' = J Sigma J^T + dilation I, with J the Jacobian of
    the pinhole map at the mean (here by central differences of the pinhole
    map itself) and Sigma = R S S^T R^T with R from scipy's quaternion
    rotation; conic = Sigma'^-1; opacity = scipy.special.expit(logit)."""
    from scipy.special import expit
    rng = np.random.default_rng(5)
    pos = np.array([0.7, -0.4, -1.0])
    cam = scenes.camera(200, 150, 180.0, scenes.look_at(pos, (0.1, 0.2, 3.0)), pos)
    prm = scenes.params()
    for _ in range(20):
        mu = np.array([rng.uniform(-0.5, 0.7), rng.uniform(-0.3, 0.6), rng.uniform(2.5, 4.0)])
        ls = rng.normal(-3.0, 0.5, 3)
        q = rng.standard_normal(4)
        op = rng.normal()
        sc = _one(mu, ls, q, op)
        proj = oracle.preprocess(sc, cam, prm)
        X = sc["means"][0].astype(np.float64)
        Jn = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            Jn[:, k] = (_pinhole(cam, X + e) - _pinhole(cam, X - e)) / 2e-6
        qq = sc["quats"][0].astype(np.float64)
        R = _rot_scipy(qq / np.linalg.norm(qq))
        S = np.diag(np.exp(sc["log_scales"][0].astype(np.float64)))
        Sig = R @ S @ S.T @ R.T
        S2 = Jn @ Sig @ Jn.T + float(np.float32(0.3)) * np.eye(2)
        K = np.linalg.inv(S2)
        P9 = proj["P9"][0]
        assert P9[0:2] == pytest.approx(_pinhole(cam, X), rel=1e-12)
        assert P9[2] == pytest.approx(K[0, 0], rel=1e-7)
        assert P9[3] == pytest.approx(K[0, 1], rel=1e-6, abs=1e-9)
        assert P9[4] == pytest.approx(K[1, 1], rel=1e-7)
        assert P9[5] == pytest.approx(expit(float(sc["opacity_logits"][0])), rel=1e-14)
        # radius: 3 sqrt of the larger eigenvalue, rounded up
        lam = np.linalg.eigvalsh(S2).max()
        assert proj["radius"][0] == math.ceil(3 * math.sqrt(lam))


def test_near_plane_culls():
    cam = scenes.camera(64, 64, 64.0)
    prm = scenes.params()
    sc = _one((0.0, 0.0, 0.1999), [-3.0] * 3, (1, 0, 0, 0), 0.0)
    assert oracle.preprocess(sc, cam, prm)["tiles"][0] == 0
    sc = _one((0.0, 0.0, 0.25), [-3.0] * 3, (1, 0, 0, 0), 0.0)
    assert oracle.preprocess(sc, cam, prm)["tiles"][0] > 0


def test_depth_key_is_fp32_of_fp64_depth():
    pos = np.array([0.3, -0.2, -0.5])
    cam = scenes.camera(64, 64, 64.0, scenes.look_at(pos, (0.0, 0.1, 3.0)), pos)
    sc, _, _, prm = scenes.tiny_scene(8, seed=3, width=64, height=64)
    proj = oracle.preprocess(sc, cam, prm)
    R = cam["world_to_cam"].astype(np.float64)
    m = sc["means"].astype(np.float64)
    tz = ((R[2, 0] * m[:, 0] + R[2, 1] * m[:, 1]) + R[2, 2] * m[:, 2]) + R[2, 3]
    assert (proj["depth"] == tz.astype(np.float32)).all()


# --------------------------------------------------------------------------
# Spherical harmonics (Sec. 3: colour in SH up to degree 3)
# --------------------------------------------------------------------------

def test_sh_orthonormal_by_quadrature():
    """int_S2 Y_i Y_j = delta_ij: Gauss-Legendre in cos(theta) (exact for
    polynomials up to degree 2n-1) times a uniform grid in phi (exact for
    trigonometric polynomials below the grid size)."""
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 16
    phis = 2 * np.pi * np.arange(nphi) / nphi
    dirs, wts = [], []
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            dirs.append((r * math.cos(ph), r * math.sin(ph), z))
            wts.append(w * 2 * np.pi / nphi)
    Y = oracle.sh_basis(3, np.array(dirs))
    G = (Y * np.array(wts)[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_harmonic_and_homogeneous():
    """Each basis function is a homogeneous harmonic polynomial of its degree:
    Y(2x) = 2^l Y(x) and its Laplacian (second central differences, exact for
    cubics up to rounding) vanishes."""
    rng = np.random.default_rng(0)
    degs = [0] + [1] * 3 + [2] * 5 + [3] * 7
    for _ in range(10):
        x = rng.standard_normal(3)
        Y1 = oracle.sh_basis(3, x)[0]
        Y2 = oracle.sh_basis(3, 2 * x)[0]
        assert Y2 == pytest.approx(Y1 * 2.0 ** np.array(degs), rel=1e-12, abs=1e-14)
        h = 1e-2
        lap = -6 * Y1
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            lap = lap + oracle.sh_basis(3, x + e)[0] + oracle.sh_basis(3, x - e)[0]
        assert np.abs(lap / h ** 2).max() < 1e-8
    assert oracle.sh_basis(0, np.array([0.0, 0.0, 1.0]))[0, 0] == pytest.approx(
        1 / (2 * math.sqrt(math.pi)), rel=1e-15)


# --------------------------------------------------------------------------
# Tile lists and compositing against a per-pixel brute force
# --------------------------------------------------------------------------

def _brute_force(proj, cam, prm):
    """Per pixel: every Gaussian whose rect covers the pixel's tile, sorted by
    (depth, id), composited front to back (Sec. 3)."""
    W, H = cam["width"], cam["height"]
    amax, amin, tmin = (float(np.float32(prm[k])) for k in ("alpha_max", "alpha_min", "t_min"))
    P9, rect, tiles, depth = proj["P9"], proj["rect"], proj["tiles"], proj["depth"]
    img = np.zeros((H, W, 3))
    Tf = np.ones((H, W))
    Hm = np.zeros((H, W))
    last = np.zeros((H, W), np.int32)
    side = oracle.tile_of(prm)
    for v in range(H):
        for u in range(W):
            tx, ty = u // side, v // side
            cand = [i for i in range(len(tiles)) if tiles[i] > 0 and rect[i, 0] <= tx < rect[i, 2]
                    and rect[i, 1] <= ty < rect[i, 3]]
            cand.sort(key=lambda i: (depth[i], i))
            T, swl = 1.0, 0.0
            for pos, i in enumerate(cand):
                g = P9[i]
                dx, dy = u + 0.5 - g[0], v + 0.5 - g[1]
                a = min(amax, g[5] * math.exp(-0.5 * (g[2] * dx * dx + 2 * g[3] * dx * dy
                                                        + g[4] * dy * dy)))
                if a < amin:
                    continue
                if T * (1 - a) < tmin:
                    break
                w = a * T
                img[v, u] += w * g[6:9]
                swl += w * math.log(w)
                T *= 1 - a
                last[v, u] = pos + 1
            Tf[v, u] = T
            Hm[v, u] = -(swl + T * math.log(T))
    return img, Tf, Hm, last


@pytest.mark.parametrize("seed,tile", [(0, 16), (1, 16), (2, 16), (3, 8), (4, 8)])
def test_tiled_equals_brute_force(seed, tile):
    scene, cams, _, prm = scenes.tiny_scene(8, seed=seed, width=48, height=40)
    prm["tile"] = tile
    scene["opacity_logits"][:] = 3.0  # long enough to reach the T stop
    cam = cams[0]
    proj = oracle.preprocess(scene, cam, prm)
    lists = oracle.build_lists(proj, cam)
    fwd = oracle.render_fwd(proj, lists, cam, prm)
    img, Tf, Hm, last = _brute_force(proj, cam, prm)
    assert np.abs(fwd["image"] - img).max() < 1e-13
    assert np.abs(fwd["final_T"] - Tf).max() < 1e-13
    assert np.abs(fwd["entropy"] - Hm).max() < 1e-13
    assert (fwd["last"] == last).all()


def test_equal_depths_blend_in_id_order():
    """Reading c6: Gaussians whose FP32 depths are equal are blended in
    ascending id order.  Five Gaussians at the same camera depth (z = 4
    exactly under the identity camera), of different colours, so that the
    order changes the image; listed in reverse x order so that a sort on
    position would disagree."""
    n = 5
    x = np.array([0.04, 0.03, 0.02, 0.01, 0.0])
    scene = {"means": np.stack([x, np.zeros(n), np.full(n, 4.0)], 1).astype(np.float32),
             "log_scales": np.full((n, 3), -2.5, np.float32),
             "quats": np.tile(np.array([1.0, 0, 0, 0], np.float32), (n, 1)),
             "opacity_logits": np.full(n, 0.5, np.float32),
             "sh": np.zeros((n, 16, 3), np.float32), "sh_degree": 0}
    for i in range(n):
        scene["sh"][i, 0, i % 3] = 1.5
    cam = scenes.camera(48, 40, 48.0)
    prm = scenes.params()
    proj = oracle.preprocess(scene, cam, prm)
    assert (proj["depth"].astype(np.float32) == np.float32(4.0)).all()
    lists = oracle.build_lists(proj, cam)
    ts, ids = lists
    for t in range(len(ts) - 1):
        seg = ids[ts[t]:ts[t + 1]]
        assert list(seg) == sorted(seg)
    assert max(np.diff(ts)) == n  # every Gaussian shares at least one tile
    fwd = oracle.render_fwd(proj, lists, cam, prm)
    img, Tf, Hm, last = _brute_force(proj, cam, prm)
    assert np.abs(fwd["image"] - img).max() < 1e-13
    assert (fwd["last"] == last).all()
    # blending in the reverse order gives a different image: the order is seen
    rev = (ts, np.concatenate([ids[ts[t]:ts[t + 1]][::-1] for t in range(len(ts) - 1)]))
    other = oracle.render_fwd(proj, rev, cam, prm)
    assert np.abs(other["image"] - img).max() > 1e-3


# --------------------------------------------------------------------------
# Gradients: central finite differences of the whole FP64 loss
# --------------------------------------------------------------------------

def _loss_and_state(scene, cams, targets, prm):
    L, views, _, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA, with_grad=False)
    ints = [np.concatenate([v["proj"]["rect"].ravel(), v["fwd"]["last"].ravel(),
                            v["fwd"]["nblend"].ravel(), v["fwd"]["neval"].ravel(),
                            v["proj"]["clamped"].ravel()]) for v in views]
    return L, ints


def _fd_check(scene, cams, targets, prm, rel_tol=2e-6):
    L0, grads, _ = None, None, None
    L0, views, grads, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA)
    margins = min(v["fwd"]["margin"].min() for v in views)
    assert margins > 1e-4, "scene too close to a threshold for finite differences"
    checked = skipped = 0
    worst = 0.0
    for key in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = scene[key]
        K = (scene["sh_degree"] + 1) ** 2
        idxs = list(np.ndindex(arr.shape))
        if key == "sh":
            idxs = [ix for ix in idxs if ix[1] < K]
        for ix in idxs:
            x0 = float(arr[ix])
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            ints = []
            for s in (+1, -1):
                sc = {k: (np.array(v, np.float64) if isinstance(v, np.ndarray) else v)
                      for k, v in scene.items()}
                sc[key][ix] = x0 + s * h
                Ls, ii = _loss_and_state(sc, cams, targets, prm)
                vals.append(Ls)
                ints.append(ii)
            if any((a != b).any() for a, b in zip(ints[0], ints[1])):
                skipped += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[key][ix]
            err = abs(fd - an)
            tol = rel_tol * max(abs(fd), abs(an)) + 1e-9
            worst = max(worst, err / (abs(fd) + 1e-12))
            assert err <= tol, (key, ix, fd, an)
            checked += 1
    assert skipped <= 0.05 * (checked + skipped)
    return checked


@pytest.mark.parametrize("seed,deg", [(0, 0), (1, 3), (2, 3)])
def test_full_gradient_matches_finite_differences(seed, deg):
    scene, cams, targets, prm = scenes.tiny_scene(6, seed=seed, width=32, height=32,
                                                  sh_degree=deg)
    assert _fd_check(scene, cams, targets, prm) > 50


def test_full_gradient_matches_finite_differences_8px_tiles():
    scene, cams, targets, prm = scenes.tiny_scene(6, seed=4, width=32, height=32, sh_degree=1)
    prm["tile"] = 8
    assert _fd_check(scene, cams, targets, prm) > 50


def test_rect_8px_tiles_from_mean_and_radius(cfg1):
    """With 8-pixel tiles the rect is the range of 8-pixel tiles that the
    square [mean - r, mean + r] meets, clamped to the grid (the 3-sigma
    rule of Sec. 3 with the tile side of the paper's runs), and it lies
    inside the 16-pixel rect at twice the resolution."""
    scene, cams, targets, prm, proj16, lists, fwd = cfg1
    cam = cams[0]
    prm8 = dict(prm, tile=8)
    proj8 = oracle.preprocess(scene, cam, prm8)
    TX, TY = oracle.tile_grid(cam, prm8)
    assert (TX, TY) == ((cam["width"] + 7) // 8, (cam["height"] + 7) // 8)
    ok = (proj8["tiles"] > 0) & (proj8["boundary"] == 0)
    mx, my = proj8["P9"][ok, 0], proj8["P9"][ok, 1]
    r = proj8["radius"][ok].astype(np.float64)
    exp = np.stack([np.clip(np.floor((mx - r) / 8), 0, TX), np.clip(np.floor((my - r) / 8), 0, TY),
                    np.clip(np.floor((mx + r) / 8) + 1, 0, TX),
                    np.clip(np.floor((my + r) / 8) + 1, 0, TY)], 1).astype(np.int64)
    assert (proj8["rect"][ok] == exp).all()
    # the radius and the projected attributes do not depend on the tiling
    assert (proj8["radius"] == proj16["radius"]).all()
    assert np.array_equal(proj8["P9"], proj16["P9"])
    both = ok & (proj16["boundary"] == 0) & (proj16["tiles"] > 0)
    r8, r16 = proj8["rect"][both], proj16["rect"][both]
    assert (r8[:, :2] >= 2 * r16[:, :2]).all() and (r8[:, 2:] <= 2 * r16[:, 2:]).all()
    # lists: every Gaussian in exactly tiles_touched 8-pixel lists
    ts, ids = oracle.build_lists(proj8, cam)
    assert len(ts) == TX * TY + 1
    assert (np.bincount(ids, minlength=proj8["tiles"].size) == proj8["tiles"]).all()


def test_gradient_fd_rotated_camera_and_fov_clamp():
    """A rotated camera, and one wide Gaussian whose mean lies outside the
    clamped field of view (x/z clamp active) but whose footprint still
    reaches the image."""
    scene, _, _, prm = scenes.tiny_scene(5, seed=4, width=32, height=32, sh_degree=1)
    pos = np.array([0.2, -0.1, -0.3])
    cam = scenes.camera(32, 32, 32.0, scenes.look_at(pos, (0.0, 0.0, 3.0)), pos)
    # Gaussian 0: far to the side, large: x/z = 0.9 > 1.3 * 16/32
    wtc = cam["world_to_cam"].astype(np.float64)
    Rw = wtc[:, :3]
    p_cam = np.array([2.7, 0.0, 3.0])
    scene["means"][0] = (Rw.T @ (p_cam - wtc[:, 3])).astype(np.float32)
    scene["log_scales"][0] = [-0.5, -0.7, -0.6]
    targets = scenes.noise_targets([cam], 9)
    proj = oracle.preprocess(scene, cam, prm)
    assert proj["tiles"][0] > 0
    assert _fd_check(scene, [cam], targets, prm) > 40


def test_render_bwd_against_fd_of_2d_attributes(cfg1):
    """The compositing gradient alone (Sec. 4.4 closed forms + Suppl. C chain)
    against central differences in the 2D attributes of a small view."""
    scene, cams, targets, prm = scenes.tiny_scene(7, seed=11, width=32, height=32)
    cam = cams[0]
    proj = oracle.preprocess(scene, cam, prm)
    lists = oracle.build_lists(proj, cam)
    fwd = oracle.render_fwd(proj, lists, cam, prm)
    L, dC, dH = oracle.loss(fwd["image"], fwd["entropy"], targets[0], scenes.GAMMA)
    g9 = oracle.render_bwd(proj, lists, cam, prm, dC, dH)
    for i in range(7):
        if proj["tiles"][i] == 0:
            continue
        for k in range(9):
            h = 1e-6 * max(1.0, abs(proj["P9"][i, k]))
            Ls = []
            for s in (1, -1):
                p2 = dict(proj)
                p2["P9"] = proj["P9"].copy()
                p2["P9"][i, k] += s * h
                f2 = oracle.render_fwd(p2, lists, cam, prm)
                # the L1 sign pattern and decisions must not move
                assert (f2["last"] == fwd["last"]).all()
                Ls.append(oracle.loss(f2["image"], f2["entropy"], targets[0], scenes.GAMMA)[0])
            fd = (Ls[0] - Ls[1]) / (2 * h)
            assert fd == pytest.approx(g9[i, k], rel=1e-5, abs=1e-9), (i, k)


# --------------------------------------------------------------------------
# Scale reset (Sec. 4.2) and loss (Sec. 3, Sec. 4.3)
# --------------------------------------------------------------------------

def test_scale_reset_multiplies_scales():
    rng = np.random.default_rng(0)
    ls = rng.normal(-4, 1, 300).astype(np.float32)
    for zeta in (0.2, 0.5, 0.9):
        out = oracle.scale_reset(ls, zeta)
        ref = zeta * np.exp(ls.astype(np.float64))
        assert np.abs(np.exp(out) / ref - 1).max() < 4 * np.finfo(np.float64).eps


def test_loss_definition():
    rng = np.random.default_rng(0)
    img = rng.random((5, 7, 3))
    ent = rng.random((5, 7))
    tgt = rng.random((5, 7, 3)).astype(np.float32)
    L, dC, dH = oracle.loss(img, ent, tgt, 0.015, 0.5)
    M = 35
    ref = 0.5 * (np.abs(img - tgt).sum() / (3 * M) + 0.015 * ent.sum() / M)
    assert L == pytest.approx(ref, rel=1e-14)
    assert dC == pytest.approx(0.5 * np.sign(img - tgt) / (3 * M), rel=1e-15)
    assert dH == pytest.approx(np.full((5, 7), 0.5 * 0.015 / M), rel=1e-15)


def test_l1_gradient_is_zero_where_image_equals_target():
    """Reading c15: sign(0) = 0, so a pixel channel that equals its target
    contributes no L1 gradient (the subgradient the definition picks)."""
    rng = np.random.default_rng(1)
    tgt = rng.random((4, 6, 3)).astype(np.float32)
    img = tgt.astype(np.float64).copy()
    img[:2] += 0.1  # rows 0-1 above the target, rows 2-3 equal to it
    _, dC, _ = oracle.loss(img, np.zeros((4, 6)), tgt, 0.015, 1.0)
    assert (dC[2:] == 0).all()
    assert np.allclose(dC[:2], 1.0 / (3 * 24), rtol=1e-15)


def test_views_average_per_view_means():
    """Reading c4: with several views the loss is the mean over views of each
    view's own pixel means (not one mean over the pooled pixels), and so are
    the gradients: two views of different sizes give the average of the two
    single-view results."""
    scene = scenes.box_scene(300, seed=4)
    cams = scenes.yaw_cameras([(48, 32), (24, 40)], [0.0, 6.0])
    targets = scenes.noise_targets(cams, 3)
    prm = scenes.params()
    L2, _, g2, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA)
    La, _, ga, _ = oracle.step(scene, cams[:1], targets[:1], prm, scenes.GAMMA)
    Lb, _, gb, _ = oracle.step(scene, cams[1:], targets[1:], prm, scenes.GAMMA)
    assert L2 == pytest.approx(0.5 * (La + Lb), rel=1e-13)
    # the pooled mean would weight the larger view by its pixel share instead
    pooled = (48 * 32 * La + 24 * 40 * Lb) / (48 * 32 + 24 * 40)
    assert abs(L2 - pooled) > 1e-6 * abs(L2)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        want = 0.5 * (np.asarray(ga[k]) + np.asarray(gb[k]))
        assert np.allclose(np.asarray(g2[k]), want, rtol=1e-11, atol=1e-15), k


def test_negative_colour_clamps_to_zero_and_masks_its_gradient():
    """Reading c9: rgb = Y00 sh0 + 0.5 is clamped below at 0.  A Gaussian
    whose red DC term makes red negative adds no red to the image and gets an
    exact zero gradient on that coefficient, while its green coefficient
    (unclamped) gets the chain-rule value, matched by a central difference."""
    y00 = 1 / (2 * math.sqrt(math.pi))
    sh0 = (-1.0 / y00, 0.3 / y00, 0.2 / y00)  # rgb = (-0.5, 0.8, 0.7)
    scene = _one((0.0, 0.0, 3.0), [math.log(0.1)] * 3, (1.0, 0.0, 0.0, 0.0), 1.0, sh0=sh0)
    cam = scenes.camera(32, 32, 32.0)
    prm = scenes.params()
    target = [np.full((32, 32, 3), 0.25, np.float32)]
    L, views, g, _ = oracle.step(scene, [cam], target, prm, scenes.GAMMA)
    img = views[0]["fwd"]["image"]
    assert (img[..., 0] == 0).all() and img[..., 1].max() > 0.1
    assert g["sh"][0, 0, 0] == 0.0 and abs(g["sh"][0, 0, 1]) > 1e-4
    h = 1e-4
    for ch, want in ((1, g["sh"][0, 0, 1]), (0, 0.0)):
        vals = []
        for sg in (1, -1):
            sc = {k: (np.array(v, np.float64) if isinstance(v, np.ndarray) else v)
                  for k, v in scene.items()}
            sc["sh"][0, 0, ch] += sg * h
            vals.append(oracle.step(sc, [cam], target, prm, scenes.GAMMA, with_grad=False)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - want) <= 1e-6 * max(abs(want), 1e-3), (ch, fd, want)


def test_fov_clamp_linearises_at_the_clamped_direction():
    """Outside the clamped field of view the EWA Jacobian is the pinhole
    Jacobian at the camera-space point whose x/z (y/z) is clamped to
    fov_clamp * (W/2)/fx ((H/2)/fy); the 2D mean itself is not clamped."""
    cam = scenes.camera(64, 48, 64.0)
    prm = scenes.params()
    lim_x = float(np.float32(1.3)) * 32 / 64.0
    for mu in ([2.4, 0.3, 3.0], [-2.7, -0.2, 3.5]):
        sc = _one(mu, [-0.3, -0.9, -0.6], (0.9, 0.2, -0.3, 0.1), 0.0)
        proj = oracle.preprocess(sc, cam, prm)
        X = sc["means"][0].astype(np.float64)
        Xc = X.copy()
        Xc[0] = np.sign(X[0]) * lim_x * X[2]
        Jn = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            Jn[:, k] = (_pinhole(cam, Xc + e) - _pinhole(cam, Xc - e)) / 2e-6
        qq = sc["quats"][0].astype(np.float64)
        R = _rot_scipy(qq / np.linalg.norm(qq))
        S = np.diag(np.exp(sc["log_scales"][0].astype(np.float64)))
        S2 = Jn @ R @ S @ S @ R.T @ Jn.T + float(np.float32(0.3)) * np.eye(2)
        K = np.linalg.inv(S2)
        P9 = proj["P9"][0]
        assert P9[0:2] == pytest.approx(_pinhole(cam, X), rel=1e-12)
        assert P9[[2, 3, 4]] == pytest.approx([K[0, 0], K[0, 1], K[1, 1]], rel=1e-6)


# --------------------------------------------------------------------------
# D-SSIM term of L_base (Sec. 3 Eq. base; SSIM as in 3DGS)
# --------------------------------------------------------------------------

def _ssim_scipy(x, y):
    """Textbook SSIM with scipy's 2D correlation for every window sum:
    mu = G * x, sigma^2 = G * x^2 - mu^2, sigma_xy = G * (x y) - mu_x mu_y,
    zero fill outside the image."""
    from scipy.signal import correlate2d
    k = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    G = np.outer(k, k) / k.sum() ** 2
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    vals = []
    for ch in range(3):
        a, b = x[..., ch], y[..., ch].astype(np.float64)
        f = lambda z: correlate2d(z, G, mode="same", boundary="fill", fillvalue=0.0)
        mx, my = f(a), f(b)
        sxx, syy, sxy = f(a * a) - mx * mx, f(b * b) - my * my, f(a * b) - mx * my
        vals.append(((2 * mx * my + c1) * (2 * sxy + c2)) /
                    ((mx * mx + my * my + c1) * (sxx + syy + c2)))
    return float(np.mean(vals))


@pytest.mark.parametrize("shape", [(9, 11), (32, 17), (40, 40)])
def test_ssim_matches_textbook_form(shape):
    rng = np.random.default_rng(shape[0])
    x = rng.random(shape + (3,))
    y = rng.random(shape + (3,)).astype(np.float32)
    # correlated pair too (high SSIM), where the variance forms differ most
    z = np.clip(x + rng.normal(0, 0.02, x.shape), 0, 1)
    for a, b in ((x, y), (z, x.astype(np.float32))):
        assert oracle.ssim(a, b) == pytest.approx(_ssim_scipy(a, b), abs=1e-12)


def test_ssim_identity_symmetry_and_constant_images():
    rng = np.random.default_rng(1)
    x = rng.random((20, 24, 3))
    xs = x.astype(np.float32).astype(np.float64)
    s, g = oracle.ssim(xs, xs.astype(np.float32), with_grad=True)
    assert s == pytest.approx(1.0, abs=1e-14) and np.abs(g).max() < 1e-14
    y = rng.random((20, 24, 3)).astype(np.float32)
    assert oracle.ssim(xs, y) == pytest.approx(oracle.ssim(y.astype(np.float64),
                                                             xs.astype(np.float32)), abs=1e-14)
    # constant images a, b: away from the border every window sees no
    # variance, S = (2ab + C1) / (a^2 + b^2 + C1); the textbook form agrees
    a = np.full((30, 30, 3), 0.7)
    b = np.full((30, 30, 3), 0.2, np.float32)
    assert oracle.ssim(a, b) == pytest.approx(_ssim_scipy(a, b), abs=1e-12)


def test_ssim_gradient_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.random((10, 13, 3))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1).astype(np.float32)
    s, g = oracle.ssim(x, y, with_grad=True)
    # central differences, h = 1e-5: truncation O(h^2) and rounding ~1e-16 / h,
    # both far below the 1e-9 floor; typical entries are 1e-5 .. 1e-3
    h = 1e-5
    for idx in [(0, 0, 0), (4, 6, 1), (9, 12, 2), (5, 0, 0), (2, 9, 1)] + \
               [tuple(int(rng.integers(0, n)) for n in x.shape) for _ in range(20)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.ssim(xp, y) - oracle.ssim(xm, y)) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-9)


def test_loss_base_reduces_and_differentiates():
    rng = np.random.default_rng(3)
    img = rng.random((12, 14, 3))
    ent = rng.random((12, 14))
    tgt = rng.random((12, 14, 3)).astype(np.float32)
    L0, d0, h0 = oracle.loss(img, ent, tgt, 0.015)
    L, dC, dH = oracle.loss_base(img, ent, tgt, 0.015, 0.0)
    assert L == pytest.approx(L0, abs=1e-15) and np.array_equal(dC, d0) and np.array_equal(dH, h0)
    lam = 0.2
    L, dC, dH = oracle.loss_base(img, ent, tgt, 0.015, lam)
    L1 = np.abs(img - tgt).mean()
    assert L == pytest.approx((1 - lam) * L1 + lam * (1 - oracle.ssim(img, tgt)) +
                              0.015 * ent.mean(), abs=1e-14)
    h = 1e-7
    for idx in [(0, 0, 0), (6, 7, 1), (11, 13, 2)]:
        ip, im = img.copy(), img.copy()
        ip[idx] += h
        im[idx] -= h
        fd = (oracle.loss_base(ip, ent, tgt, 0.015, lam)[0] -
              oracle.loss_base(im, ent, tgt, 0.015, lam)[0]) / (2 * h)
        assert fd == pytest.approx(dC[idx], rel=1e-5, abs=1e-9)


# --------------------------------------------------------------------------
# Regression: the oracle's outputs on two small scenes, as stored by
# tests/golden/make_oracle_regression.py (which calls only the oracle).  The
# pins above tie the oracle to the paper; this ties it to itself over time, so
# that a change of its arithmetic is seen and has to be justified.
# --------------------------------------------------------------------------

def test_oracle_outputs_unchanged_on_stored_cases():
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    stored = json.load(open(os.path.join(here, "oracle_regression_tiny.json")))
    for c in stored["cases"]:
        scene, cams, targets, prm = scenes.tiny_scene(8, seed=c["seed"], width=40, height=36,
                                                      sh_degree=c["sh_degree"])
        prm["tile"] = c["tile"]
        L, views, grads, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA)
        f = views[0]["fwd"]
        assert L == pytest.approx(c["loss"], rel=1e-12)
        assert float(np.sum(f["image"])) == pytest.approx(c["image_sum"], rel=1e-12)
        assert float(np.sum(f["final_T"])) == pytest.approx(c["final_T_sum"], rel=1e-12)
        assert float(np.sum(f["entropy"])) == pytest.approx(c["entropy_sum"], rel=1e-12)
        assert int(np.sum(f["last"])) == c["last_sum"]
        y, x = c["brightest_pixel"]
        assert list(f["image"][y, x]) == pytest.approx(c["brightest_rgb"], rel=1e-12)
        K = (c["sh_degree"] + 1) ** 2
        for k, want in c["grads"].items():
            got = np.asarray(grads[k])
            got = (got[:, :K] if k == "sh" else got).ravel()
            np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-15, err_msg=k)
