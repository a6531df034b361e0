"""Pins of the oracle's compositing (Eq. 2 / Eq. 4) and of its invariants.

Closed forms (one isotropic Gaussian, two Gaussians on the axis), special
cases (zero opacity, the transmittance stop), the back-to-front form of the
compositing sum, invariance under permutation of the input, layer-prefix
equivalence (progressive rendering, Eq. 4) and the motion identities
(Sec. 3.2).
"""
import math

import numpy as np
import pytest

from synth import scenes

Y00 = 0.5 / math.sqrt(math.pi)


def _scene(means, log_scales, logits, rgb, quats=None, gid=None, n_groups=1):
    n = len(means)
    sh = np.zeros((n, 1, 3), np.float32)
    sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / Y00
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    return scenes.Scene(np.asarray(means, np.float32), np.asarray(log_scales, np.float32), q,
                        np.asarray(logits, np.float32), sh,
                        np.zeros(n, np.int32) if gid is None else np.asarray(gid, np.int32),
                        np.array([0, n], np.int64), 0, n_groups)


def _cam(W=64, H=48, cx=None, cy=None, eye=(0, 0, -3)):
    c = scenes.look_at_camera(eye, (0, 0, 0), W, H)
    if cx is not None:
        c.cx = float(np.float32(cx))  # camera values are FP32 on both sides
    if cy is not None:
        c.cy = float(np.float32(cy))
    return c


def test_single_isotropic_gaussian_closed_form(oracle_lib):
    cam = _cam(64, 48, cx=31.3, cy=22.8)
    bg = (0.1, 0.2, 0.3)
    opts = oracle_lib.default_options(bg=bg)
    ls, logit, rgb = -2.2, 0.7, np.array([0.8, 0.4, 0.1])
    sc = _scene([[0, 0, 0]], [[ls] * 3], [logit], [rgb])
    r = oracle_lib.render(sc, None, 0, cam, opts)
    s = math.exp(np.float32(ls))
    var = (cam.fx * s / 3.0) ** 2 + float(np.float32(0.3))
    rad = math.ceil(3 * math.sqrt(var))
    assert abs(3 * math.sqrt(var) - round(3 * math.sqrt(var))) > 1e-3
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    rgb32 = (np.float32((rgb - 0.5) / Y00).astype(np.float64) * Y00 + 0.5)
    img = r["image"]
    bgv = np.array(bg, np.float32).astype(np.float64)
    for py in range(cam.height):
        for px in range(cam.width):
            dx, dy = px + 0.5 - cam.cx, py + 0.5 - cam.cy
            a = min(0.99, o * math.exp(-0.5 * (dx * dx + dy * dy) / var))
            if abs(dx) <= rad and abs(dy) <= rad and a >= 1 / 255:
                expect = rgb32 * a + bgv * (1 - a)
            else:
                expect = bgv
            assert np.allclose(img[:, py, px], expect, atol=1e-12, rtol=0), (px, py)


def test_zero_opacity_gives_background(oracle_lib):
    w = scenes.tiny(n=300)
    sc = w.scene
    sc.opacity_logits[:] = -1000.0
    bg = (0.25, 0.5, 0.75)
    r = oracle_lib.render(sc, None, 0, w.cameras[0], oracle_lib.default_options(bg=bg))
    assert np.array_equal(r["image"], np.broadcast_to(np.array(bg, np.float32).astype(np.float64)[:, None, None],
                                                      r["image"].shape))
    assert r["n_blended"].max() == 0


def test_two_gaussians_on_axis(oracle_lib):
    cam = _cam(33, 33)  # centre pixel (16, 16) has its centre exactly at (cx, cy)
    bg = (0.05, 0.1, 0.15)
    opts = oracle_lib.default_options(bg=bg)
    c1, c2 = np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.7, 0.3])
    sc = _scene([[0, 0, 0.5], [0, 0, 0]], [[-2.5] * 3, [-2.0] * 3], [0.3, -0.4], [c2, c1])
    r = oracle_lib.render(sc, None, 0, cam, opts)
    # index 1 is nearer (z = 3) than index 0 (z = 3.5)
    o1 = 1 / (1 + math.exp(-float(np.float32(-0.4))))
    o2 = 1 / (1 + math.exp(-float(np.float32(0.3))))
    k1 = np.float32((c1 - 0.5) / Y00).astype(np.float64) * Y00 + 0.5
    k2 = np.float32((c2 - 0.5) / Y00).astype(np.float64) * Y00 + 0.5
    bgv = np.array(bg, np.float32).astype(np.float64)
    expect = k1 * o1 + k2 * o2 * (1 - o1) + bgv * (1 - o1) * (1 - o2)
    assert np.allclose(r["image"][:, 16, 16], expect, atol=1e-13, rtol=0)
    assert r["n_blended"][16, 16] == 2
    assert abs(r["T"][16, 16] - (1 - o1) * (1 - o2)) < 1e-14


def test_transmittance_stop_boundary(oracle_lib):
    """alpha = 0.99 twice leaves T = (1 - 0.99)^2, which is 1.0000000000000018e-4 in FP64:
    not below 1e-4, so the second is blended and the third stops the pixel."""
    cam = _cam(33, 33)
    opts = oracle_lib.default_options()
    cols = [np.array([0.9, 0.1, 0.1]), np.array([0.1, 0.9, 0.1]), np.array([0.1, 0.1, 0.9])]
    sc = _scene([[0, 0, 0], [0, 0, 0.5], [0, 0, 1.0]], [[-2.0] * 3] * 3, [12.0] * 3, cols)
    r = oracle_lib.render(sc, None, 0, cam, opts)
    k = [np.float32((c - 0.5) / Y00).astype(np.float64) * Y00 + 0.5 for c in cols]
    a = 0.99
    assert (1 - a) * (1 - a) >= 1e-4
    expect = k[0] * a + k[1] * a * (1 - a)
    assert r["n_blended"][16, 16] == 2
    assert np.allclose(r["image"][:, 16, 16], expect, atol=1e-14, rtol=0)
    assert r["ambiguous"][16, 16]  # the FP32 renderer may stop one step earlier


def _low_opacity_scene(n, seed, deg=0):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.6, 0.6, (n, 3)).astype(np.float32)
    ls = rng.normal(-2.6, 0.3, (n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(-2.5, 0.5, n).astype(np.float32)
    K = (deg + 1) ** 2
    sh = rng.normal(0, 0.3, (n, K, 3)).astype(np.float32)
    return scenes.Scene(means, ls, q.astype(np.float32), logits, sh, np.zeros(n, np.int32),
                        np.array([0, n], np.int64), deg, 1)


def test_back_to_front_equals_front_to_back(oracle_lib):
    sc = _low_opacity_scene(120, 11, deg=1)
    cam = _cam(24, 20)
    bg = (0.3, 0.1, 0.2)
    opts = oracle_lib.default_options(bg=bg)
    r = oracle_lib.render(sc, None, 0, cam, opts)
    b = r["bins"]
    assert r["T"].min() > 1e-3  # no stop on this scene
    geo = [oracle_lib.geom(sc, None, 0, cam, opts, j) if b["visible"][j] else None for j in range(sc.n)]
    order = [j for j in np.lexsort((b["sel"], b["depth"])) if b["visible"][j]]
    bgv = np.array(bg, np.float32).astype(np.float64)
    for py in range(cam.height):
        for px in range(cam.width):
            layers = []
            for j in order:
                x0, x1, y0, y1 = b["rect"][j]
                if not (x0 <= px <= x1 and y0 <= py <= y1):
                    continue
                g = geo[j]
                dx, dy = px + 0.5 - g["u"], py + 0.5 - g["v"]
                ca, cb, cc = g["conic"]
                pw = -0.5 * (ca * dx * dx + cc * dy * dy) - cb * dx * dy
                if pw > 0:
                    continue
                a = min(0.99, g["opacity"] * math.exp(pw))
                if a < 1 / 255:
                    continue
                layers.append((a, g["rgb"]))
            col = bgv.copy()
            for a, c in reversed(layers):   # back to front: C <- a c + (1 - a) C
                col = a * c + (1 - a) * col
            assert np.allclose(r["image"][:, py, px], col, atol=1e-12, rtol=0), (px, py)


def test_order_invariance(oracle_lib):
    w = scenes.tiny(seed=5, n=400, size=48)
    sc, cam = w.scene, w.cameras[0]
    opts = oracle_lib.default_options()
    r0 = oracle_lib.render(sc, None, 0, cam, opts)
    d = r0["bins"]["depth"][r0["bins"]["visible"] == 1]
    assert len(np.unique(d)) == len(d)  # distinct depths: the order does not depend on indices
    perm = np.random.default_rng(1).permutation(sc.n)
    sp = scenes.Scene(sc.means[perm], sc.log_scales[perm], sc.quats[perm], sc.opacity_logits[perm],
                      sc.sh[perm], sc.group_id[perm], sc.layer_offsets, sc.sh_degree, 1)
    r1 = oracle_lib.render(sp, None, 0, cam, opts)
    assert np.allclose(r0["image"], r1["image"], atol=1e-13, rtol=0)


def _small_hier(n=3000, seed=21, groups=8):
    rng = np.random.default_rng(seed)
    return scenes.make_hier_scene(rng, n, 6, 3, groups), scenes.random_motion(rng, groups, 4)


def test_level_equals_prefix_render(oracle_lib):
    sc, mo = _small_hier()
    cam = scenes.orbit_camera(0.4, 4.0, 64, 40)
    opts = oracle_lib.default_options()
    for level in (1, 3, 6):
        full = oracle_lib.render(sc, mo, 2, cam, opts, scenes.level_mask(level))
        pre = sc.subset(np.arange(sc.layer_offsets[level]))
        alone = oracle_lib.render(pre, mo, 2, cam, opts, 1)
        assert np.array_equal(full["image"], alone["image"])
    # an arbitrary union of layers is the render of that union alone
    mask = 0b101001
    idx = scenes.selected_indices(sc.layer_offsets, mask)
    a = oracle_lib.render(sc, mo, 2, cam, opts, mask)
    b = oracle_lib.render(sc.subset(idx), mo, 2, cam, opts, 1)
    assert np.array_equal(a["image"], b["image"])


def test_identity_motion_is_no_motion(oracle_lib):
    sc, _ = _small_hier(1500)
    cam = scenes.orbit_camera(1.0, 4.0, 48, 48)
    opts = oracle_lib.default_options()
    ident = scenes.identity_motion(sc.n_groups)
    a = oracle_lib.render(sc, None, 0, cam, opts, 63)
    b = oracle_lib.render(sc, ident, 0, cam, opts, 63)
    assert np.array_equal(a["image"], b["image"])


def test_translation_motion_is_pretranslated_scene(oracle_lib):
    sc, mo = _small_hier(1500)
    mo.q[:] = np.array([1, 0, 0, 0], np.float32)
    cam = scenes.orbit_camera(0.2, 4.0, 48, 48)
    opts = oracle_lib.default_options()
    a = oracle_lib.render(sc, mo, 3, cam, opts, 63)
    moved = sc.subset(np.arange(sc.n))
    moved.means = (sc.means + mo.t[3][sc.group_id]).astype(np.float32)
    b = oracle_lib.render(moved, None, 0, cam, opts, 63)
    assert np.array_equal(a["bins"]["rect"], b["bins"]["rect"])
    assert np.allclose(a["image"], b["image"], atol=1e-6, rtol=0)


def test_rotation_of_isotropic_gaussians_changes_nothing(oracle_lib):
    sc, mo = _small_hier(1500)
    sc.log_scales[:] = sc.log_scales[:, :1]          # isotropic
    mo.t[:] = 0.0
    cam = scenes.orbit_camera(0.7, 4.0, 48, 48)
    opts = oracle_lib.default_options()
    a = oracle_lib.render(sc, None, 0, cam, opts, 63)
    b = oracle_lib.render(sc, mo, 3, cam, opts, 63)
    assert np.allclose(a["image"], b["image"], atol=1e-9, rtol=0)


def test_samples_equal_full_frame(oracle_lib):
    w = scenes.tiny(n=500, size=40)
    cam = w.cameras[0]
    opts = oracle_lib.default_options(bg=(0.2, 0.2, 0.2))
    full = oracle_lib.render(w.scene, None, 0, cam, opts)
    pix = scenes.sample_pixels(3, cam.width, cam.height, 200)
    s = oracle_lib.render(w.scene, None, 0, cam, opts, pixels=pix)
    assert np.array_equal(s["image"], full["image"][:, pix[:, 1], pix[:, 0]].T)
    assert np.array_equal(s["T"], full["T"][pix[:, 1], pix[:, 0]])


def test_pixel_square_is_tile_shape_invariant(oracle_lib):
    w = scenes.tiny(n=600, size=256)   # footprints of several pixels
    cam = w.cameras[0]
    imgs = [oracle_lib.render(w.scene, None, 0, cam, oracle_lib.default_options(tile=t))["image"]
            for t in ((16, 16), (8, 32), (32, 8))]
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[0], imgs[2])
    # whole-tile membership (the lineage's rule) does depend on the tile shape
    tiles = [oracle_lib.render(w.scene, None, 0, cam,
                               oracle_lib.default_options(tile=t, membership=1))["image"]
             for t in ((16, 16), (32, 8))]
    assert not np.array_equal(tiles[0], tiles[1])


def test_tile_lists_cover_rectangles(oracle_lib):
    """Without the alpha cull every tile of every rectangle is listed; with it, the lists
    are a subset; lists are depth-ordered either way, and one tile's list equals its
    slice of the full lists."""
    w = scenes.tiny(n=300, size=64)
    cam = w.cameras[0]
    bc = oracle_lib.bin_f32(w.scene, None, 0, cam, oracle_lib.default_options(), 1)
    tlc = oracle_lib.tile_lists(bc, cam)
    b = oracle_lib.bin_f32(w.scene, None, 0, cam, oracle_lib.default_options(alpha_cull=0), 1)
    tl = oracle_lib.tile_lists(b, cam)
    full = set(zip(tl["tile_of_entry"].tolist(), tl["gauss_of_entry"].tolist()))
    culled = set(zip(tlc["tile_of_entry"].tolist(), tlc["gauss_of_entry"].tolist()))
    assert culled < full
    for t in range(tlc["n_tiles"]):
        s, e = tlc["ranges"][t]
        assert np.array_equal(tlc["gauss_of_entry"][s:e], oracle_lib.tile_list(bc, cam, t))
    tr = b["trect"][b["visible"] == 1]
    assert len(tl["gauss_of_entry"]) == int(((tr[:, 1] - tr[:, 0] + 1) * (tr[:, 3] - tr[:, 2] + 1)).sum())
    for t in range(tl["n_tiles"]):
        s, e = tl["ranges"][t]
        g = tl["gauss_of_entry"][s:e]
        d = b["depth"][g]  # selection = identity for one layer
        assert np.all(np.diff(d) >= 0)
