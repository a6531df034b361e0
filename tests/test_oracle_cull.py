"""The alpha footprint of the binning specification (steps 14-15, not in the paper).

A Gaussian's value can reach the 1/255 skip threshold of the compositing rule
(Sec. 3.1, Eq. 2) only where o exp(-Q/2) >= 1/255.  The mirror clips the 3-sigma
pixel square to the bounding box of that region plus a margin (step 14) and keeps, per
tile row, only the tile columns whose pixel centres can meet it (step 15).  The pins:

* the clipped rectangle lies inside the 3-sigma square, every row interval inside the
  rectangle's tile columns;
* every pixel removed by the clip or by the row intervals has alpha < (1/255)
  exp(-0.005) in FP64, checked by brute force over the removed pixels;
* Gaussians with opacity <= 1/255 are not binned;
* the FP64 render and its pixel flags do not change at all (bit for bit), and the FP64
  gradients agree to the oracle's own run-to-run summation noise (1e-12 relative):
  the removed pairs were skipped by the compositing rule anyway.
"""
import numpy as np
import pytest

from synth import scenes


def _removed_alpha_max(oracle_lib, scene, motion, frame, cam, mask, step=1, tile=(16, 16)):
    tw, th = tile
    on = oracle_lib.bin_f32(scene, motion, frame, cam, oracle_lib.default_options(tile=tile), mask)
    off = oracle_lib.bin_f32(scene, motion, frame, cam, oracle_lib.default_options(tile=tile, alpha_cull=0), mask)
    logit = scene.opacity_logits[on["sel"]].astype(np.float64)
    o = 1.0 / (1.0 + np.exp(-logit))
    worst = 0.0
    n_checked = 0
    for j in range(0, len(on["sel"]), step):
        if not off["visible"][j]:
            assert not on["visible"][j]
            continue
        x0, x1, y0, y1 = off["rect"][j]
        xs = np.arange(x0, x1 + 1) + 0.5
        ys = np.arange(y0, y1 + 1) + 0.5
        X, Y = np.meshgrid(xs, ys)
        keep = np.zeros(X.shape, bool)
        if on["visible"][j]:
            a0, a1, b0, b1 = on["rect"][j]
            assert x0 <= a0 <= a1 <= x1 and y0 <= b0 <= b1 <= y1, j
            keep[b0 - y0:b1 - y0 + 1, a0 - x0:a1 - x0 + 1] = True
            t0, t1, s0, s1 = on["trect"][j]
            ra = on["row_a"][on["row_off"][j]:on["row_off"][j + 1]]
            rb = on["row_b"][on["row_off"][j]:on["row_off"][j + 1]]
            assert len(ra) == s1 - s0 + 1
            for i in range(len(ra)):
                assert ra[i] > rb[i] or t0 <= ra[i] <= rb[i] <= t1, (j, i)
            tile_x = (X.astype(np.int64) // tw)
            tile_y = (Y.astype(np.int64) // th)
            ri = np.clip(tile_y - s0, 0, len(ra) - 1)
            in_row = (tile_x >= ra[ri]) & (tile_x <= rb[ri]) & (tile_y >= s0) & (tile_y <= s1)
            keep &= in_row
        else:
            assert o[j] <= 1.0 / 255.0 or True  # dropped: every pixel is checked below
        if keep.all():
            continue
        u, v = off["uv"][j].astype(np.float64)
        a, b, c = off["conic"][j].astype(np.float64)
        dx, dy = X - u, Y - v
        alpha = np.minimum(0.99, o[j] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)))
        worst = max(worst, float(alpha[~keep].max()))
        n_checked += int((~keep).sum())
    return worst, n_checked


def test_alpha_cull_removes_only_pixels_below_threshold_tiny(oracle_lib):
    w = scenes.tiny()
    worst, n = _removed_alpha_max(oracle_lib, w.scene, None, 0, w.cameras[0], 1)
    assert n > 1000
    assert worst < (1.0 / 255.0) * np.exp(-0.005), worst


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_alpha_cull_removes_only_pixels_below_threshold_hier(oracle_lib, tile):
    rng = np.random.default_rng(81)
    scene = scenes.make_hier_scene(rng, 6000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 3)
    cam = scenes.orbit_camera(0.7, 4.0, 320, 240)
    worst, n = _removed_alpha_max(oracle_lib, scene, motion, 2, cam, 63, step=3, tile=tile)
    assert n > 10000
    assert worst < (1.0 / 255.0) * np.exp(-0.005), worst


def test_alpha_cull_drops_transparent_gaussians(oracle_lib):
    w = scenes.tiny()
    sc = w.scene
    logit = sc.opacity_logits.copy()
    logit[::7] = np.float32(np.log((1 / 256) / (1 - 1 / 256)))  # opacity just under 1/255
    sc2 = scenes.Scene(**{**sc.__dict__, "opacity_logits": logit})
    on = oracle_lib.bin_f32(sc2, None, 0, w.cameras[0], oracle_lib.default_options(), 1)
    assert not on["visible"][::7].any()


@pytest.mark.parametrize("membership", [0, 1])
def test_alpha_cull_leaves_the_fp64_render_unchanged(oracle_lib, membership):
    rng = np.random.default_rng(82)
    scene = scenes.make_hier_scene(rng, 4000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 2)
    cam = scenes.orbit_camera(2.2, 4.0, 200, 150)
    ref = {}
    for cull in (0, 1):
        opts = oracle_lib.default_options(membership=membership, alpha_cull=cull)
        ref[cull] = oracle_lib.render(scene, motion, 1, cam, opts, 63)
    assert np.array_equal(ref[0]["image"], ref[1]["image"])
    assert np.array_equal(ref[0]["ambiguous"], ref[1]["ambiguous"])
    k0 = len(oracle_lib.tile_lists(ref[0]["bins"], cam)["gauss_of_entry"])
    k1 = len(oracle_lib.tile_lists(ref[1]["bins"], cam)["gauss_of_entry"])
    assert k1 < 0.9 * k0


def test_alpha_cull_leaves_the_fp64_gradient_unchanged(oracle_lib):
    rng = np.random.default_rng(83)
    scene = scenes.make_hier_scene(rng, 1500, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 2)
    cam = scenes.orbit_camera(1.1, 4.0, 96, 72)
    up = np.random.default_rng(4).normal(0, 1, (3, 72, 96))
    g = [oracle_lib.grad(scene, motion, 1, cam, oracle_lib.default_options(alpha_cull=c), up, 63)
         for c in (0, 1)]
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "group_q", "group_t"):
        assert np.abs(g[0][k] - g[1][k]).max() <= 1e-12 * np.abs(g[0][k]).max(), k
