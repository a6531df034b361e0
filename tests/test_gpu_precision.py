"""Reduced-precision storage: BF16 geometry and opacity, FP8-E4M3 SH, per-channel FP32
scales, all arithmetic in FP32.

The GPU render of the quantised scene is compared with the FP64 oracle run on the
same dequantised values (value = fl32(float(stored) * scale)): tile lists
bit-exact, max |pixel| <= 1e-4 on non-ambiguous pixels, PSNR >= 60 dB over all
pixels.  The quantisation error itself (against the FP32 scene) is reported,
not barred.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


@pytest.fixture(scope="module")
def small_q():
    rng = np.random.default_rng(61)
    scene = scenes.make_hier_scene(rng, 8000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 3)
    q = scenes.quantize_scene(scene)
    return scene, motion, q, oracle.dequantize(q, scene)


def _gpu(gc, gs, motion, frame, cam, mask, saved=None):
    r = gc.Renderer(0)
    saved = gc.Saved(r)
    mo = gc.MotionFrame.from_motion(motion, frame) if motion is not None else None
    img = r.forward(gs, mo, mask, cam, saved)
    torch.cuda.synchronize()
    ranges, ids = r.tile_lists(saved)
    return r, saved, mo, img, ids.cpu().numpy()


@pytest.mark.parametrize("mask", [0b111111, 0b000011])
def test_quantised_matches_oracle_on_dequantised(gc, small_q, mask):
    scene, motion, q, deq = small_q
    cam = scenes.orbit_camera(0.4, 4.0, 232, 168)
    gsq = gc.GaussianSet.from_quantized(q, scene)
    _, _, _, img, ids = _gpu(gc, gsq, motion, 2, cam, mask)
    ref = oracle.render(deq, motion, 2, cam, oracle.default_options(), mask)
    tl = oracle.tile_lists(ref["bins"], cam)
    assert np.array_equal(ids, tl["gauss_of_entry"])
    g = img.cpu().numpy().astype(np.float64)
    ok = ~ref["ambiguous"]
    assert np.abs(g - ref["image"]).max(axis=0)[ok].max() <= 1e-4
    assert psnr(g, ref["image"]) >= 60.0
    # the FP32 renderer on the dequantised values gives the same image bit for bit
    gsd = gc.GaussianSet.from_scene(deq)
    _, _, _, img32, _ = _gpu(gc, gsd, motion, 2, cam, mask)
    assert torch.equal(img, img32)


def test_quantisation_error_is_reported_not_barred(gc, small_q):
    scene, motion, q, deq = small_q
    cam = scenes.orbit_camera(0.4, 4.0, 232, 168)
    _, _, _, a, _ = _gpu(gc, gc.GaussianSet.from_quantized(q, scene), motion, 1, cam, 63)
    _, _, _, b, _ = _gpu(gc, gc.GaussianSet.from_scene(scene), motion, 1, cam, 63)
    p = psnr(a.cpu().numpy(), b.cpu().numpy())
    assert p > 20.0   # sanity: the quantised scene is still the same scene
    print(f"quantisation PSNR vs FP32 scene: {p:.2f} dB")


def test_quantised_backward_matches_oracle(gc, small_q):
    scene, motion, q, deq = small_q
    cam = scenes.orbit_camera(0.9, 4.0, 160, 120)
    gsq = gc.GaussianSet.from_quantized(q, scene)
    r, saved, mo, img, _ = _gpu(gc, gsq, motion, 1, cam, 63)
    ref = oracle.render(deq, motion, 1, cam, oracle.default_options(), 63)
    up = np.random.default_rng(1).normal(0, 1, (3, cam.height, cam.width)) * (~ref["ambiguous"])[None]
    up = up.astype(np.float32)
    g = r.backward(saved, gsq, mo, torch.from_numpy(up).cuda())
    og = oracle.grad(deq, motion, 1, cam, oracle.default_options(), up.astype(np.float64), 63, bins=ref["bins"])
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "group_q", "group_t"):
        a = g[k].cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(a - og[k]) / np.linalg.norm(og[k])
        assert rel <= 1e-4, (k, rel)


def test_prec4k_at_scale(gc):
    """1M Gaussians, 3840x2160, BF16/FP8 storage (about 2.3e8 tile entries): the lists of
    256 sampled tiles bit-exact, 2,048 sampled pixels against the oracle on the
    dequantised scene."""
    w = scenes.prec4k()
    cam = w.cameras[0]
    q = scenes.quantize_scene(w.scene)
    deq = oracle.dequantize(q, w.scene)
    gsq = gc.GaussianSet.from_quantized(q, w.scene)
    r = gc.Renderer(0)
    saved = gc.Saved(r)
    img = r.forward(gsq, gc.MotionFrame.from_motion(w.motion, 1), 63, cam, saved)
    ranges, ids = r.tile_lists(saved)
    opts = oracle.default_options()
    bins = oracle.bin_f32(deq, w.motion, 1, cam, opts, 63)
    rng = np.random.default_rng(12)
    n_tiles = ranges.shape[0]
    sample = np.unique(np.concatenate([rng.choice(n_tiles, 224, replace=False),
                                       n_tiles // 2 + np.arange(-16, 16)]))
    rg = ranges.cpu().numpy()
    for t in sample:
        got = ids[int(rg[t, 0]):int(rg[t, 1])].cpu().numpy()
        assert np.array_equal(got, oracle.tile_list(bins, cam, int(t))), t
    del ids
    pix = scenes.sample_pixels(11, cam.width, cam.height, 2048)
    ref = oracle.render(deq, w.motion, 1, cam, opts, 63, pixels=pix, bins=bins)
    g = img.cpu().numpy()[:, pix[:, 1], pix[:, 0]].T.astype(np.float64)
    ok = ~ref["ambiguous"]
    err = np.abs(g - ref["image"]).max(axis=1)
    assert err[ok].max() <= 1e-4
    assert psnr(g, ref["image"]) >= 60.0
