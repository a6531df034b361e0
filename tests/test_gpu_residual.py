"""Residual deformation (Sec. 3.2, Eq. 7) on the GPU: per-Gaussian log-scale, opacity-logit
and SH residuals of a frame, added before activation inside the preprocess and the chain
rule.  Bars: tile lists bit-exact against the oracle's FP32 binning mirror with the same
residuals, pixels within 1e-4 of the FP64 oracle on non-ambiguous pixels, gradients within
the backward bars of the oracle's; images, lists and gradients identical bit for bit to the
GPU render of the scene with the residuals added beforehand (one FP32 addition each, as on
the device); the multi-level and batched forms equal the single-level render."""
import numpy as np
import pytest
import torch

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(41)
    scene = scenes.make_hier_scene(rng, 6000, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 4)
    res = scenes.random_residual(6, scene.n, 3, frame=3, ls_sigma=0.05, logit_sigma=0.3, sh_sigma=0.05)
    return scene, motion, res


def _gpu(gc, scene, motion, frame, cam, mask, residual=None, tile=(16, 16), up=None):
    r = gc.Renderer(0, tile=tile, bg=(0.1, 0.2, 0.3))
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, frame, residual=residual)
    saved = gc.Saved(r)
    img = r.forward(gs, mo, mask, cam, saved)
    ranges, ids = r.tile_lists(saved)
    out = {"image": img.cpu().numpy().astype(np.float64), "ranges": ranges.cpu().numpy(), "ids": ids.cpu().numpy()}
    if up is not None:
        g = r.backward(saved, gs, mo, torch.from_numpy(up.astype(np.float32)).cuda())
        out["grads"] = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
def test_residual_forward_matches_oracle_and_pre_added(gc, case, tile):
    scene, motion, res = case
    cam = scenes.orbit_camera(0.9, 4.0, 184, 128)
    mask = scenes.level_mask(6)
    got = _gpu(gc, scene, motion, 2, cam, mask, res, tile)
    opts = oracle.default_options(tile=tile, bg=(0.1, 0.2, 0.3))
    ref = oracle.render(scene, motion, 2, cam, opts, mask, residual=res)
    tiles = oracle.tile_lists(ref["bins"], cam, tile)
    assert np.array_equal(got["ids"], tiles["gauss_of_entry"])
    assert np.array_equal(got["ranges"][:, 1] - got["ranges"][:, 0], tiles["ranges"][:, 1] - tiles["ranges"][:, 0])
    ok = ~ref["ambiguous"]
    assert ok.mean() > 0.95
    assert np.abs(got["image"] - ref["image"]).max(axis=0)[ok].max() <= 1e-4
    # the residual matters, and equals adding it to the scene beforehand (FP32 sums)
    plain = _gpu(gc, scene, motion, 2, cam, mask, None, tile)
    assert np.abs(plain["image"] - got["image"]).max() > 1e-2
    pre = _gpu(gc, scenes.apply_residual(scene, res), motion, 2, cam, mask, None, tile)
    assert np.array_equal(pre["image"], got["image"])
    assert np.array_equal(pre["ids"], got["ids"])


def test_residual_backward_matches_oracle_and_pre_added(gc, case):
    scene, motion, res = case
    cam = scenes.orbit_camera(0.3, 4.0, 128, 96)
    mask = scenes.level_mask(4)
    opts = oracle.default_options(bg=(0.1, 0.2, 0.3))
    ref = oracle.render(scene, motion, 1, cam, opts, mask, residual=res)
    up = np.random.default_rng(2).normal(0, 1, (3, cam.height, cam.width)) * (~ref["ambiguous"])[None]
    up = up.astype(np.float32).astype(np.float64)
    got = _gpu(gc, scene, motion, 1, cam, mask, res, up=up)["grads"]
    want = oracle.grad(scene, motion, 1, cam, opts, up, mask, bins=ref["bins"], residual=res)
    for k in NAMES + ("group_q", "group_t"):
        a, b = got[k], np.asarray(want[k]).reshape(got[k].shape)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-4, k
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-6, k
    pre = _gpu(gc, scenes.apply_residual(scene, res), motion, 1, cam, mask, None, up=up)["grads"]
    for k in NAMES + ("group_q", "group_t"):
        assert np.array_equal(pre[k], got[k]), k


def test_residual_without_group_motion(gc, case):
    scene, _, res = case
    cam = scenes.orbit_camera(0.2, 4.0, 96, 80)
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(None, 0, residual=res)
    img = r.forward(gs, mo, 0b111, cam)
    pre = r.forward(gc.GaussianSet.from_scene(scenes.apply_residual(scene, res)), None, 0b111, cam)
    torch.cuda.synchronize()
    assert torch.equal(img, pre)


def test_residual_levels_and_batch_equal_single(gc, case):
    scene, motion, res = case
    cam = scenes.orbit_camera(1.7, 4.0, 160, 112)
    r = gc.Renderer(0, tile=(8, 32))
    gs = gc.GaussianSet.from_scene(scene)
    frames = [gc.MotionFrame.from_motion(motion, f, residual=scenes.random_residual(6, scene.n, 3, f))
              for f in range(3)]
    singles = {(f, l): r.forward(gs, frames[f], scenes.level_mask(l), cam).clone()
               for f in range(3) for l in (1, 3, 6)}
    imgs = r.levels_forward(gs, frames[2], 6, cam)
    torch.cuda.synchronize()
    for l in (1, 3, 6):
        assert torch.equal(imgs[l - 1], singles[(2, l)]), l
    reqs = [(cam, f, scenes.level_mask(l)) for f in range(3) for l in (1, 3, 6)]
    outs = r.batch_forward(gs, frames, reqs)
    torch.cuda.synchronize()
    for (c, f, m), o in zip(reqs, outs):
        l = {scenes.level_mask(x): x for x in (1, 3, 6)}[m]
        assert torch.equal(o, singles[(f, l)]), (f, l)


def test_backward_refuses_other_residuals(gc, case):
    scene, motion, res = case
    cam = scenes.orbit_camera(0.2, 4.0, 64, 48)
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, 1, residual=res)
    saved = gc.Saved(r)
    img = r.forward(gs, mo, 1, cam, saved)
    other = gc.MotionFrame.from_motion(motion, 1)
    with pytest.raises(gc.GCError, match="residual"):
        r.backward(saved, gs, other, torch.zeros_like(img))
