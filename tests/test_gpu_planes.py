"""The paper's decoded attribute format on the GPU (Sec. 3.4): per-layer uint16 / uint32
position planes and uint8 planes for every other channel, dequantised by the per-layer,
per-channel min / max affine map inside the preprocess and the chain rule.  The oracle
dequantises the same planes (``oracle.dequantize_planes``); bars: the GPU render of the
planes equals the GPU render of the oracle-dequantised FP32 scene bit for bit (images, tile
lists, gradients), and matches the FP64 oracle on it (non-ambiguous pixels within 1e-4); the
multi-level and batched forms equal the single-level render."""
import numpy as np
import pytest
import torch

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(53)
    scene = scenes.make_hier_scene(rng, 7000, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 3)
    return scene, motion


def _run(gc, gs, mo, cam, mask, tile=(16, 16), up=None):
    r = gc.Renderer(0, tile=tile, bg=(0.05, 0.1, 0.2))
    saved = gc.Saved(r)
    img = r.forward(gs, mo, mask, cam, saved)
    ranges, ids = r.tile_lists(saved)
    out = {"image": img.clone(), "ids": ids.clone(), "ranges": ranges.clone()}
    if up is not None:
        out["grads"] = {k: v.clone() for k, v in r.backward(saved, gs, mo, up).items()}
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("pos_bits,width,tile", [(16, 96, (16, 16)), (32, 61, (8, 32))])
def test_planes_forward_backward(gc, case, pos_bits, width, tile):
    scene, motion = case
    planes = scenes.quantize_planes(scene, plane_width=width, pos_bits=pos_bits)
    deq = oracle.dequantize_planes(planes, scene)
    cam = scenes.orbit_camera(1.2, 4.0, 176, 120)
    mask = scenes.level_mask(6)
    mo = gc.MotionFrame.from_motion(motion, 2)
    up = torch.randn((3, cam.height, cam.width), generator=torch.Generator().manual_seed(3)).cuda()
    got = _run(gc, gc.GaussianSet.from_planes(planes, scene), mo, cam, mask, tile, up)
    want = _run(gc, gc.GaussianSet.from_scene(deq), mo, cam, mask, tile, up)
    assert torch.equal(got["image"], want["image"])
    assert torch.equal(got["ids"], want["ids"]) and torch.equal(got["ranges"], want["ranges"])
    for k in want["grads"]:
        assert torch.equal(got["grads"][k], want["grads"][k]), k
    # and the dequantised scene against the FP64 oracle
    opts = oracle.default_options(tile=tile, bg=(0.05, 0.1, 0.2))
    ref = oracle.render(deq, motion, 2, cam, opts, mask)
    ok = ~ref["ambiguous"]
    err = np.abs(got["image"].cpu().numpy().astype(np.float64) - ref["image"]).max(axis=0)
    assert ok.mean() > 0.95 and err[ok].max() <= 1e-4
    tiles = oracle.tile_lists(ref["bins"], cam, tile)
    assert np.array_equal(got["ids"].cpu().numpy(), tiles["gauss_of_entry"])


def test_planes_levels_and_batch(gc, case):
    scene, motion = case
    planes = scenes.quantize_planes(scene, plane_width=128)
    gs = gc.GaussianSet.from_planes(planes, scene)
    cam = scenes.orbit_camera(2.2, 4.0, 160, 96)
    r = gc.Renderer(0, tile=(8, 32))
    frames = [gc.MotionFrame.from_motion(motion, f) for f in range(3)]
    singles = {(f, l): r.forward(gs, frames[f], scenes.level_mask(l), cam).clone() for f in range(3) for l in (2, 6)}
    imgs = r.levels_forward(gs, frames[1], 6, cam)
    torch.cuda.synchronize()
    assert torch.equal(imgs[1], singles[(1, 2)]) and torch.equal(imgs[5], singles[(1, 6)])
    reqs = [(cam, f, scenes.level_mask(l)) for f in range(3) for l in (2, 6)]
    outs = r.batch_forward(gs, frames, reqs)
    torch.cuda.synchronize()
    for (c, f, m), o in zip(reqs, outs):
        assert torch.equal(o, singles[(f, 2 if m == scenes.level_mask(2) else 6)]), (f, m)


def test_planes_argument_errors(gc, case):
    scene, _ = case
    planes = scenes.quantize_planes(scene, plane_width=64)
    cam = scenes.orbit_camera(0.0, 4.0, 64, 48)
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_planes(planes, scene)
    gs.struct.pos_bits = 8
    with pytest.raises(gc.GCError, match="pos_bits"):
        r.forward(gs, None, 1, cam)
    gs.struct.pos_bits = 16
    gs.struct.plane_pitch = 10
    with pytest.raises(gc.GCError, match="pitch"):
        r.forward(gs, None, 1, cam)
