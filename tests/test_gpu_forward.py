"""GPU forward parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: tile lists bit-exact against the oracle's FP32 binning mirror; per-pixel
count of blended Gaussians identical and max |pixel| <= 1e-4 on pixels where
no per-pixel decision is within its FP32 margin (the oracle's ambiguity flag).
"""
import numpy as np
import pytest
import torch

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-4


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


def _render_gpu(gc, scene, motion, frame, cam, mask, tile=(16, 16), bg=(0, 0, 0), membership=0,
                key_capacity=0):
    r = gc.Renderer(0, tile=tile, bg=bg, membership=membership, key_capacity=key_capacity)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, frame) if motion is not None else None
    saved = gc.Saved(r)
    img = r.forward(gs, mo, mask, cam, saved)
    torch.cuda.synchronize()
    ranges, ids = r.tile_lists(saved)
    T, nb = r.pixel_state(saved)
    st = r.stats(saved)
    return {"image": img.cpu().numpy().astype(np.float64), "ranges": ranges.cpu().numpy(),
            "ids": ids.cpu().numpy(), "T": T.cpu().numpy(), "nb": nb.cpu().numpy(), "stats": st}


def _compare(gpu, ref, tiles, what=""):
    # tile lists: bit-exact
    assert np.array_equal(gpu["ids"], tiles["gauss_of_entry"]), what
    assert np.array_equal(gpu["ranges"][:, 0][gpu["ranges"][:, 1] > gpu["ranges"][:, 0]],
                          tiles["ranges"][:, 0][tiles["ranges"][:, 1] > tiles["ranges"][:, 0]]), what
    assert np.array_equal(gpu["ranges"][:, 1] - gpu["ranges"][:, 0],
                          tiles["ranges"][:, 1] - tiles["ranges"][:, 0]), what
    ok = ~ref["ambiguous"]
    err = np.abs(gpu["image"] - ref["image"]).max(axis=0)
    assert ok.mean() > 0.95, what
    assert err[ok].max() <= PIX_TOL, (what, float(err[ok].max()))
    assert np.array_equal(gpu["nb"][ok], ref["n_blended"][ok]), what
    assert np.abs(gpu["T"][ok] - ref["T"][ok]).max() <= 1e-4, what


def _oracle(scene, motion, frame, cam, mask, tile=(16, 16), bg=(0, 0, 0), membership=0):
    opts = oracle.default_options(tile=tile, bg=bg, membership=membership)
    ref = oracle.render(scene, motion, frame, cam, opts, mask)
    tiles = oracle.tile_lists(ref["bins"], cam, tile)
    return ref, tiles


def test_tiny_full_frame(gc):
    w = scenes.tiny()
    cam = w.cameras[0]
    gpu = _render_gpu(gc, w.scene, None, 0, cam, 1)
    ref, tiles = _oracle(w.scene, None, 0, cam, 1)
    _compare(gpu, ref, tiles, "tiny")
    assert gpu["stats"]["n_keys"] == len(tiles["gauss_of_entry"])
    assert gpu["stats"]["n_visible"] == int(ref["bins"]["visible"].sum())


@pytest.fixture(scope="module")
def hier_small():
    rng = np.random.default_rng(31)
    scene = scenes.make_hier_scene(rng, 6000, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 4)
    return scene, motion


@pytest.mark.parametrize("mask", [1, 0b111, 0b111111, 0b101010])
def test_ragged_layers_motion_sh3(gc, hier_small, mask):
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.6, 4.0, 200, 136)   # 12.5 x 8.5 tiles: ragged edges
    bg = (0.2, 0.1, 0.05)
    gpu = _render_gpu(gc, scene, motion, 2, cam, mask, bg=bg)
    ref, tiles = _oracle(scene, motion, 2, cam, mask, bg=bg)
    _compare(gpu, ref, tiles, f"mask {mask}")


@pytest.mark.parametrize("tile", [(8, 32), (32, 8)])
def test_tile_shapes(gc, hier_small, tile):
    scene, motion = hier_small
    cam = scenes.orbit_camera(1.1, 4.0, 176, 120)
    gpu = _render_gpu(gc, scene, motion, 3, cam, 63, tile=tile)
    ref, tiles = _oracle(scene, motion, 3, cam, 63, tile=tile)
    _compare(gpu, ref, tiles, f"tile {tile}")
    base = _render_gpu(gc, scene, motion, 3, cam, 63)
    assert np.array_equal(base["image"], gpu["image"])  # pixel-square rule: tile-shape invariant


def test_whole_tile_membership(gc, hier_small):
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.3, 4.0, 160, 96)
    gpu = _render_gpu(gc, scene, motion, 1, cam, 63, membership=1)
    ref, tiles = _oracle(scene, motion, 1, cam, 63, membership=1)
    _compare(gpu, ref, tiles, "tile membership")


def test_empty_and_culled(gc, hier_small):
    scene, motion = hier_small
    bg = (0.3, 0.6, 0.9)
    cam = scenes.orbit_camera(0.0, 4.0, 40, 24)
    bgimg = np.broadcast_to(np.array(bg, np.float32).astype(np.float64)[:, None, None], (3, 24, 40))
    # no layer selected
    g = _render_gpu(gc, scene, motion, 0, cam, 0, bg=bg)
    assert np.array_equal(g["image"], bgimg) and g["stats"]["n_keys"] == 0
    # camera looking away from every Gaussian
    away = scenes.look_at_camera((0, 0, -4), (0, 0, -8), 40, 24)
    g = _render_gpu(gc, scene, motion, 0, away, 63, bg=bg)
    assert np.array_equal(g["image"], bgimg) and g["stats"]["n_visible"] == 0
    # an empty scene
    empty = scene.subset(np.arange(0))
    g = _render_gpu(gc, empty, None, 0, cam, 1, bg=bg)
    assert np.array_equal(g["image"], bgimg)


def test_degenerate_quaternion_and_behind_camera(gc):
    w = scenes.tiny(n=64, size=48)
    sc = w.scene
    sc.quats[3] = 0.0                      # zero quaternion: culled
    sc.means[5] = np.array([0, 0, -3.1])   # behind the camera
    sc.means[6] = np.array([0, 0, -2.85])  # in front of the camera but inside the near plane
    cam = w.cameras[0]
    gpu = _render_gpu(gc, sc, None, 0, cam, 1)
    ref, tiles = _oracle(sc, None, 0, cam, 1)
    assert not ref["bins"]["visible"][3] and not ref["bins"]["visible"][5] and not ref["bins"]["visible"][6]
    _compare(gpu, ref, tiles, "degenerate")


def test_deterministic(gc, hier_small):
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.9, 4.0, 128, 128)
    a = _render_gpu(gc, scene, motion, 1, cam, 63)
    b = _render_gpu(gc, scene, motion, 1, cam, 63)
    assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["ids"], b["ids"])


def test_fixed_capacity(gc, hier_small):
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.9, 4.0, 128, 128)
    a = _render_gpu(gc, scene, motion, 1, cam, 63)
    k = a["stats"]["n_keys"]
    b = _render_gpu(gc, scene, motion, 1, cam, 63, key_capacity=k + 100)
    assert np.array_equal(a["image"], b["image"])
    r = gc.Renderer(0, key_capacity=k // 2)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, 1)
    saved = gc.Saved(r)
    img = r.forward(gs, mo, 63, cam, saved)
    # over its capacity a frame places no entry (8 tile columns: binning by tile row), so the
    # image is the background and the backward, whose partials buffer the capacity sizes,
    # writes no partial
    g = r.backward(saved, gs, mo, torch.ones_like(img))
    torch.cuda.synchronize()
    assert not img.any()
    for name, v in g.items():
        assert not v.any(), name
    with pytest.raises(gc.GCError) as e:
        r.check()
    assert "GC_ERR_CAPACITY" in str(e.value)


@pytest.fixture(scope="module")
def hier1080():
    return scenes.hier1080()


@pytest.mark.parametrize("frame,level", [(0, 6), (17, 1), (29, 4)])
def test_hier1080_at_scale(gc, hier1080, frame, level):
    """Full 1920x1080 render of the 300k-Gaussian scene: tile lists bit-exact over
    every tile; pixels compared on 4,096 seeded samples (the oracle computes them
    one by one)."""
    w = hier1080
    cam = w.cameras[frame]
    mask = scenes.level_mask(level)
    gpu = _render_gpu(gc, w.scene, w.motion, frame, cam, mask)
    opts = oracle.default_options()
    bins = oracle.bin_f32(w.scene, w.motion, frame, cam, opts, mask)
    tiles = oracle.tile_lists(bins, cam)
    assert np.array_equal(gpu["ids"], tiles["gauss_of_entry"])
    assert np.array_equal(gpu["ranges"][:, 1] - gpu["ranges"][:, 0], tiles["ranges"][:, 1] - tiles["ranges"][:, 0])
    pix = scenes.sample_pixels(100 + frame, cam.width, cam.height, 4096)
    ref = oracle.render(w.scene, w.motion, frame, cam, opts, mask, pixels=pix, bins=bins)
    ok = ~ref["ambiguous"]
    g = gpu["image"][:, pix[:, 1], pix[:, 0]].T
    err = np.abs(g - ref["image"]).max(axis=1)
    assert ok.mean() > 0.95
    assert err[ok].max() <= PIX_TOL, float(err[ok].max())
    assert np.array_equal(gpu["nb"][pix[:, 1], pix[:, 0]][ok], ref["n_blended"][ok])


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_alpha_cull_changes_lists_not_results(gc, tile):
    """The alpha footprint shortens the tile lists; images and per-pixel state are
    bit-identical to the 3-sigma-only lists (the removed pairs were skipped by the
    compositing rule anyway) and the gradients agree up to the order of the per-Gaussian
    sum over tiles (the removed tiles held exact zeros)."""
    rng = np.random.default_rng(91)
    scene = scenes.make_hier_scene(rng, 20000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 2)
    cam = scenes.orbit_camera(0.9, 4.0, 400, 300)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, 1)
    up = torch.randn((3, 300, 400), generator=torch.Generator().manual_seed(2)).cuda()
    out = {}
    for cull in (False, True):
        r = gc.Renderer(0, tile=tile, alpha_cull=cull)
        saved = gc.Saved(r)
        img = r.forward(gs, mo, 63, cam, saved)
        T, nb = r.pixel_state(saved)
        g = r.backward(saved, gs, mo, up)
        torch.cuda.synchronize()
        out[cull] = (img, T, nb, {k: v.clone() for k, v in g.items()}, r.stats(saved)["n_keys"])
    assert torch.equal(out[False][0], out[True][0])
    assert torch.equal(out[False][1], out[True][1])
    assert torch.equal(out[False][2], out[True][2])
    for k in out[False][3]:
        a, b = out[True][3][k], out[False][3][k]
        assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max()), k
    assert out[True][4] < 0.85 * out[False][4]


def test_frame_over_255_tile_columns(gc, hier_small):
    """4,160 x 1,040 px (260 columns of 16 px tiles): past binning by tile row, the frame takes the
    full-key tile sort; its lists are bit-exact against the oracle's FP32 binning mirror and
    its pixels within the bar on 4,096 seeded samples."""
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.9, 4.0, 4160, 1040)
    gpu = _render_gpu(gc, scene, motion, 1, cam, 63)
    opts = oracle.default_options()
    bins = oracle.bin_f32(scene, motion, 1, cam, opts, 63)
    tiles = oracle.tile_lists(bins, cam)
    assert len(tiles["gauss_of_entry"]) > 0
    assert np.array_equal(gpu["ids"], tiles["gauss_of_entry"])
    assert np.array_equal(gpu["ranges"][:, 1] - gpu["ranges"][:, 0], tiles["ranges"][:, 1] - tiles["ranges"][:, 0])
    pix = scenes.sample_pixels(41, cam.width, cam.height, 4096)
    ref = oracle.render(scene, motion, 1, cam, opts, 63, pixels=pix, bins=bins)
    ok = ~ref["ambiguous"]
    g = gpu["image"][:, pix[:, 1], pix[:, 0]].T
    assert ok.mean() > 0.95
    assert np.abs(g - ref["image"]).max(axis=1)[ok].max() <= PIX_TOL
