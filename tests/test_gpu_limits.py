"""The limit of binning by tile row on the selection size.

Row-binned list words hold the column and the rank in 24 bits, so an image with more than
2^24 selected Gaussians takes the full-key tile sort.  The test uses 2^24 + 2,000 Gaussians
placed behind the camera, which the near plane culls, plus 3,000 visible ones at the end of
the index range.  That image must equal, bit for bit, the visible Gaussians rendered alone:
- image, tile lists and gradients in one view;
- images in a batch.

The visible ones alone go through row binning, and the depth order of the visible Gaussians
is the same in both, so the lists and every blend match."""
import numpy as np
import pytest
import torch

from synth import scenes

pytestmark = pytest.mark.gpu

N_HIDDEN = (1 << 24) + 2000
NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


@pytest.fixture(scope="module")
def scenes_pair():
    rng = np.random.default_rng(97)
    vis = scenes.make_hier_scene(rng, 3000, 1, 0, 1)
    n = N_HIDDEN + vis.n
    means = np.empty((n, 3), np.float32)
    means[:N_HIDDEN] = (0.0, 0.0, -10.0)            # behind the eye at z = -4
    means[:N_HIDDEN, 0] = rng.uniform(-1, 1, N_HIDDEN).astype(np.float32)
    means[N_HIDDEN:] = vis.means

    def cat(hidden_row, arr):
        out = np.empty((n,) + arr.shape[1:], arr.dtype)
        out[:N_HIDDEN] = hidden_row
        out[N_HIDDEN:] = arr
        return out

    big = scenes.Scene(means, cat(-3.0, vis.log_scales), cat((1.0, 0.0, 0.0, 0.0), vis.quats),
                       cat(0.0, vis.opacity_logits), cat(0.5, vis.sh), cat(0, vis.group_id),
                       np.array([0, n], np.int64), 0, 1)
    return big, vis


def test_selection_past_2_24_takes_the_key_sort(gc, scenes_pair):
    big, vis = scenes_pair
    cam = scenes.orbit_camera(0.0, 4.0, 160, 120)
    r = gc.Renderer(0, tile=(16, 16))
    out = {}
    for name, sc in (("big", big), ("vis", vis)):
        gs = gc.GaussianSet.from_scene(sc)
        saved = gc.Saved(r)
        img = r.forward(gs, None, 1, cam, saved)
        ranges, ids = r.tile_lists(saved)
        up = torch.randn(img.shape, generator=torch.Generator(device="cuda").manual_seed(3), device="cuda")
        g = r.backward(saved, gs, None, up)
        torch.cuda.synchronize()
        out[name] = (img.clone(), ranges.clone(), ids.clone(), {k: g[k].clone() for k in NAMES}, r.stats(saved))
        del gs, saved, g
        torch.cuda.empty_cache()
    ib, rb, idb, gb, sb = out["big"]
    iv, rv, idv, gv, sv = out["vis"]
    assert sb["n_selected"] == big.n and sv["n_selected"] == vis.n
    assert sv["n_keys"] > 0 and sb["n_keys"] == sv["n_keys"]
    assert torch.equal(ib, iv)
    assert torch.equal(rb, rv)
    assert torch.equal(idb - N_HIDDEN, idv)
    for k in NAMES:
        assert torch.equal(gb[k][N_HIDDEN:], gv[k]), k
        assert not gb[k][:N_HIDDEN].any(), k


def test_batch_with_a_selection_past_2_24(gc, scenes_pair):
    big, vis = scenes_pair
    cams = [scenes.orbit_camera(0.0, 4.0, 160, 120), scenes.orbit_camera(0.4, 4.2, 128, 96)]
    r = gc.Renderer(0, tile=(8, 32))
    gs_big = gc.GaussianSet.from_scene(big)
    imgs = [x.clone() for x in r.batch_forward(gs_big, [], [(c, -1, 1) for c in cams])]
    r.check()
    del gs_big
    torch.cuda.empty_cache()
    gs_vis = gc.GaussianSet.from_scene(vis)
    for c, got in zip(cams, imgs):
        one = r.forward(gs_vis, None, 1, c)
        torch.cuda.synchronize()
        assert torch.equal(got, one)
