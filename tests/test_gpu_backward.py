"""GPU backward parity: gc_render_backward against the oracle's FP64 reverse mode.

The upstream gradient dL/dimage is zero on pixels the oracle flags as
ambiguous (a per-pixel skip/stop decision within its FP32 margin), so both
sides differentiate the same piecewise-smooth function.  Bars (FP32 against
FP64): per-tensor relative L2 error <= 1e-4 and every element within
1e-3 * max|g| + 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu

REL_L2 = 1e-4
ELEM = 1e-3

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


def _run(gc, scene, motion, frame, cam, mask, up, tile=(16, 16), bg=(0, 0, 0)):
    r = gc.Renderer(0, tile=tile, bg=bg)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, frame) if motion is not None else None
    saved = gc.Saved(r)
    img = r.forward(gs, mo, mask, cam, saved)
    g = r.backward(saved, gs, mo, torch.from_numpy(up.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return img.cpu().numpy(), {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def _upstream(ref, cam, seed, sparse_pixels=None):
    rng = np.random.default_rng(seed)
    up = rng.normal(0, 1, (3, cam.height, cam.width))
    if sparse_pixels is not None:
        keep = np.zeros((cam.height, cam.width), bool)
        keep[sparse_pixels[:, 1], sparse_pixels[:, 0]] = True
        up *= keep[None]
    up *= ~ref["ambiguous"][None]
    return up.astype(np.float32).astype(np.float64)


def _compare(got, want, names, what=""):
    for k in names:
        a, b = got[k], want[k]
        nb = np.linalg.norm(b)
        assert nb > 0, (what, k)
        rel = np.linalg.norm(a - b) / nb
        assert rel <= REL_L2, (what, k, rel)
        assert np.abs(a - b).max() <= ELEM * np.abs(b).max() + 1e-6, (what, k, np.abs(a - b).max())


def test_tiny(gc):
    w = scenes.tiny()
    cam = w.cameras[0]
    opts = oracle.default_options()
    ref = oracle.render(w.scene, None, 0, cam, opts, 1)
    up = _upstream(ref, cam, 0)
    _, g = _run(gc, w.scene, None, 0, cam, 1, up)
    og = oracle.grad(w.scene, None, 0, cam, opts, up, 1, bins=ref["bins"])
    _compare(g, og, NAMES, "tiny")


@pytest.fixture(scope="module")
def hier_small():
    rng = np.random.default_rng(51)
    scene = scenes.make_hier_scene(rng, 6000, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 4)
    return scene, motion


@pytest.mark.parametrize("mask,tile", [(0b111111, (16, 16)), (0b000111, (16, 16)),
                                       (0b101010, (8, 32)), (0b011011, (32, 8))])
def test_layers_motion_sh3(gc, hier_small, mask, tile):
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.5, 4.0, 200, 136)
    bg = (0.2, 0.1, 0.05)
    opts = oracle.default_options(tile=tile, bg=bg)
    ref = oracle.render(scene, motion, 2, cam, opts, mask)
    up = _upstream(ref, cam, mask)
    _, g = _run(gc, scene, motion, 2, cam, mask, up, tile=tile, bg=bg)
    og = oracle.grad(scene, motion, 2, cam, opts, up, mask, bins=ref["bins"])
    _compare(g, og, NAMES + ("group_q", "group_t"), f"mask {mask} tile {tile}")
    # unselected layers get exactly zero
    sel = scenes.selected_indices(scene.layer_offsets, mask)
    unsel = np.setdiff1d(np.arange(scene.n), sel)
    for k in NAMES:
        assert not np.any(g[k][unsel])


def test_deterministic(gc, hier_small):
    scene, motion = hier_small
    cam = scenes.orbit_camera(1.2, 4.0, 128, 128)
    up = np.random.default_rng(3).normal(0, 1, (3, 128, 128))
    _, a = _run(gc, scene, motion, 1, cam, 63, up)
    _, b = _run(gc, scene, motion, 1, cam, 63, up)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_autograd_l1_loss(gc, hier_small):
    """torch.autograd through the binding: L1 loss against a target render."""
    scene, motion = hier_small
    cam = scenes.orbit_camera(0.2, 4.0, 160, 120)
    r = gc.Renderer(0)
    dev = "cuda"
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).to(dev).requires_grad_(True)
         for k in NAMES}
    gid = torch.from_numpy(scene.group_id.astype(np.int32)).to(dev)
    gq = torch.from_numpy(motion.q[1]).to(dev).requires_grad_(True)
    gt = torch.from_numpy(motion.t[1]).to(dev).requires_grad_(True)
    target_scene = scene.subset(np.arange(scene.n))
    target_scene.means = (scene.means + np.random.default_rng(5).normal(0, 0.01, scene.means.shape)).astype(np.float32)
    tgs = gc.GaussianSet.from_scene(target_scene)
    target = r.forward(tgs, gc.MotionFrame.from_motion(motion, 1), 63, cam).detach().clone()
    img = gc.render(r, scene.layer_offsets, scene.sh_degree, 63, cam, t["means"], t["log_scales"],
                    t["quats"], t["opacity_logits"], t["sh"], gid, gq, gt)
    loss = (img - target).abs().mean()
    loss.backward()
    up = (torch.sign(img - target) / img.numel()).detach().cpu().numpy().astype(np.float64)
    og = oracle.grad(scene, motion, 1, cam, oracle.default_options(), up, 63)
    got = {k: t[k].grad.cpu().numpy().astype(np.float64) for k in NAMES}
    got["group_q"] = gq.grad.cpu().numpy().astype(np.float64)
    got["group_t"] = gt.grad.cpu().numpy().astype(np.float64)
    for k in got:
        rel = np.linalg.norm(got[k] - og[k]) / np.linalg.norm(og[k])
        assert rel <= 1e-3, (k, rel)   # includes ambiguous pixels, hence the looser bar


def test_diff_workload_at_scale(gc):
    """The differentiation workload (200k Gaussians, 1352x1014, SH 3, 32 groups):
    dL/dimage is nonzero on 4,096 seeded pixels, which the oracle differentiates
    one by one; the GPU runs its full backward."""
    w = scenes.diff()
    cam = w.cameras[0]
    opts = oracle.default_options()
    mask = 63
    bins = oracle.bin_f32(w.scene, w.motion, 1, cam, opts, mask)
    pix = scenes.sample_pixels(7, cam.width, cam.height, 4096)
    ref = oracle.render(w.scene, w.motion, 1, cam, opts, mask, pixels=pix, bins=bins)
    up = np.zeros((3, cam.height, cam.width))
    vals = np.random.default_rng(9).normal(0, 1, (len(pix), 3)) * (~ref["ambiguous"])[:, None]
    up[:, pix[:, 1], pix[:, 0]] = vals.T
    up = up.astype(np.float32).astype(np.float64)
    _, g = _run(gc, w.scene, w.motion, 1, cam, mask, up)
    og = oracle.grad(w.scene, w.motion, 1, cam, opts, up, mask, bins=bins)
    _compare(g, og, NAMES + ("group_q", "group_t"), "diff at scale")


@pytest.mark.parametrize("levels", [0, 6])
def test_second_backward_on_one_state_equals_a_fresh_one(gc, levels):
    """The partials buffer and the per-entry flags must be all zero again after a backward:
    a second backward on the same saved state, with another upstream gradient, gives the
    same bits as that backward on a fresh state (single-level and six-level passes)."""
    rng = np.random.default_rng(71)
    scene = scenes.make_hier_scene(rng, 4000, 6, 2, 4)
    cam = scenes.orbit_camera(0.7, 4.0, 144, 112)
    r = gc.Renderer(0, tile=(8, 32))
    gs = gc.GaussianSet.from_scene(scene)
    gen = torch.Generator(device="cuda").manual_seed(9)
    n_img = levels if levels else 1
    ups = [[torch.randn((3, cam.height, cam.width), generator=gen, device="cuda") for _ in range(n_img)]
           for _ in range(2)]

    def fwd(saved):
        if levels:
            r.levels_forward(gs, None, levels, cam, saved)
        else:
            r.forward(gs, None, scenes.level_mask(6), cam, saved)

    def bwd(saved, up):
        g = r.levels_backward(saved, gs, None, up) if levels else r.backward(saved, gs, None, up[0])
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in g.items()}

    s1 = gc.Saved(r)
    fwd(s1)
    first = bwd(s1, ups[0])
    second = bwd(s1, ups[1])
    s2 = gc.Saved(r)
    fwd(s2)
    fresh = bwd(s2, ups[1])
    for k in NAMES:
        assert torch.equal(second[k], fresh[k]), k
        assert not torch.equal(first[k], second[k]), k
