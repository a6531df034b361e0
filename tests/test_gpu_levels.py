"""Single-pass multi-level render (levels 1..L of one view from one list, Eq. 4 nested
layers): every level image equals the single-level render of its layer mask bit for
bit; the one-pass backward equals the sum of the single-level backwards up to float
summation order, and the FP64 oracle's gradients summed over the levels."""
import numpy as np
import pytest
import torch

import oracle
from synth import scenes

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh", "group_q", "group_t")


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(101)
    scene = scenes.make_hier_scene(rng, 8000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 3)
    return scene, motion


@pytest.mark.parametrize("tile,L", [((16, 16), 6), ((8, 32), 6), ((32, 8), 4), ((16, 16), 1)])
def test_levels_equal_single_level_renders(gc, small, tile, L):
    scene, motion = small
    cam = scenes.orbit_camera(1.3, 4.0, 230, 170)
    r = gc.Renderer(0, tile=tile, bg=(0.2, 0.1, 0.05))
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, 2)
    imgs = r.levels_forward(gs, mo, L, cam)
    for l in range(1, L + 1):
        one = r.forward(gs, mo, scenes.level_mask(l), cam)
        torch.cuda.synchronize()
        assert torch.equal(imgs[l - 1], one), (tile, l)


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_levels_backward_matches_single_sum_and_oracle(gc, small, tile):
    scene, motion = small
    cam = scenes.orbit_camera(0.4, 4.0, 128, 96)
    L = 6
    opts = oracle.default_options(tile=tile)
    refs = [oracle.render(scene, motion, 1, cam, opts, scenes.level_mask(l)) for l in range(1, L + 1)]
    rng = np.random.default_rng(3)
    ups = [(rng.normal(0, 1, (3, 96, 128)) * (~ref["ambiguous"])[None]).astype(np.float32) for ref in refs]
    r = gc.Renderer(0, tile=tile)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, 1)
    saved = gc.Saved(r)
    r.levels_forward(gs, mo, L, cam, saved)
    dls = [torch.from_numpy(u).cuda() for u in ups]
    got = r.levels_backward(saved, gs, mo, dls)
    torch.cuda.synchronize()
    got = {k: v.clone() for k, v in got.items()}
    # against the in-order sum of single-level GPU backwards
    acc = {k: torch.zeros_like(v) for k, v in got.items()}
    for l in range(1, L + 1):
        s1 = gc.Saved(r)
        r.forward(gs, mo, scenes.level_mask(l), cam, s1)
        g1 = r.backward(s1, gs, mo, dls[l - 1])
        for k in acc:
            acc[k] += g1[k]
    torch.cuda.synchronize()
    for k in acc:
        a, b = got[k], acc[k]
        assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max()) + 1e-7, k
    # against the FP64 oracle, summed over the levels
    want = None
    for l in range(1, L + 1):
        og = oracle.grad(scene, motion, 1, cam, opts, ups[l - 1].astype(np.float64), scenes.level_mask(l),
                         bins=refs[l - 1]["bins"])
        want = {k: og[k] for k in NAMES} if want is None else {k: want[k] + og[k] for k in NAMES}
    for k in NAMES:
        a = got[k].cpu().numpy().astype(np.float64)
        b = np.asarray(want[k]).reshape(a.shape)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-4, k
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-6, k


@pytest.mark.parametrize("L", [7, 8])
def test_seven_and_eight_levels(gc, L):
    """The largest level counts (the reverse pass's shared memory passes 48 KB at eight): the
    level images equal the single renders bit for bit, and the one-pass backward equals the
    in-order sum of the single-level backwards."""
    rng = np.random.default_rng(211)
    scene = scenes.make_hier_scene(rng, 6000, 8, 1, 4)
    cam = scenes.orbit_camera(0.9, 4.0, 160, 120)
    r = gc.Renderer(0, tile=(8, 32))
    gs = gc.GaussianSet.from_scene(scene)
    saved = gc.Saved(r)
    imgs = [x.clone() for x in r.levels_forward(gs, None, L, cam, saved)]
    g = torch.Generator(device="cuda").manual_seed(5)
    dls = [torch.randn(imgs[0].shape, generator=g, device="cuda") for _ in range(L)]
    got = {k: v.clone() for k, v in r.levels_backward(saved, gs, None, dls).items()}
    acc = None
    for l in range(1, L + 1):
        s1 = gc.Saved(r)
        one = r.forward(gs, None, scenes.level_mask(l), cam, s1)
        torch.cuda.synchronize()
        assert torch.equal(imgs[l - 1], one), l
        g1 = r.backward(s1, gs, None, dls[l - 1])
        acc = {k: v.clone() for k, v in g1.items()} if acc is None else {k: acc[k] + g1[k] for k in acc}
    torch.cuda.synchronize()
    # FP32 summation order only (per entry over the levels here, per level over the entries
    # there), on unmasked N(0, 1) upstream gradients for every level; the rotation's chain
    # rule cancels large terms, so the bound is on the relative L2 norm and a few units of
    # 1e-5 of the largest element.  A level missing or blended twice is off by O(1).
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a, b = got[k].double(), acc[k].double()
        assert float((a - b).norm()) <= 3e-5 * float(b.norm()), k
        assert float((a - b).abs().max()) <= 5e-5 * float(b.abs().max()) + 1e-6, k


def test_levels_argument_errors(gc, small):
    scene, motion = small
    cam = scenes.orbit_camera(0.4, 4.0, 64, 48)
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    with pytest.raises(gc.GCError):
        r.levels_forward(gs, None, 7, cam)  # the set has 6 layers
    saved = gc.Saved(r)
    imgs = r.levels_forward(gs, None, 3, cam, saved)
    with pytest.raises(gc.GCError, match="multi-level"):
        r.backward(saved, gs, None, torch.zeros_like(imgs[0]))


def test_levels_at_1080p(gc):
    """hier1080 frame 7: the six level images of one pass equal the six single renders."""
    w = scenes.hier1080(n_frames=8)
    cam = w.cameras[7]
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(w.scene)
    mo = gc.MotionFrame.from_motion(w.motion, 7)
    imgs = r.levels_forward(gs, mo, 6, cam)
    for l in range(1, 7):
        one = r.forward(gs, mo, scenes.level_mask(l), cam)
        torch.cuda.synchronize()
        assert torch.equal(imgs[l - 1], one), l


def test_levels_at_4k_with_a_wider_tile_grid(gc, small):
    """3840x2160 (32,400 16x16 tiles, 15-bit tile keys): the six level images of one pass
    equal the single renders, and the lists of the top level equal its single render's."""
    scene, motion = small
    cam = scenes.orbit_camera(2.9, 3.2, 3840, 2160)
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    mo = gc.MotionFrame.from_motion(motion, 1)
    saved = gc.Saved(r)
    imgs = r.levels_forward(gs, mo, 6, cam, saved)
    for l in (1, 4, 6):
        one = r.forward(gs, mo, scenes.level_mask(l), cam)
        torch.cuda.synchronize()
        assert torch.equal(imgs[l - 1], one), l


HEADLINE_TILE = (8, 32)  # the tile shape the throughput benchmark renders the multi-level step with


def test_levels_backward_at_1080p_headline(gc):
    """The timed forward + backward at the size and tile shape it is timed at: hier1080
    (300k Gaussians, SH 3, 64 groups) frame 7, levels L1..L6 of 1920x1080 in one pass,
    8x32 tiles.  (1) With a dense dL/dimage per level, the one-pass backward equals the
    in-order sum of the six single-level backwards up to float summation order: the one pass
    sums each pixel's levels before the pixels, the single renders the pixels of each level,
    and both recover each pixel's transmittance in reverse by dividing by (1 - alpha) per
    blended entry (the one pass multiplies by one reciprocal per entry, the single render takes
    a fast divide), so an entry m blended entries deep carries a relative error of up to about
    2 m ulp in T that differs between the two; pixels here blend up to a few hundred entries
    (m x 2 ulp ~ 4e-5).  Bars: relative L2 <= 5e-5 per tensor, every element within 1e-4 of the
    tensor's largest.  (2) With
    dL/dimage nonzero on 4,096 seeded non-ambiguous pixels per level, it matches the FP64
    oracle's gradient summed over the levels (rel L2 <= 1e-4, elementwise <= 1e-3 max + 1e-6)."""
    w = scenes.hier1080(n_frames=8)
    f, L, (W, H) = 7, 6, (1920, 1080)
    cam = w.cameras[f]
    r = gc.Renderer(0, tile=HEADLINE_TILE)
    gs = gc.GaussianSet.from_scene(w.scene)
    mo = gc.MotionFrame.from_motion(w.motion, f)
    gen = torch.Generator(device="cuda").manual_seed(5)
    dense = [torch.randn((3, H, W), generator=gen, device="cuda") for _ in range(L)]
    saved = gc.Saved(r)
    r.levels_forward(gs, mo, L, cam, saved)
    got = {k: v.clone() for k, v in r.levels_backward(saved, gs, mo, dense).items()}
    acc = None
    for l in range(1, L + 1):
        s1 = gc.Saved(r)
        r.forward(gs, mo, scenes.level_mask(l), cam, s1)
        g1 = r.backward(s1, gs, mo, dense[l - 1])
        acc = {k: v.clone() for k, v in g1.items()} if acc is None else {k: acc[k] + g1[k] for k in acc}
    torch.cuda.synchronize()
    for k in NAMES:
        a, b = got[k].double(), acc[k].double()
        bmax = float(b.abs().max())
        assert bmax > 0, k
        rel = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
        emax = float((a - b).abs().max())
        assert rel <= 5e-5 and emax <= 1e-4 * bmax, (k, rel, emax / bmax)
    del dense, acc

    opts = oracle.default_options(tile=HEADLINE_TILE)
    rng = np.random.default_rng(77)
    ups, want = [], None
    for l in range(1, L + 1):
        mask = scenes.level_mask(l)
        bins = oracle.bin_f32(w.scene, w.motion, f, cam, opts, mask)
        pix = scenes.sample_pixels(700 + l, W, H, 4096)
        ref = oracle.render(w.scene, w.motion, f, cam, opts, mask, pixels=pix, bins=bins)
        up = np.zeros((3, H, W))
        vals = rng.normal(0, 1, (len(pix), 3)) * (~ref["ambiguous"])[:, None]
        up[:, pix[:, 1], pix[:, 0]] = vals.T
        up = up.astype(np.float32).astype(np.float64)
        ups.append(up)
        og = oracle.grad(w.scene, w.motion, f, cam, opts, up, mask, bins=bins)
        want = {k: np.asarray(og[k]) for k in NAMES} if want is None else \
            {k: want[k] + np.asarray(og[k]) for k in NAMES}
    r.levels_forward(gs, mo, L, cam, saved)
    got = r.levels_backward(saved, gs, mo, [torch.from_numpy(u.astype(np.float32)).cuda() for u in ups])
    torch.cuda.synchronize()
    for k in NAMES:
        a = got[k].cpu().numpy().astype(np.float64)
        b = want[k].reshape(a.shape)
        assert np.linalg.norm(b) > 0, k
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 1e-4, (k, rel)
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-6, (k, np.abs(a - b).max())
