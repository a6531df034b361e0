"""The per-Gaussian motion source on the GPU (Sec. 3.2, rigid transformation): hash-grid
encoding of the frame t-1 positions and the translation / rotation MLPs, forward and backward,
against the FP64 oracle (``oracle.motion_net``); then fed to the renderer as one rigid motion
per Gaussian (gc_motion.per_gaussian), whose images, lists and motion gradients are checked
against the oracle with group = Gaussian and against the GPU's group-motion path."""
import numpy as np
import pytest
import torch

import oracle
from oracle import motion_net as mn
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("levels,log2_T,n", [(16, 15, 20_077), (5, 12, 20_077), (1, 4, 20_077),
                                             (16, 19, 296 * 128 * 2 + 77)])
def test_field_forward_backward_matches_oracle(gc, levels, log2_T, n):
    """n = 20,077: one chunk of 128 Gaussians per block, ragged last chunk; the last case gives
    every block of the persistent backward two or three chunks."""
    rng = np.random.default_rng(7 + levels)
    p = scenes.motion_field_params(rng, n_levels=levels, log2_T=log2_T, n_min=4 if levels == 1 else 16)
    mu = rng.uniform(-1.6, 1.6, (n, 3)).astype(np.float32)    # some outside the box: clamped
    t_ref, q_ref = mn.forward(mu, p)
    r = gc.Renderer(0)
    field = gc.MotionField(p)
    mu_d = torch.from_numpy(mu).cuda()
    q, t = r.motion_field_forward(field, mu_d)
    # the training form keeps the encodings: same q and t bit for bit
    enc = torch.full((n, 32), float("nan"), device="cuda")
    q_s, t_s = r.motion_field_forward(field, mu_d, encodings=enc)
    torch.cuda.synchronize()
    assert torch.equal(q_s, q) and torch.equal(t_s, t)
    assert bool(torch.isfinite(enc).all()) and not enc[:, 2 * levels:].any()
    q, t = q.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    assert np.abs(t - t_ref).max() <= 1e-5 * np.abs(t_ref).max() + 1e-7
    assert np.abs(q - q_ref).max() <= 1e-5 * np.abs(q_ref).max() + 1e-7
    d_t = rng.normal(0, 1, (n, 3)).astype(np.float32)
    d_q = rng.normal(0, 1, (n, 4)).astype(np.float32)
    want = mn.backward(mu, p, d_t.astype(np.float64), d_q.astype(np.float64))
    got = r.motion_field_backward(field, mu_d, torch.from_numpy(d_q).cuda(), torch.from_numpy(d_t).cuda())
    torch.cuda.synchronize()
    for k in gc.MotionField.NAMES:
        a = got[k].cpu().numpy().astype(np.float64)
        assert _rel(a, want[k]) <= 1e-4, (k, _rel(a, want[k]))
    # the weight gradients are summed in a fixed order: bit-reproducible
    again = r.motion_field_backward(field, mu_d, torch.from_numpy(d_q).cuda(), torch.from_numpy(d_t).cuda())
    # with the forward's encodings: the same weight gradients bit for bit, the table gradient
    # (vector atomics, order not fixed) within float summation order
    saved = r.motion_field_backward(field, mu_d, torch.from_numpy(d_q).cuda(), torch.from_numpy(d_t).cuda(),
                                    encodings=enc)
    torch.cuda.synchronize()
    for k in ("w1t", "b1t", "w2t", "b2t", "w1r", "b1r", "w2r", "b2r"):
        assert torch.equal(got[k], again[k]), k
        assert torch.equal(got[k], saved[k]), k
    # (each table entry sums up to hundreds of Gaussians' corner terms with float atomics in
    # no fixed order: a few 1e-6 relative between two runs)
    a, b = saved["table"].double(), got["table"].double()
    assert float((a - b).norm() / b.norm()) <= 1e-5
    sv_t = saved["table"].cpu().numpy().astype(np.float64)
    assert _rel(sv_t, want["table"]) <= 1e-4


def test_field_drives_the_renderer(gc):
    rng = np.random.default_rng(61)
    scene = scenes.make_hier_scene(rng, 5000, 4, 3, 8)
    p = scenes.motion_field_params(rng, n_levels=8, log2_T=14)
    r = gc.Renderer(0, tile=(8, 32), bg=(0.1, 0.1, 0.1))
    field = gc.MotionField(p)
    gs = gc.GaussianSet.from_scene(scene)
    q, t = r.motion_field_forward(field, gs.tensors["means"])
    mo = gc.MotionFrame(q, t, per_gaussian=True)
    cam = scenes.orbit_camera(0.5, 4.0, 160, 112)
    mask = scenes.level_mask(4)
    saved = gc.Saved(r)
    img = r.forward(gs, mo, mask, cam, saved)
    ranges, ids = r.tile_lists(saved)
    # the oracle with one group per Gaussian and the GPU's motion as the group table
    per = scenes.Scene(scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh,
                       np.arange(scene.n, dtype=np.int32), scene.layer_offsets, scene.sh_degree, scene.n)
    motion = scenes.Motion(q.cpu().numpy()[None].astype(np.float32), t.cpu().numpy()[None].astype(np.float32))
    opts = oracle.default_options(tile=(8, 32), bg=(0.1, 0.1, 0.1))
    ref = oracle.render(per, motion, 0, cam, opts, mask)
    tiles = oracle.tile_lists(ref["bins"], cam, (8, 32))
    assert np.array_equal(ids.cpu().numpy(), tiles["gauss_of_entry"])
    ok = ~ref["ambiguous"]
    assert ok.mean() > 0.95
    assert np.abs(img.cpu().numpy().astype(np.float64) - ref["image"]).max(axis=0)[ok].max() <= 1e-4
    # the same as group motion with group id = Gaussian index
    gs_g = gc.GaussianSet.from_scene(per)
    img_g = r.forward(gs_g, gc.MotionFrame(q, t), mask, cam)
    torch.cuda.synchronize()
    assert torch.equal(img, img_g)
    # motion gradients per Gaussian, then through the motion source
    up = (np.random.default_rng(5).normal(0, 1, (3, cam.height, cam.width)) * (~ref["ambiguous"])[None])
    up = up.astype(np.float32)
    g = r.backward(saved, gs, mo, torch.from_numpy(up).cuda())
    want = oracle.grad(per, motion, 0, cam, opts, up.astype(np.float64), mask, bins=ref["bins"])
    for k in ("group_q", "group_t"):
        a = g[k].cpu().numpy().astype(np.float64)
        assert a.shape == want[k].shape
        assert _rel(a, want[k]) <= 1e-4, k
    fg = r.motion_field_backward(field, gs.tensors["means"], g["group_q"], g["group_t"])
    fw = mn.backward(scene.means, p, want["group_t"], want["group_q"])
    for k in gc.MotionField.NAMES:
        assert _rel(fg[k].cpu().numpy().astype(np.float64), fw[k]) <= 1e-3, k


def test_field_argument_errors(gc):
    rng = np.random.default_rng(1)
    p = scenes.motion_field_params(rng, n_levels=4, log2_T=10)
    r = gc.Renderer(0)
    field = gc.MotionField(p)
    # saved encodings must be 16-byte aligned rows
    buf = torch.zeros(4 * 32 + 1, device="cuda")
    with pytest.raises(gc.GCError, match="aligned"):
        r.motion_field_forward(field, torch.zeros((4, 3), device="cuda"), encodings=buf[1:].view(4, 32))
    with pytest.raises(gc.GCError, match="aligned"):
        r.motion_field_backward(field, torch.zeros((4, 3), device="cuda"), torch.zeros((4, 4), device="cuda"),
                                torch.zeros((4, 3), device="cuda"), encodings=buf[1:].view(4, 32))
    field.struct.n_levels = 17
    with pytest.raises(gc.GCError, match="n_levels"):
        r.motion_field_forward(field, torch.zeros((4, 3), device="cuda"))
    field.struct.n_levels = 4
    field.struct.hi[1] = field.struct.lo[1]
    with pytest.raises(gc.GCError, match="hi"):
        r.motion_field_forward(field, torch.zeros((4, 3), device="cuda"))
