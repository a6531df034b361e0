"""Batched requests (many cameras, resolutions, motion frames and layer masks of one
Gaussian set in one pass): parity with the single-request path and with the oracle.

* every batched image equals gc_render_forward of that request alone, bit for bit
  (same projection, same stable orders, same per-tile blend);
* one request of the batch against the FP64 oracle directly (max |pixel| <= 1e-4 on
  non-ambiguous pixels);
* batched gradients against the oracle's FP64 gradients summed over the requests
  (relative L2 <= 1e-4, every element within 1e-3 max|g| + 1e-6), motion gradients per
  (frame, group); and against the in-order sum of single-request GPU gradients;
* fixed key capacity: a CUDA graph of forward + backward replays to the eager result;
  overflow is reported by gc_check; accumulate=1 over two half batches equals one batch.
"""
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
def small():
    rng = np.random.default_rng(71)
    scene = scenes.make_hier_scene(rng, 6000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 3)
    reqs = [
        scenes.Request(scenes.orbit_camera(0.3, 4.0, 200, 150), 1, 0b111111),
        scenes.Request(scenes.orbit_camera(1.9, 4.5, 96, 64), -1, 0b000001),
        scenes.Request(scenes.orbit_camera(4.0, 3.5, 131, 77), 2, 0b000111),   # ragged tiles
        scenes.Request(scenes.orbit_camera(0.3, 4.0, 64, 48), 0, 0),           # empty selection
        scenes.Request(scenes.orbit_camera(5.5, 4.2, 160, 120), 1, 0b110110),  # non-prefix mask
        scenes.Request(scenes.orbit_camera(2.6, 4.0, 120, 90), 2, 0b011111),
    ]
    return scene, motion, reqs


def _frames(gc, motion):
    return [gc.MotionFrame.from_motion(motion, f) for f in range(motion.q.shape[0])]


def _batch_triplets(reqs):
    return [(r.camera, r.frame, r.layer_mask) for r in reqs]


def _single(gc, r, gs, frames, req, up=None):
    saved = gc.Saved(r)
    mo = frames[req.frame] if req.frame >= 0 else None
    img = r.forward(gs, mo, req.layer_mask, req.camera, saved)
    g = None
    if up is not None:
        g = r.backward(saved, gs, mo, up)
    return img, g


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_batch_images_equal_single_renders(gc, small, tile):
    scene, motion, reqs = small
    r = gc.Renderer(0, tile=tile, bg=(0.1, 0.2, 0.3))
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    saved = gc.Saved(r)
    imgs = r.batch_forward(gs, frames, _batch_triplets(reqs), saved)
    r.check()
    for q, req in enumerate(reqs):
        one, _ = _single(gc, r, gs, frames, req)
        assert torch.equal(imgs[q], one), (tile, q)


def test_batch_request_against_oracle(gc, small):
    scene, motion, reqs = small
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    imgs = r.batch_forward(gs, _frames(gc, motion), _batch_triplets(reqs))
    torch.cuda.synchronize()
    for q in (0, 2, 4):
        req = reqs[q]
        ref = oracle.render(scene, motion if req.frame >= 0 else None, max(req.frame, 0), req.camera,
                            oracle.default_options(), req.layer_mask)
        g = imgs[q].cpu().numpy().astype(np.float64)
        ok = ~ref["ambiguous"]
        assert np.abs(g - ref["image"]).max(axis=0)[ok].max() <= 1e-4, q


def _upstreams(reqs, refs, seed):
    rng = np.random.default_rng(seed)
    ups = []
    for req, ref in zip(reqs, refs):
        cam = req.camera
        up = rng.normal(0, 1, (3, cam.height, cam.width)) * (~ref["ambiguous"])[None]
        ups.append(up.astype(np.float32))
    return ups


def test_batch_backward_matches_oracle_and_single_sum(gc, small):
    scene, motion, reqs = small
    opts = oracle.default_options()
    refs, bins = [], []
    for req in reqs:
        mo = motion if req.frame >= 0 else None
        b = oracle.bin_f32(scene, mo, max(req.frame, 0), req.camera, opts, req.layer_mask)
        bins.append(b)
        refs.append(oracle.render(scene, mo, max(req.frame, 0), req.camera, opts, req.layer_mask, bins=b))
    ups = _upstreams(reqs, refs, 5)

    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    saved = gc.Saved(r)
    r.batch_forward(gs, frames, _batch_triplets(reqs), saved)
    dls = [torch.from_numpy(u).cuda() for u in ups]
    got = r.batch_backward(saved, gs, frames, dls)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in got.items()}

    # oracle: FP64 gradients of every request, summed; motion per (frame, group)
    n_frames, G = motion.q.shape[0], motion.q.shape[1]
    want = {k: 0.0 for k in NAMES}
    want["group_q"] = np.zeros((n_frames, G, 4))
    want["group_t"] = np.zeros((n_frames, G, 3))
    for req, up, b in zip(reqs, ups, bins):
        mo = motion if req.frame >= 0 else None
        og = oracle.grad(scene, mo, max(req.frame, 0), req.camera, opts, up.astype(np.float64),
                         req.layer_mask, bins=b)
        for k in NAMES:
            want[k] = want[k] + og[k]
        if req.frame >= 0:
            want["group_q"][req.frame] += og["group_q"]
            want["group_t"][req.frame] += og["group_t"]
    for k in NAMES + ("group_q", "group_t"):
        a, b = got[k], np.asarray(want[k]).reshape(got[k].shape)
        nb = np.linalg.norm(b)
        assert nb > 0, k
        assert np.linalg.norm(a - b) / nb <= 1e-4, (k, np.linalg.norm(a - b) / nb)
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-6, k

    # the in-order sum of single-request GPU gradients (FP32): equal up to the order of
    # the float additions inside each Gaussian's chain rule
    acc = {k: torch.zeros_like(torch.from_numpy(got[k])).cuda().float() for k in got}
    for q, req in enumerate(reqs):
        _, g = _single(gc, r, gs, frames, req, dls[q])
        for k in NAMES:
            acc[k] += g[k]
        if req.frame >= 0:
            acc["group_q"][req.frame] += g["group_q"]
            acc["group_t"][req.frame] += g["group_t"]
    for k in acc:
        a = got[k]
        b = acc[k].cpu().numpy().astype(np.float64)
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max() + 1e-7, k


def test_batch_graph_replay_and_capacity(gc, small):
    scene, motion, reqs = small
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    trip = _batch_triplets(reqs)
    # exact key count from an auto-capacity pass
    r0 = gc.Renderer(0)
    s0 = gc.Saved(r0)
    ref_imgs = r0.batch_forward(gs, frames, trip, s0)
    dls = [torch.randn_like(x) for x in ref_imgs]
    ref_g = r0.batch_backward(s0, gs, frames, dls)
    torch.cuda.synchronize()

    r = gc.Renderer(0, key_capacity=400_000)
    saved = gc.Saved(r)
    stream = torch.cuda.Stream()
    outs = [torch.empty_like(x) for x in ref_imgs]
    grads = r.batch_grads(gs, frames)
    with torch.cuda.stream(stream):
        r.batch_forward(gs, frames, trip, saved, outs=outs)        # eager: sizes and uploads
        r.batch_backward(saved, gs, frames, dls, grads=grads)
    stream.synchronize()
    r.check(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        r.batch_forward(gs, frames, trip, saved, outs=outs)
        r.batch_backward(saved, gs, frames, dls, grads=grads)
    for o in outs:
        o.zero_()
    for v in grads.values():
        v.fill_(7.0)
    graph.replay()
    torch.cuda.synchronize()
    r.check()
    for a, b in zip(outs, ref_imgs):
        assert torch.equal(a, b)
    for k in ref_g:
        assert torch.equal(grads[k], ref_g[k]), k
    # a bound state refuses other requests
    with pytest.raises(gc.GCError):
        r.batch_forward(gs, frames, trip[:3], saved)
    del graph

    # too small a capacity: nothing placed (the images are the background, the backward
    # writes no partial and gives zero gradients), reported by gc_check
    rs = gc.Renderer(0, key_capacity=2048)
    ss = gc.Saved(rs)
    imgs = rs.batch_forward(gs, frames, trip, ss)
    gz = rs.batch_backward(ss, gs, frames, dls)
    torch.cuda.synchronize()
    for x in imgs:
        assert not x.any()
    for k, v in gz.items():
        assert not v.any(), k
    with pytest.raises(gc.GCError, match="capacity"):
        rs.check()


def test_batch_accumulate_over_half_batches(gc, small):
    scene, motion, reqs = small
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    trip = _batch_triplets(reqs)
    r = gc.Renderer(0)
    s_all, s_a, s_b = gc.Saved(r), gc.Saved(r), gc.Saved(r)
    imgs = r.batch_forward(gs, frames, trip, s_all)
    dls = [torch.randn_like(x) for x in imgs]
    full = r.batch_backward(s_all, gs, frames, dls)
    r.batch_forward(gs, frames, trip[:3], s_a)
    r.batch_forward(gs, frames, trip[3:], s_b)
    acc = r.batch_grads(gs, frames)
    r.batch_backward(s_a, gs, frames, dls[:3], grads=acc)
    r.batch_backward(s_b, gs, frames, dls[3:], grads=acc, accumulate=True)
    torch.cuda.synchronize()
    for k in full:
        a, b = acc[k], full[k]
        assert torch.allclose(a, b, rtol=0, atol=1e-5 * float(b.abs().max()) + 1e-7), k


def test_batch_workload_at_scale(gc):
    """500k Gaussians, 16 views x 8 frames = 128 requests of mixed level and resolution:
    eight sampled requests equal their single-request renders bit for bit; gradients are
    finite and the backward is deterministic."""
    w = scenes.batch()
    gs = gc.GaussianSet.from_scene(w.scene)
    frames = _frames(gc, w.motion)
    trip = [(q.camera, q.frame, q.layer_mask) for q in w.requests]
    r = gc.Renderer(0)
    saved = gc.Saved(r)
    imgs = r.batch_forward(gs, frames, trip, saved)
    r.check()
    for q in (0, 9, 31, 50, 77, 100, 126, 127):
        one, _ = _single(gc, r, gs, frames, w.requests[q])
        assert torch.equal(imgs[q], one), q
    gen = torch.Generator(device="cuda").manual_seed(3)
    dls = [torch.randn(x.shape, generator=gen, device="cuda") for x in imgs]
    g1 = r.batch_backward(saved, gs, frames, dls)
    g1 = {k: v.clone() for k, v in g1.items()}
    g2 = r.batch_backward(saved, gs, frames, dls)
    torch.cuda.synchronize()
    for k in g1:
        assert torch.isfinite(g1[k]).all(), k
        assert torch.equal(g1[k], g2[k]), k
    del saved, g1, g2
    # eight requests at full size: batched gradients equal the in-order sum of the
    # single-request gradients up to float summation order
    pick = (3, 20, 45, 64, 90, 101, 118, 125)
    sub = gc.Saved(r)
    r.batch_forward(gs, frames, [trip[q] for q in pick], sub, outs=[imgs[q] for q in pick])
    got = r.batch_backward(sub, gs, frames, [dls[q] for q in pick])
    acc = {k: torch.zeros_like(v) for k, v in got.items()}
    for q in pick:
        req = w.requests[q]
        _, g = _single(gc, r, gs, frames, req, dls[q])
        for k in NAMES:
            acc[k] += g[k]
        acc["group_q"][req.frame] += g["group_q"]
        acc["group_t"][req.frame] += g["group_t"]
    torch.cuda.synchronize()
    for k in acc:
        a, b = got[k], acc[k]
        assert torch.allclose(a, b, rtol=0, atol=1e-5 * float(b.abs().max()) + 1e-7), k


def test_batch_graph_step(gc, small):
    """A step of 6 requests in batches of 2 as one native CUDA graph (three batches on three
    branches of the graph): images equal the single renders bit for bit after a replay;
    gradients equal the eager batches summed in batch order bit for bit, and one eager batch
    over all requests up to float summation order."""
    scene, motion, reqs = small
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    trip = _batch_triplets(reqs)
    r = gc.Renderer(0)
    s_all = gc.Saved(r)
    ref = r.batch_forward(gs, frames, trip, s_all)
    dls = [torch.randn_like(x) for x in ref]
    ref_g = r.batch_backward(s_all, gs, frames, dls)
    torch.cuda.synchronize()
    graph = gc.BatchGraph(r, gs, frames, trip, 2, dL_dimages=dls)
    assert graph.n_batches == 3 and graph.kernel_nodes > 0 and graph.key_capacity % 2048 == 0
    for o in graph.outs:
        o.zero_()
    for v in graph.grads.values():
        v.fill_(3.0)
    graph.launch()
    graph.check()
    for q in range(len(reqs)):
        assert torch.equal(graph.outs[q], ref[q]), q
    for k, b in ref_g.items():
        a = graph.grads[k]
        assert torch.allclose(a, b, rtol=0, atol=1e-5 * float(b.abs().max()) + 1e-7), k
    # the same batches eagerly, one after the other: the branched graph sums in batch order
    seq = r.batch_grads(gs, frames)
    for b in range(3):
        sb = gc.Saved(r)
        r.batch_forward(gs, frames, trip[2 * b:2 * b + 2], sb)
        r.batch_backward(sb, gs, frames, dls[2 * b:2 * b + 2], grads=seq, accumulate=b > 0)
    torch.cuda.synchronize()
    for k in seq:
        assert torch.equal(seq[k], graph.grads[k]), k
    graph.launch()  # replays are deterministic
    g1 = {k: v.clone() for k, v in graph.grads.items()}
    graph.launch()
    graph.check()
    for k in g1:
        assert torch.equal(g1[k], graph.grads[k]), k
    graph.close()


def test_autotuner_picks_a_measured_configuration(gc, small):
    scene, motion, reqs = small
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    trip = _batch_triplets(reqs)
    r = gc.Renderer(0)
    outs = [torch.empty((3, q.camera.height, q.camera.width), device="cuda") for q in reqs]
    dls = [torch.randn_like(x) for x in outs]
    res = r.tune_batch(gs, frames, trip, dL_dimages=dls, depths=(2, 6), iters=2, outs=outs)
    ents = res["entries"]
    assert len(ents) == 6
    assert {e["tile"] for e in ents} == {(16, 16), (8, 32), (32, 8)}
    assert all(e["ms"] > 0 for e in ents)
    best = res["best"]
    assert best["ms"] == min(e["ms"] for e in ents)
    assert (r.options.tile_w, r.options.tile_h) == best["tile"]
    # the tuned renderer still renders every request exactly like the single path
    imgs = r.batch_forward(gs, frames, trip)
    for q, req in enumerate(reqs):
        one, _ = _single(gc, r, gs, frames, req)
        assert torch.equal(imgs[q], one), q


def test_batch_with_a_request_over_255_tile_columns(gc, small):
    """A 4,200 x 1,050 px request (263 columns of 16 px tiles) is past binning by tile row, so the
    batch takes the per-request key sort instead: every image still equals its single render
    (the wide one takes the single path's key sort too), and the gradients the in-order sum of
    the single-request gradients (up to the order of the float additions of the chain rule)."""
    scene, motion, reqs = small
    wide = scenes.Request(scenes.orbit_camera(0.8, 4.0, 4200, 1050), 1, 0b001111)
    reqs = list(reqs[:3]) + [wide] + list(reqs[3:])
    r = gc.Renderer(0)
    gs = gc.GaussianSet.from_scene(scene)
    frames = _frames(gc, motion)
    saved = gc.Saved(r)
    imgs = r.batch_forward(gs, frames, _batch_triplets(reqs), saved)
    gen = torch.Generator(device="cuda").manual_seed(9)
    dls = [torch.randn(x.shape, generator=gen, device="cuda") for x in imgs]
    got = {k: v.clone() for k, v in r.batch_backward(saved, gs, frames, dls).items()}
    r.check()
    acc = {k: torch.zeros_like(v) for k, v in got.items()}
    for q, req in enumerate(reqs):
        one, g = _single(gc, r, gs, frames, req, dls[q])
        assert torch.equal(imgs[q], one), q
        for k in NAMES:
            acc[k] += g[k]
        if req.frame >= 0:
            acc["group_q"][req.frame] += g["group_q"]
            acc["group_t"][req.frame] += g["group_t"]
    torch.cuda.synchronize()
    assert imgs[3].any()
    for k in acc:
        a, b = got[k].double(), acc[k].double()
        assert (a - b).abs().max() <= 1e-5 * b.abs().max() + 1e-7, k
