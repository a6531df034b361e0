"""A multi-frame step of the single-pass multi-level render (Eq. 4 levels of every frame,
Sec. 3.3) as one CUDA graph (gc_levels_graph): replays equal the eager calls (images bit for
bit, per-frame gradients), frames may differ in resolution, and an overflow of the fixed key
capacity in any frame of a step - not only the last one - is reported, eagerly by gc_check
and for the graph by its check and at creation."""
import numpy as np
import pytest
import torch

from synth import scenes

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh", "group_q", "group_t")


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(211)
    scene = scenes.make_hier_scene(rng, 8000, 6, 3, 16)
    motion = scenes.random_motion(rng, 16, 3)
    return scene, motion


def _cams():
    # three frames, three resolutions (the largest first)
    return [scenes.orbit_camera(0.3, 4.0, 248, 152), scenes.orbit_camera(1.1, 4.0, 120, 88),
            scenes.orbit_camera(2.0, 4.0, 200, 136)]


def _setup(gc, small, tile=(8, 32), **kw):
    scene, motion = small
    r = gc.Renderer(0, tile=tile, bg=(0.1, 0.2, 0.3), **kw)
    gs = gc.GaussianSet.from_scene(scene)
    frames = [gc.MotionFrame.from_motion(motion, f) for f in range(3)]
    return r, gs, frames, _cams()


def test_graph_forward_equals_eager(gc, small):
    r, gs, frames, cams = _setup(gc, small)
    L = 6
    eager = [img.clone() for f in range(3) for img in r.levels_forward(gs, frames[f], L, cams[f])]
    g = gc.LevelsGraph(r, gs, frames, cams, L)
    assert g.kernel_nodes >= 3 * 8 and g.key_capacity > 0 and g.key_capacity % 2048 == 0
    for rep in range(2):
        for o in g.outs:
            o.fill_(-1.0)
        g.launch()
        g.check()
        torch.cuda.synchronize()
        for a, b in zip(eager, g.outs):
            assert a.shape == b.shape
            assert torch.equal(a, b), rep
    # the graph reads the motion tables in place: new contents, new images
    scene, motion = small
    moved = scenes.random_motion(np.random.default_rng(5), 16, 3)
    for f in range(3):
        frames[f].q.copy_(torch.from_numpy(moved.q[f]))
        frames[f].t.copy_(torch.from_numpy(moved.t[f]))
    g.launch()
    g.check()
    again = [img.clone() for f in range(3) for img in r.levels_forward(gs, frames[f], L, cams[f])]
    torch.cuda.synchronize()
    for a, b in zip(again, g.outs):
        assert torch.equal(a, b)
    g.close()


def test_graph_forward_backward_per_frame_gradients(gc, small):
    r, gs, frames, cams = _setup(gc, small, tile=(16, 16))
    L = 4
    gen = torch.Generator(device="cuda").manual_seed(9)
    dls = [torch.randn((3, c.height, c.width), generator=gen, device="cuda") for c in cams for _ in range(L)]
    want = []
    for f in range(3):
        saved = gc.Saved(r)
        r.levels_forward(gs, frames[f], L, cams[f], saved)
        gr = r.levels_backward(saved, gs, frames[f], dls[L * f:L * f + L])
        want.append({k: v.clone() for k, v in gr.items()})
    grads = [r._single_grads(gs, frames[f]) for f in range(3)]
    g = gc.LevelsGraph(r, gs, frames, cams, L, dL_dimages=dls, grads=grads)
    for gr in grads:
        for v in gr.values():
            v.fill_(7.0)
    g.launch()
    g.check()
    torch.cuda.synchronize()
    for f in range(3):
        for k in NAMES:
            a, b = grads[f][k], want[f][k]
            rel = float((a - b).norm() / max(float(b.norm()), 1e-30))
            assert rel <= 1e-6, (f, k, rel)
    g.close()


@pytest.mark.parametrize("chains", [2, 3])
def test_chains_equal_one_chain(gc, small, chains):
    """Frames split over independent graph branches (each with its own saved state) give
    the images of one chain bit for bit; with a gradient set shared by every frame the
    backwards stay in frame order, so it ends as the last frame's, equal to one chain's.
    Five frames (uneven over the chains), three resolutions, forward and training step."""
    scene, motion = small
    r = gc.Renderer(0, tile=(8, 32), bg=(0.1, 0.2, 0.3))
    gs = gc.GaussianSet.from_scene(scene)
    frames = [gc.MotionFrame.from_motion(motion, f % 3) for f in range(5)]
    cams = [_cams()[f % 3] for f in range(5)]
    L = 6
    gen = torch.Generator(device="cuda").manual_seed(17)
    dls = [torch.randn((3, c.height, c.width), generator=gen, device="cuda") for c in cams for _ in range(L)]
    results = []
    for nc in (1, chains):
        shared = r._single_grads(gs, frames[0])
        own = [r._single_grads(gs, frames[f]) for f in range(5)]
        gf = gc.LevelsGraph(r, gs, frames, cams, L, chains=nc)
        gs_ = gc.LevelsGraph(r, gs, frames, cams, L, dL_dimages=dls, grads=[shared] * 5, chains=nc)
        go = gc.LevelsGraph(r, gs, frames, cams, L, dL_dimages=dls, grads=own, chains=nc)
        for g in (gf, gs_, go):
            for o in g.outs:
                o.fill_(-1.0)
            g.launch()
            g.check()
        torch.cuda.synchronize()
        results.append(([o.clone() for o in gf.outs], {k: v.clone() for k, v in shared.items()},
                        [{k: v.clone() for k, v in gr.items()} for gr in own]))
        for g in (gf, gs_, go):
            g.close()
    (i1, s1, o1), (i2, s2, o2) = results
    for a, b in zip(i1, i2):
        assert torch.equal(a, b)
    for k in NAMES:
        assert torch.equal(s1[k], s2[k]), k
        for f in range(5):
            assert torch.equal(o1[f][k], o2[f][k]), (f, k)


def test_overflow_in_any_frame_is_reported(gc, small):
    r0, gs, frames, cams = _setup(gc, small)
    need = []
    for f in range(3):
        r0.levels_forward(gs, frames[f], 6, cams[f])
        need.append(r0.stats()["n_keys"])
    assert need[0] > need[1] and need[0] > need[2]
    cap = (need[0] + max(need[1], need[2])) // 2   # enough for frames 1 and 2, not for frame 0
    r, gs, frames, cams = _setup(gc, small, key_capacity=cap)
    for f in range(3):
        r.levels_forward(gs, frames[f], 6, cams[f])
    with pytest.raises(gc.GCError, match="capacity"):
        r.check()
    # the record is cleared by the check; frames within the capacity pass
    for f in (1, 2):
        r.levels_forward(gs, frames[f], 6, cams[f])
    r.check()
    # a graph at that capacity is refused at creation (its eager pass overflows in frame 0)
    with pytest.raises(gc.GCError, match="capacity"):
        gc.LevelsGraph(r, gs, frames, cams, 6)
    # and a graph whose capacity fits every frame replays cleanly
    r.set_options(key_capacity=need[0] + 4096)
    g = gc.LevelsGraph(r, gs, frames, cams, 6)
    g.launch()
    g.check()
    g.close()


def test_capacity_change_keeps_the_overflow_record_exact(gc, small):
    """Only overflows are recorded: counts that fitted an earlier, larger capacity do not fail
    a check after the capacity shrinks, and an overflow under a small capacity is still
    reported after the capacity grows."""
    r0, gs, frames, cams = _setup(gc, small)
    need = []
    for f in range(3):
        r0.levels_forward(gs, frames[f], 6, cams[f])
        need.append(r0.stats()["n_keys"])
    small_cap = (need[0] + max(need[1], need[2])) // 2   # fits frames 1 and 2, not frame 0
    r, gs, frames, cams = _setup(gc, small, key_capacity=need[0] + 4096)
    r.levels_forward(gs, frames[0], 6, cams[0])           # fits the large capacity
    r.set_options(key_capacity=small_cap)
    for f in (1, 2):
        r.levels_forward(gs, frames[f], 6, cams[f])
    r.check()                                             # no frame overflowed
    r.levels_forward(gs, frames[0], 6, cams[0])           # overflows the small capacity
    r.set_options(key_capacity=need[0] + 4096)
    r.levels_forward(gs, frames[1], 6, cams[1])
    with pytest.raises(gc.GCError, match="capacity"):
        r.check()
    r.levels_forward(gs, frames[2], 6, cams[2])
    r.check()                                             # the record was cleared by the check


def test_graph_argument_errors(gc, small):
    r, gs, frames, cams = _setup(gc, small)
    with pytest.raises(ValueError):
        gc.LevelsGraph(r, gs, frames[:2], cams, 6)
    with pytest.raises(ValueError):
        gc.LevelsGraph(r, gs, [frames[0], None, frames[2]], cams, 6)
    with pytest.raises(gc.GCError):
        gc.LevelsGraph(r, gs, frames, cams, 0)


def test_graph_shared_gradient_set_and_static_scene(gc, small):
    """One gradient set named by every frame holds the last frame's gradients; a step without
    motion tables (static scene) replays like its eager calls."""
    r, gs, frames, cams = _setup(gc, small, tile=(16, 16))
    L = 3
    gen = torch.Generator(device="cuda").manual_seed(19)
    dls = [torch.randn((3, c.height, c.width), generator=gen, device="cuda") for c in cams for _ in range(L)]
    saved = gc.Saved(r)
    r.levels_forward(gs, frames[2], L, cams[2], saved)
    want = {k: v.clone() for k, v in r.levels_backward(saved, gs, frames[2], dls[2 * L:3 * L]).items()}
    shared = r._single_grads(gs, frames[0])
    g = gc.LevelsGraph(r, gs, frames, cams, L, dL_dimages=dls, grads=[shared] * 3)
    g.launch()
    g.check()
    torch.cuda.synchronize()
    for k in NAMES:
        rel = float((shared[k] - want[k]).norm() / max(float(want[k].norm()), 1e-30))
        assert rel <= 1e-6, (k, rel)
    g.close()
    static = [None, None, None]
    eager = [img.clone() for f in range(3) for img in r.levels_forward(gs, None, L, cams[f])]
    gs_static = gc.LevelsGraph(r, gs, static, cams, L)
    gs_static.launch()
    gs_static.check()
    torch.cuda.synchronize()
    for a, b in zip(eager, gs_static.outs):
        assert torch.equal(a, b)
    gs_static.close()
