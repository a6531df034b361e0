"""The allocation-free forward entry point (gc_render_forward_noalloc).

It serves callers that cannot allocate device memory while rendering (a
playback thread with a frame deadline, plugins inside another application's
CUDA context under a fixed memory budget): all its scratch is one static device
array in the library.  This file is collected last.  Two calls in a row, on
different scenes, cameras and layer masks, must each give the image of the
regular entry point gc_render_forward under the same options bit for bit (both
run the same kernels on the same sorted lists).  Requests beyond the stated
maximum are refused with GC_ERR_CAPACITY and leave the image untouched: the
selection, pixel and tile limits before any GPU work, the pair limit after the
depth sort and scan have counted the pairs.  An empty selection gives the
background.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import scenes

pytestmark = pytest.mark.gpu

GC_ERR_CAPACITY = 3


def _noalloc(gs, mo, mask, cam, opts=None):
    from paper_2509_17513_b300 import _abi
    from paper_2509_17513_b300.render import camera_struct
    cs = camera_struct(cam)
    img = torch.full((3, cam.height, cam.width), float("nan"), device="cuda")
    err = C.create_string_buffer(256)
    st = _abi.lib().gc_render_forward_noalloc(
        C.byref(opts) if opts is not None else None, C.byref(gs.struct),
        C.byref(mo.struct) if mo is not None else None, mask, C.byref(cs),
        C.c_void_p(img.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream),
        err, C.sizeof(err))
    return st, img, err.value.decode()


def test_noalloc_matches_regular_forward_twice():
    import paper_2509_17513_b300 as gc
    from paper_2509_17513_b300 import _abi
    # call 1: the tiny scene, no motion, black background, NULL options (= gc_default_options)
    w = scenes.tiny()
    cam1 = w.cameras[0]
    gs1 = gc.GaussianSet.from_scene(w.scene)
    st, a1, msg = _noalloc(gs1, None, 1, cam1)
    assert st == 0, msg
    # call 2: a layered SH-3 scene with group motion, a ragged image, a non-prefix mask, a
    # background and 8x32 tiles; the array still holds call 1's contents
    rng = np.random.default_rng(41)
    sc = scenes.make_hier_scene(rng, 20000, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 3)
    cam2 = scenes.orbit_camera(0.8, 4.0, 200, 136)
    gs2 = gc.GaussianSet.from_scene(sc)
    mo2 = gc.MotionFrame.from_motion(motion, 2)
    o = _abi.Options()
    _abi.lib().gc_default_options(C.byref(o))
    o.tile_w, o.tile_h = 8, 32
    o.bg[0], o.bg[1], o.bg[2] = 0.1, 0.2, 0.3
    st, a2, msg = _noalloc(gs2, mo2, 0b110101, cam2, o)
    assert st == 0, msg
    torch.cuda.synchronize()

    r1 = gc.Renderer(0)  # the library defaults
    b1 = r1.forward(gs1, None, 1, cam1)
    r2 = gc.Renderer(0, tile=(8, 32), bg=(0.1, 0.2, 0.3))
    b2 = r2.forward(gs2, mo2, 0b110101, cam2)
    torch.cuda.synchronize()
    for a, b in ((a1, b1), (a2, b2)):
        assert torch.isfinite(a).all()
        assert torch.equal(a, b), (a - b).abs().max().item()
    assert (a1.mean() > 0.01).item() and (a2.mean() > 0.01).item()
    r1.close()
    r2.close()


def test_noalloc_refuses_oversized_requests():
    import paper_2509_17513_b300 as gc
    rng = np.random.default_rng(3)
    sc = scenes.make_hier_scene(rng, 40000, 1, 0, 1)   # 40,000 > 32,768 selected
    gs = gc.GaussianSet.from_scene(sc)
    cam = scenes.orbit_camera(0.0, 4.0, 64, 64)
    st, img, msg = _noalloc(gs, None, 1, cam)
    assert st == GC_ERR_CAPACITY and "32768" in msg
    torch.cuda.synchronize()
    assert torch.isnan(img).all()                       # nothing written
    small = gc.GaussianSet.from_scene(scenes.tiny(n=100).scene)
    big = scenes.orbit_camera(0.0, 4.0, 1024, 1024)     # 1,048,576 > 262,144 pixels
    st, img, msg = _noalloc(small, None, 1, big)
    assert st == GC_ERR_CAPACITY and "262144" in msg
    # the tile limit: within the pixel limit only partial tiles exceed 4,096 tiles, e.g. a
    # 1 x 262,144 image in 8 x 32 tiles is 1 x 8,192 tiles
    from paper_2509_17513_b300 import _abi
    o = _abi.Options()
    _abi.lib().gc_default_options(C.byref(o))
    o.tile_w, o.tile_h = 8, 32
    thin = scenes.look_at_camera((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 1, 262144)
    st, img, msg = _noalloc(small, None, 1, thin, o)
    assert st == GC_ERR_CAPACITY and "4096 tiles" in msg


def test_noalloc_refuses_too_many_pairs_and_renders_empty_selection():
    import paper_2509_17513_b300 as gc
    # 30,000 large, nearly opaque Gaussians filling a 512 x 512 view: within the selection
    # and pixel limits, but each covers about a hundred 16 x 16 tiles (> 1,048,576 pairs)
    rng = np.random.default_rng(17)
    n = 30000
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sc = scenes.Scene(means, np.full((n, 3), -1.5, np.float32), q.astype(np.float32),
                      np.full(n, 3.0, np.float32), rng.uniform(0.0, 1.0, (n, 1, 3)).astype(np.float32),
                      np.zeros(n, np.int32), np.array([0, n // 2, n], np.int64), 0)
    gs = gc.GaussianSet.from_scene(sc)
    cam = scenes.orbit_camera(0.3, 4.0, 512, 512)
    r = gc.Renderer(0)
    r.forward(gs, None, 0b11, cam)
    torch.cuda.synchronize()
    need = r.stats()["n_keys"]
    assert need > (1 << 20), need
    st, img, msg = _noalloc(gs, None, 0b11, cam)
    assert st == GC_ERR_CAPACITY and str(need) in msg and "1048576" in msg
    torch.cuda.synchronize()
    assert torch.isnan(img).all()                       # refused before the blend
    # an empty selection (no layer bit set) and an empty set give the background
    from paper_2509_17513_b300 import _abi
    o = _abi.Options()
    _abi.lib().gc_default_options(C.byref(o))
    o.bg[0], o.bg[1], o.bg[2] = 0.25, 0.5, 0.75
    for g_set, mask in ((gs, 0b100), (gc.GaussianSet.from_scene(sc.subset(np.arange(0))), 1)):
        st, img, msg = _noalloc(g_set, None, mask, cam, o)
        assert st == 0, msg
        torch.cuda.synchronize()
        bg = torch.tensor([0.25, 0.5, 0.75], device="cuda").view(3, 1, 1).expand_as(img)
        assert torch.equal(img, bg)
    r.close()
