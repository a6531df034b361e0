"""The allocation-free forward entry point (gc_render_forward_noalloc).

It serves callers that cannot allocate device memory while rendering (a
playback thread with a frame deadline, code capturing a CUDA graph, plugins
under a fixed memory budget): all its scratch is one static device array in
the library.  This file is collected last.  Two calls in a row, on different
scenes, cameras and layer masks, must each match the regular entry point
gc_render_forward within the tolerance of the other parity tests (1e-4), and
requests beyond the stated maximum must be refused before any GPU work.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _noalloc(gc, gs, mo, mask, cam, opts=None):
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
    # call 1: the tiny scene, no motion, black background, default options
    w = scenes.tiny()
    cam1 = w.cameras[0]
    gs1 = gc.GaussianSet.from_scene(w.scene)
    st, a1, msg = _noalloc(gc, gs1, None, 1, cam1)
    assert st == 0, msg
    # call 2: a layered SH-3 scene with group motion, a ragged image, a non-prefix mask, a
    # background and 8x32 tiles; the array still holds call 1's contents
    rng = np.random.default_rng(41)
    sc = scenes.make_hier_scene(rng, 20000, 6, 3, 8)
    motion = scenes.random_motion(rng, 8, 3)
    cam2 = scenes.orbit_camera(0.8, 4.0, 200, 136)
    gs2 = gc.GaussianSet.from_scene(sc)
    mo2 = gc.MotionFrame.from_motion(motion, 2)
    from paper_2509_17513_b300 import _abi
    o = _abi.Options()
    _abi.lib().gc_default_options(C.byref(o))
    o.tile_w, o.tile_h = 8, 32
    o.bg[0], o.bg[1], o.bg[2] = 0.1, 0.2, 0.3
    st, a2, msg = _noalloc(gc, gs2, mo2, 0b110101, cam2, o)
    assert st == 0, msg
    torch.cuda.synchronize()

    r1 = gc.Renderer(0)
    b1 = r1.forward(gs1, None, 1, cam1)
    r2 = gc.Renderer(0, tile=(8, 32), bg=(0.1, 0.2, 0.3))
    b2 = r2.forward(gs2, mo2, 0b110101, cam2)
    torch.cuda.synchronize()
    for a, b in ((a1, b1), (a2, b2)):
        assert torch.isfinite(a).all()
        assert (a - b).abs().max().item() <= TOL
    assert (a1.mean() > 0.01).item() and (a2.mean() > 0.01).item()


def test_noalloc_refuses_oversized_requests():
    import paper_2509_17513_b300 as gc
    rng = np.random.default_rng(3)
    sc = scenes.make_hier_scene(rng, 40000, 1, 0, 1)   # 40,000 > 32,768 selected
    gs = gc.GaussianSet.from_scene(sc)
    cam = scenes.orbit_camera(0.0, 4.0, 64, 64)
    st, img, msg = _noalloc(gc, gs, None, 1, cam)
    assert st == 3 and "32768" in msg
    assert torch.isnan(img).all()                       # nothing written
    small = gc.GaussianSet.from_scene(scenes.tiny(n=100).scene)
    big = scenes.orbit_camera(0.0, 4.0, 1024, 1024)     # 1,048,576 > 262,144 pixels
    st, img, msg = _noalloc(gc, small, None, 1, big)
    assert st == 3 and "262144" in msg
