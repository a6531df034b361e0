"""Thin PyTorch binding of the C ABI: marshals tensors into gc4d.h structs.

PyTorch provides device memory and the stream; every step of the render runs
in libgc4d.so.  ``Renderer.forward`` / ``Renderer.backward`` are the two calls
of the boundary; ``render`` is a ``torch.autograd.Function`` on top of them.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import check, lib

ATTRS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def camera_struct(cam) -> _abi.Camera:
    """Any object with width, height, fx, fy, cx, cy, R (3x3), t (3), campos (3)."""
    c = _abi.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float32).reshape(-1)
    for k in range(9):
        c.R[k] = float(R[k])
    t = np.asarray(cam.t, np.float32).reshape(-1)
    p = np.asarray(cam.campos, np.float32).reshape(-1)
    for k in range(3):
        c.t[k] = float(t[k])
        c.campos[k] = float(p[k])
    return c


class GaussianSet:
    """Device tensors of a Gaussian set plus the host struct that points at them.

    FP32: ``means`` (N,3), ``log_scales`` (N,3), ``quats`` (N,4), ``opacity_logits``
    (N,), ``sh`` (N,K,3), optional ``group_id`` (N,) int32.  Reduced precision:
    ``means_bf16`` etc. as int16/uint8 bit patterns plus ``scales``.
    """

    def __init__(self, layer_offsets, sh_degree: int, precision: int = _abi.GC_PREC_FP32, **t):
        self.tensors = {k: v for k, v in t.items() if v is not None}
        for k, v in self.tensors.items():
            if not v.is_cuda or not v.is_contiguous():
                raise ValueError(f"{k} must be a contiguous CUDA tensor")
        self.layer_offsets = np.ascontiguousarray(np.asarray(layer_offsets, np.int64))
        self.sh_degree = int(sh_degree)
        self.precision = int(precision)
        s = _abi.Gaussians()
        s.n = int(self.layer_offsets[-1])
        s.n_layers = len(self.layer_offsets) - 1
        s.layer_offsets = self.layer_offsets.ctypes.data
        s.sh_degree = self.sh_degree
        s.precision = self.precision
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh", "group_id",
                     "means_bf16", "log_scales_bf16", "quats_bf16", "opacity_bf16", "sh_e4m3",
                     "scales"):
            v = self.tensors.get(name)
            setattr(s, name, None if v is None else v.data_ptr())
        self.struct = s

    @property
    def n(self) -> int:
        return int(self.layer_offsets[-1])

    @staticmethod
    def from_scene(scene, device="cuda") -> "GaussianSet":
        def f(a):
            return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return GaussianSet(scene.layer_offsets, scene.sh_degree, _abi.GC_PREC_FP32,
                           means=f(scene.means), log_scales=f(scene.log_scales),
                           quats=f(scene.quats), opacity_logits=f(scene.opacity_logits),
                           sh=f(scene.sh),
                           group_id=torch.from_numpy(np.ascontiguousarray(scene.group_id, np.int32)).to(device))

    @staticmethod
    def from_planes(planes: dict, scene, device="cuda") -> "GaussianSet":
        """Set in the paper's decoded attribute format (Sec. 3.4) from
        ``synth.scenes.quantize_planes`` output: per layer a uint8 plane buffer and a
        uint16/uint32 position plane buffer, plus the (lo, step) dequantisation table."""
        gs = GaussianSet(scene.layer_offsets, scene.sh_degree, _abi.GC_PREC_PLANES,
                         dequant=torch.from_numpy(np.ascontiguousarray(planes["dequant"], np.float32)).to(device),
                         group_id=torch.from_numpy(np.ascontiguousarray(scene.group_id, np.int32)).to(device))
        L = len(planes["u8"])
        gs.plane_tensors = []
        u8p = (C.c_void_p * L)()
        posp = (C.c_void_p * L)()
        for l in range(L):
            a = torch.from_numpy(np.ascontiguousarray(planes["u8"][l])).to(device)
            pos = np.ascontiguousarray(planes["pos"][l])
            p = torch.from_numpy(pos.view(np.int16) if pos.dtype == np.uint16 else pos.view(np.int32)).to(device)
            gs.plane_tensors += [a, p]
            u8p[l] = a.data_ptr() if a.numel() else None
            posp[l] = p.data_ptr() if p.numel() else None
        gs.plane_ptrs = (u8p, posp)
        s = gs.struct
        s.plane_width = int(planes["plane_width"])
        s.pos_bits = int(planes["pos_bits"])
        s.plane_pitch = int(planes["pitch"])
        s.pos_pitch = int(planes["pos_pitch"])
        s.planes_u8 = C.cast(u8p, C.c_void_p).value
        s.planes_pos = C.cast(posp, C.c_void_p).value
        s.dequant = gs.tensors["dequant"].data_ptr()
        return gs

    @staticmethod
    def from_quantized(q: dict, scene, device="cuda") -> "GaussianSet":
        """Reduced-precision set from ``synth.scenes.quantize_scene`` output."""
        def u16(a):
            return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).to(device)
        scales = np.concatenate([q["means_scale"], q["log_scales_scale"], q["quats_scale"],
                                 q["opacity_scale"], q["sh_scale"].reshape(-1)]).astype(np.float32)
        return GaussianSet(scene.layer_offsets, scene.sh_degree, _abi.GC_PREC_BF16_FP8,
                           means_bf16=u16(q["means"]), log_scales_bf16=u16(q["log_scales"]),
                           quats_bf16=u16(q["quats"]), opacity_bf16=u16(q["opacity_logits"]),
                           sh_e4m3=torch.from_numpy(np.ascontiguousarray(q["sh"])).to(device),
                           scales=torch.from_numpy(scales).to(device),
                           group_id=torch.from_numpy(np.ascontiguousarray(scene.group_id, np.int32)).to(device))


class MotionFrame:
    """One frame: cumulative group motion q (G,4), t (G,3) (both None: no group motion) and,
    optionally, the frame's residual deformation (Sec. 3.2, Eq. 7) as CUDA float32 tensors
    res_log_scales (n,3), res_opacity_logits (n,), res_sh (n,K,3), each None for none."""

    def __init__(self, q: torch.Tensor | None, t: torch.Tensor | None, res_log_scales=None,
                 res_opacity_logits=None, res_sh=None, per_gaussian: bool = False):
        self.q = q.contiguous() if q is not None else None
        self.t = t.contiguous() if t is not None else None
        self.res = [x.contiguous() if x is not None else None
                    for x in (res_log_scales, res_opacity_logits, res_sh)]
        s = _abi.Motion()
        s.n_groups = int(q.shape[0]) if q is not None else 1
        s.q = self.q.data_ptr() if q is not None else None
        s.t = self.t.data_ptr() if t is not None else None
        s.res_log_scales, s.res_opacity_logits, s.res_sh = [x.data_ptr() if x is not None else None
                                                            for x in self.res]
        s.per_gaussian = 1 if per_gaussian else 0
        self.struct = s

    @staticmethod
    def from_motion(motion, frame: int, device="cuda", residual=None) -> "MotionFrame":
        """Frame `frame` of a synthetic motion (None: no group motion), with an optional
        residual (an object with ls, logit, sh arrays, any None)."""
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device) if a is not None else None
        q = dev(motion.q[frame]) if motion is not None else None
        t = dev(motion.t[frame]) if motion is not None else None
        if residual is None:
            return MotionFrame(q, t)
        return MotionFrame(q, t, dev(residual.ls), dev(residual.logit), dev(residual.sh))


class MotionField:
    """Parameters of a per-Gaussian motion source (Sec. 3.2): hash-grid table (L, T, 2) and the
    translation / rotation MLPs, as CUDA float32 tensors (``synth.scenes.motion_field_params``
    layout), plus the level resolutions and the box of the positions."""

    NAMES = ("table", "w1t", "b1t", "w2t", "b2t", "w1r", "b1r", "w2r", "b2r")

    def __init__(self, params: dict, device="cuda"):
        self.t = {k: torch.as_tensor(np.ascontiguousarray(params[k], np.float32)).to(device).contiguous()
                  for k in self.NAMES}
        L, T, _ = self.t["table"].shape
        s = _abi.MotionField()
        s.n_levels = int(L)
        s.log2_table = int(T).bit_length() - 1
        for l, r in enumerate(np.asarray(params["res"]).tolist()):
            s.resolution[l] = int(r)
        for a in range(3):
            s.lo[a] = float(params["lo"][a])
            s.hi[a] = float(params["hi"][a])
        for k in self.NAMES:
            setattr(s, k, self.t[k].data_ptr())
        self.struct = s


class Saved:
    """A library-owned saved forward state (for the backward pass)."""

    def __init__(self, renderer: "Renderer"):
        self.renderer = renderer
        h = C.c_void_p()
        check(lib().gc_saved_create(renderer.ctx, C.byref(h)), renderer.ctx)
        self.handle = h

    def __del__(self):
        try:
            if self.handle and self.renderer.ctx:
                lib().gc_saved_destroy(self.renderer.ctx, self.handle)
                self.handle = None
        except Exception:
            pass


class Renderer:
    """A gc4d context on one CUDA device."""

    def __init__(self, device: int = 0, tile=(16, 16), near=0.2, dilation=0.3, clamp=1.3,
                 bg=(0.0, 0.0, 0.0), membership: int = _abi.GC_MEMBER_PIXEL,
                 key_capacity: int = 0, alpha_cull: bool = True):
        L = lib()
        o = _abi.Options()
        check(L.gc_default_options(C.byref(o)))
        o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
        o.near_plane, o.dilation, o.frustum_clamp = near, dilation, clamp
        for k in range(3):
            o.bg[k] = float(bg[k])
        o.membership = int(membership)
        o.key_capacity = int(key_capacity)
        o.alpha_cull = 1 if alpha_cull else 0
        self.options = o
        self.device = int(device)
        h = C.c_void_p()
        check(L.gc_create(C.byref(h), self.device, C.byref(o)))
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            lib().gc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        o = self.options
        if "tile" in kw:
            o.tile_w, o.tile_h = kw["tile"]
        if "key_capacity" in kw:
            o.key_capacity = int(kw["key_capacity"])
        if "bg" in kw:
            for k in range(3):
                o.bg[k] = float(kw["bg"][k])
        if "membership" in kw:
            o.membership = int(kw["membership"])
        if "alpha_cull" in kw:
            o.alpha_cull = 1 if kw["alpha_cull"] else 0
        check(lib().gc_set_options(self.ctx, C.byref(o)), self.ctx)

    def forward(self, gs: GaussianSet, motion: MotionFrame | None, layer_mask: int, camera,
                saved: Saved | None = None, out: torch.Tensor | None = None, stream=None):
        cam = camera_struct(camera)
        if out is None:
            out = torch.empty((3, cam.height, cam.width), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        st = lib().gc_render_forward(self.ctx, C.byref(gs.struct),
                                     C.byref(motion.struct) if motion is not None else None,
                                     int(layer_mask) & 0xFFFFFFFF, C.byref(cam), _ptr(out),
                                     saved.handle if saved is not None else None, _stream(stream))
        check(st, self.ctx)
        return out

    def backward(self, saved: Saved | None, gs: GaussianSet, motion: MotionFrame | None,
                 dL_dimage: torch.Tensor, grads: dict | None = None, stream=None) -> dict:
        dev = f"cuda:{self.device}"
        K = (gs.sh_degree + 1) ** 2
        n = gs.n
        if grads is None:
            grads = {"means": torch.empty((n, 3), device=dev), "log_scales": torch.empty((n, 3), device=dev),
                     "quats": torch.empty((n, 4), device=dev), "opacity_logits": torch.empty(n, device=dev),
                     "sh": torch.empty((n, K, 3), device=dev)}
            if motion is not None and motion.q is not None:
                G = motion.q.shape[0]
                grads["group_q"] = torch.empty((G, 4), device=dev)
                grads["group_t"] = torch.empty((G, 3), device=dev)
        g = _abi.Grads()
        g.d_means = grads["means"].data_ptr() if "means" in grads else None
        g.d_log_scales = grads["log_scales"].data_ptr() if "log_scales" in grads else None
        g.d_quats = grads["quats"].data_ptr() if "quats" in grads else None
        g.d_opacity_logits = grads["opacity_logits"].data_ptr() if "opacity_logits" in grads else None
        g.d_sh = grads["sh"].data_ptr() if "sh" in grads else None
        g.d_group_q = grads["group_q"].data_ptr() if "group_q" in grads else None
        g.d_group_t = grads["group_t"].data_ptr() if "group_t" in grads else None
        dl = dL_dimage.contiguous()
        st = lib().gc_render_backward(self.ctx, saved.handle if saved is not None else None,
                                      C.byref(gs.struct),
                                      C.byref(motion.struct) if motion is not None else None,
                                      _ptr(dl), C.byref(g), _stream(stream))
        check(st, self.ctx)
        return grads

    # ---- multi-level render -----------------------------------------------------------

    def levels_forward(self, gs: GaussianSet, motion: MotionFrame | None, levels: int, camera,
                       saved: Saved | None = None, outs: list | None = None, stream=None) -> list:
        """Levels 1..levels of one view in one pass; returns one (3, H, W) image per level."""
        cam = camera_struct(camera)
        if outs is None:
            outs = [torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=f"cuda:{self.device}")
                    for _ in range(levels)]
        ptrs = (C.c_void_p * levels)(*[o.data_ptr() for o in outs])
        st = lib().gc_render_levels_forward(self.ctx, C.byref(gs.struct),
                                            C.byref(motion.struct) if motion is not None else None, int(levels),
                                            C.byref(cam), ptrs, saved.handle if saved is not None else None,
                                            _stream(stream))
        check(st, self.ctx)
        return outs

    def levels_backward(self, saved: Saved | None, gs: GaussianSet, motion: MotionFrame | None,
                        dL_dimages: list, grads: dict | None = None, stream=None) -> dict:
        """Gradients of sum_l <dL_dimages[l], image_l> of a multi-level forward."""
        if grads is None:
            grads = self._single_grads(gs, motion)
        g = self._grads_struct(grads)
        dls = [d.contiguous() for d in dL_dimages]
        ptrs = (C.c_void_p * len(dls))(*[d.data_ptr() for d in dls])
        st = lib().gc_render_levels_backward(self.ctx, saved.handle if saved is not None else None,
                                             C.byref(gs.struct), C.byref(motion.struct) if motion is not None else None,
                                             ptrs, C.byref(g), _stream(stream))
        check(st, self.ctx)
        return grads

    def _single_grads(self, gs: GaussianSet, motion: MotionFrame | None) -> dict:
        dev = f"cuda:{self.device}"
        K = (gs.sh_degree + 1) ** 2
        n = gs.n
        grads = {"means": torch.empty((n, 3), device=dev), "log_scales": torch.empty((n, 3), device=dev),
                 "quats": torch.empty((n, 4), device=dev), "opacity_logits": torch.empty(n, device=dev),
                 "sh": torch.empty((n, K, 3), device=dev)}
        if motion is not None and motion.q is not None:
            G = motion.q.shape[0]
            grads["group_q"] = torch.empty((G, 4), device=dev)
            grads["group_t"] = torch.empty((G, 3), device=dev)
        return grads

    # ---- per-Gaussian motion source ---------------------------------------------------

    def motion_field_forward(self, field: "MotionField", means: torch.Tensor, encodings: torch.Tensor | None = None,
                             stream=None):
        """(q (n,4), t (n,3)): each Gaussian's rotation and translation from the motion source
        at the frame t-1 positions ``means``; use as MotionFrame(q, t, per_gaussian=True).
        encodings: optional (n, 32) FP32 tensor that receives the hash-grid encodings for
        motion_field_backward (a training step)."""
        n = int(means.shape[0])
        dev = means.device
        q = torch.empty((n, 4), device=dev)
        t = torch.empty((n, 3), device=dev)
        if encodings is None:
            check(lib().gc_motion_field_forward(self.ctx, C.byref(field.struct), means.contiguous().data_ptr(), n,
                                                q.data_ptr(), t.data_ptr(), _stream(stream)), self.ctx)
        else:
            check(lib().gc_motion_field_forward_save(self.ctx, C.byref(field.struct), means.contiguous().data_ptr(),
                                                     n, q.data_ptr(), t.data_ptr(), encodings.data_ptr(),
                                                     _stream(stream)), self.ctx)
        return q, t

    def motion_field_backward(self, field: "MotionField", means: torch.Tensor, d_q: torch.Tensor,
                              d_t: torch.Tensor, encodings: torch.Tensor | None = None, stream=None) -> dict:
        """Gradients of the motion source's table and weights given dL/dq, dL/dt; with the
        forward's saved ``encodings`` the table is not gathered again."""
        g = {k: torch.empty_like(v) for k, v in field.t.items()}
        s = _abi.MotionFieldGrads()
        for k in MotionField.NAMES:
            setattr(s, k, g[k].data_ptr())
        args = (self.ctx, C.byref(field.struct), means.contiguous().data_ptr(), int(means.shape[0]))
        tail = (d_q.contiguous().data_ptr(), d_t.contiguous().data_ptr(), C.byref(s), _stream(stream))
        if encodings is None:
            check(lib().gc_motion_field_backward(*args, *tail), self.ctx)
        else:
            check(lib().gc_motion_field_backward_saved(*args, encodings.data_ptr(), *tail), self.ctx)
        return g

    # ---- KDE rate estimate --------------------------------------------------------------

    def kde_rate(self, y: torch.Tensor, stream=None) -> torch.Tensor:
        """Bits per symbol of every row of ``y`` (C, N) under the Silverman-bandwidth kernel
        density of its rounded values (Sec. 3.3); NaN for an unsupported row."""
        y = y.contiguous()
        C_, N = int(y.shape[0]), int(y.shape[1])
        out = torch.empty(C_, device=y.device)
        check(lib().gc_kde_rate(self.ctx, y.data_ptr(), C_, N, N, out.data_ptr(), _stream(stream)), self.ctx)
        return out

    def kde_rate_grad(self, y: torch.Tensor, d_rate: torch.Tensor | None = None, grad: bool = True,
                      stream=None):
        """Training form of the rate (Sec. 3.3): ``y`` (C, N) holds noise-injected values; the
        density of their rounded values is held fixed and the rate is taken at the values
        themselves.  Returns (rate (C,), dL/dy (C, N) or None), dL/dy = d_rate[c] dR_c/dy
        (d_rate None = ones)."""
        y = y.contiguous()
        C_, N = int(y.shape[0]), int(y.shape[1])
        out = torch.empty(C_, device=y.device)
        dy = torch.empty_like(y) if grad else None
        dr = d_rate.contiguous() if d_rate is not None else None
        check(lib().gc_kde_rate_grad(self.ctx, y.data_ptr(), C_, N, N, dr.data_ptr() if dr is not None else None,
                                     out.data_ptr(), dy.data_ptr() if dy is not None else None, _stream(stream)),
              self.ctx)
        return out, dy

    # ---- L1 photometric loss ------------------------------------------------------------

    def l1_loss(self, image: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None,
                loss: torch.Tensor | None = None, scale: float | None = None, stream=None):
        """Mean (or ``scale``-weighted) L1 distance of ``image`` to ``target`` and its gradient
        scale * sign(image - target), written into ``grad`` (allocated when None) and ``loss``
        (a one-element device tensor, allocated when None).  Returns (loss, grad)."""
        if image.shape != target.shape or not image.is_contiguous() or not target.is_contiguous():
            raise ValueError("image and target must be contiguous and of the same shape")
        n = image.numel()
        grad = torch.empty_like(image) if grad is None else grad
        loss = torch.empty(1, device=image.device) if loss is None else loss
        s = (1.0 / n if n else 1.0) if scale is None else float(scale)
        check(lib().gc_l1_loss(self.ctx, image.data_ptr(), target.data_ptr(), n, s, grad.data_ptr(),
                               loss.data_ptr(), _stream(stream)), self.ctx)
        return loss, grad

    # ---- batched requests -------------------------------------------------------------

    def batch_forward(self, gs: GaussianSet, frames: list, requests: list, saved: Saved | None = None,
                      outs: list | None = None, stream=None) -> list:
        """Renders every request (camera, frame index or -1, layer mask) of one Gaussian set
        in one batched pass; returns one (3, H, W) image per request."""
        reqs, outs = self._requests(requests, outs)
        fr, nf = self._frames(frames)
        st = lib().gc_render_batch_forward(self.ctx, C.byref(gs.struct), fr, nf,
                                           reqs, len(requests), saved.handle if saved is not None else None,
                                           _stream(stream))
        check(st, self.ctx)
        return outs

    def batch_grads(self, gs: GaussianSet, frames: list) -> dict:
        """Zeroed gradient buffers for batch_backward."""
        dev = f"cuda:{self.device}"
        K = (gs.sh_degree + 1) ** 2
        n = gs.n
        g = {"means": torch.zeros((n, 3), device=dev), "log_scales": torch.zeros((n, 3), device=dev),
             "quats": torch.zeros((n, 4), device=dev), "opacity_logits": torch.zeros(n, device=dev),
             "sh": torch.zeros((n, K, 3), device=dev)}
        if frames:
            G = frames[0].q.shape[0]
            g["group_q"] = torch.zeros((len(frames), G, 4), device=dev)
            g["group_t"] = torch.zeros((len(frames), G, 3), device=dev)
        return g

    def batch_backward(self, saved: Saved | None, gs: GaussianSet, frames: list, dL_dimages: list,
                       grads: dict | None = None, accumulate: bool = False, stream=None) -> dict:
        """Gradients of a batched forward, summed over its requests in order; the motion
        gradients are per (frame, group).  accumulate=True adds into `grads`."""
        if grads is None:
            grads = self.batch_grads(gs, frames)
        g = self._grads_struct(grads)
        dls = [d.contiguous() for d in dL_dimages]
        ptrs = (C.c_void_p * len(dls))(*[d.data_ptr() for d in dls])
        fr, nf = self._frames(frames)
        st = lib().gc_render_batch_backward(self.ctx, saved.handle if saved is not None else None,
                                            C.byref(gs.struct), fr, nf, ptrs,
                                            1 if accumulate else 0, C.byref(g), _stream(stream))
        check(st, self.ctx)
        return grads

    def tune_batch(self, gs: GaussianSet, frames: list, requests: list, dL_dimages: list | None = None,
                   grads: dict | None = None, depths=(16, 32, 64, 128), iters: int = 3, outs: list | None = None,
                   stream=None) -> dict:
        """Autotuner over tile shape x batch depth (native, gc_tune_batch).  Sets the best
        tile shape in this renderer's options and returns every measurement."""
        reqs, outs = self._requests(requests, outs)
        fr, nf = self._frames(frames)
        g, ptrs = None, None
        if dL_dimages is not None:
            grads = grads if grads is not None else self.batch_grads(gs, frames)
            g = self._grads_struct(grads)
            ptrs = (C.c_void_p * len(dL_dimages))(*[d.data_ptr() for d in dL_dimages])
        ds = (C.c_int32 * len(depths))(*[int(d) for d in depths])
        entries = (_abi.TuneEntry * (3 * len(depths)))()
        best = _abi.TuneEntry()
        st = lib().gc_tune_batch(self.ctx, C.byref(gs.struct), fr, nf, reqs, len(requests), ptrs,
                                 C.byref(g) if g is not None else None, ds, len(depths), int(iters), entries,
                                 C.byref(best), _stream(stream))
        check(st, self.ctx)
        self.options.tile_w, self.options.tile_h = best.tile_w, best.tile_h

        def row(e):
            return {"tile": (e.tile_w, e.tile_h), "depth": e.depth, "key_capacity": e.key_capacity, "ms": e.ms}
        return {"best": row(best), "entries": [row(e) for e in entries]}

    def _requests(self, requests, outs):
        dev = f"cuda:{self.device}"
        n = len(requests)
        reqs = (_abi.Request * n)()
        if outs is None:
            outs = [torch.empty((3, int(c.height), int(c.width)), dtype=torch.float32, device=dev)
                    for c, _, _ in requests]
        for q, (cam, frame, mask) in enumerate(requests):
            reqs[q].camera = camera_struct(cam)
            reqs[q].frame = int(frame)
            reqs[q].layer_mask = int(mask) & 0xFFFFFFFF
            reqs[q].image = outs[q].data_ptr()
        return reqs, outs

    @staticmethod
    def _frames(frames):
        fr = (_abi.Motion * max(len(frames), 1))()
        for f, m in enumerate(frames):
            fr[f] = m.struct
        return (fr if frames else None), len(frames)

    @staticmethod
    def _grads_struct(grads: dict) -> _abi.Grads:
        g = _abi.Grads()
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "group_q", "group_t"):
            setattr(g, "d_" + k, grads[k].data_ptr() if k in grads else None)
        return g

    def stats(self, saved: Saved | None = None, stream=None) -> dict:
        s = _abi.Stats()
        check(lib().gc_saved_stats(self.ctx, saved.handle if saved else None, C.byref(s),
                                   _stream(stream)), self.ctx)
        return {"n_selected": s.n_selected, "n_visible": s.n_visible, "n_keys": s.n_keys,
                "n_tiles": s.n_tiles, "width": s.width, "height": s.height}

    def tile_lists(self, saved: Saved | None = None, stream=None):
        st = self.stats(saved, stream)
        dev = f"cuda:{self.device}"
        ranges = torch.zeros((st["n_tiles"], 2), dtype=torch.int32, device=dev)
        ids = torch.zeros(max(st["n_keys"], 1), dtype=torch.int64, device=dev)
        check(lib().gc_saved_tile_lists(self.ctx, saved.handle if saved else None, _ptr(ranges),
                                        _ptr(ids), ids.numel(), _stream(stream)), self.ctx)
        return ranges, ids[:st["n_keys"]]

    def pixel_state(self, saved: Saved | None = None, stream=None, with_walked: bool = False):
        """(final T, blended count[, walked count, list position after the last blended])."""
        st = self.stats(saved, stream)
        dev = f"cuda:{self.device}"
        shape = (st["height"], st["width"])
        T = torch.empty(shape, device=dev)
        nb = torch.empty(shape, dtype=torch.int32, device=dev)
        nw = torch.empty(shape, dtype=torch.int32, device=dev) if with_walked else None
        nc = torch.empty(shape, dtype=torch.int32, device=dev) if with_walked else None
        check(lib().gc_saved_pixel_state(self.ctx, saved.handle if saved else None, _ptr(T), _ptr(nb),
                                         _ptr(nw), _ptr(nc), _stream(stream)), self.ctx)
        return (T, nb, nw, nc) if with_walked else (T, nb)

    def profile(self, enable: bool = True, flush_l2: bool = False):
        """Per-stage CUDA-event timing; flush_l2 writes a 256 MB buffer before every stage
        (outside the stage's events)."""
        check(lib().gc_profile_enable(self.ctx, (2 if flush_l2 else 1) if enable else 0), self.ctx)

    def profile_read(self) -> dict:
        """Per-stage summed ms and call counts since the last read, and kernel launches."""
        ms = (C.c_double * len(_abi.STAGES))()
        calls = (C.c_int64 * len(_abi.STAGES))()
        launches = C.c_uint64()
        check(lib().gc_profile_read(self.ctx, ms, calls, C.byref(launches)), self.ctx)
        return {"stage_ms": {n: ms[i] for i, n in enumerate(_abi.STAGES)},
                "stage_calls": {n: calls[i] for i, n in enumerate(_abi.STAGES)},
                "kernel_launches": int(launches.value)}

    def check(self, stream=None):
        check(lib().gc_check(self.ctx, _stream(stream)), self.ctx)


class LevelsGraph:
    """A multi-frame step of the single-pass multi-level render as one CUDA graph
    (gc_levels_graph): per frame the images of levels 1..levels and, with dL_dimages, their
    backward into that frame's gradient set.  frames: one MotionFrame (or None) per frame;
    outs / dL_dimages: n_frames * levels tensors (3, H, W), frame-major; grads: one dict per
    frame (the same dict may repeat).  chains: independent branches of the graph (frame f
    on chain f mod chains, each with its own saved state), so that one frame's sorts run
    beside another frame's blend; results equal those of chains = 1.  The tensors given here
    are the ones every launch reads and writes: update them in place."""

    def __init__(self, renderer: Renderer, gs: GaussianSet, frames: list, cameras: list, levels: int,
                 outs: list | None = None, dL_dimages: list | None = None, grads: list | None = None,
                 chains: int = 1, stream=None):
        nf = len(cameras)
        if len(frames) != nf:
            raise ValueError("one motion frame (or None) per camera")
        self.renderer, self.gs, self.frames, self.levels = renderer, gs, frames, int(levels)
        self._cams = (_abi.Camera * nf)(*[camera_struct(c) for c in cameras])
        if outs is None:
            outs = [torch.empty((3, c.height, c.width), dtype=torch.float32, device=f"cuda:{renderer.device}")
                    for c in cameras for _ in range(levels)]
        if len(outs) != nf * levels:
            raise ValueError("outs needs n_frames * levels images")
        self.outs = outs
        self._imgs = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        motions = None
        if any(f is not None for f in frames):
            if not all(f is not None for f in frames):
                raise ValueError("either every frame has a motion or none has")
            motions = (_abi.Motion * nf)(*[f.struct for f in frames])
        self._motions = motions
        self.dL, self.grads, dls, gstructs = dL_dimages, None, None, None
        if dL_dimages is not None:
            if len(dL_dimages) != nf * levels:
                raise ValueError("dL_dimages needs n_frames * levels tensors")
            dls = (C.c_void_p * len(dL_dimages))(*[d.data_ptr() for d in dL_dimages])
            if grads is None:
                g0 = renderer._single_grads(gs, frames[0])
                grads = [g0] * nf
            if len(grads) != nf:
                raise ValueError("grads needs one dict per frame")
            self.grads = grads
            gstructs = (_abi.Grads * nf)(*[renderer._grads_struct(g) for g in grads])
        self._dls, self._gstructs = dls, gstructs
        h = C.c_void_p()
        st = lib().gc_levels_graph_create(renderer.ctx, C.byref(gs.struct), motions, nf, self._cams, self.levels,
                                          self._imgs, dls, gstructs, int(chains), _stream(stream), C.byref(h))
        check(st, renderer.ctx)
        self.handle = h
        cap, nodes = C.c_int64(), C.c_int64()
        check(lib().gc_levels_graph_info(h, C.byref(cap), C.byref(nodes)), renderer.ctx)
        self.key_capacity, self.kernel_nodes = cap.value, nodes.value

    def launch(self, stream=None):
        check(lib().gc_levels_graph_launch(self.handle, _stream(stream)), self.renderer.ctx)

    def check(self, stream=None):
        check(lib().gc_levels_graph_check(self.handle, _stream(stream)), self.renderer.ctx)

    def close(self):
        if getattr(self, "handle", None):
            lib().gc_levels_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchGraph:
    """A whole step over many requests as one CUDA graph (gc_batch_graph): batches of
    `depth` requests, each a batched forward and, with dL_dimages, a batched backward
    whose gradients are summed over all requests.  The tensors given here are the ones
    every launch reads and writes: update them in place."""

    def __init__(self, renderer: Renderer, gs: GaussianSet, frames: list, requests: list, depth: int,
                 dL_dimages: list | None = None, grads: dict | None = None, outs: list | None = None,
                 stream=None):
        self.renderer = renderer
        self.gs, self.frames = gs, frames
        self.reqs, self.outs = renderer._requests(requests, outs)
        self._fr, nf = renderer._frames(frames)
        self.dL = dL_dimages
        self.grads = None
        g, ptrs = None, None
        if dL_dimages is not None:
            self.grads = grads if grads is not None else renderer.batch_grads(gs, frames)
            self._g = g = renderer._grads_struct(self.grads)
            self._ptrs = ptrs = (C.c_void_p * len(dL_dimages))(*[d.data_ptr() for d in dL_dimages])
        h = C.c_void_p()
        st = lib().gc_batch_graph_create(renderer.ctx, C.byref(gs.struct), self._fr, nf, self.reqs, len(requests),
                                         int(depth), ptrs, C.byref(g) if g is not None else None,
                                         _stream(stream), C.byref(h))
        check(st, renderer.ctx)
        self.handle = h
        cap, nodes, nb = C.c_int64(), C.c_int64(), C.c_int32()
        check(lib().gc_batch_graph_info(h, C.byref(cap), C.byref(nodes), C.byref(nb)), renderer.ctx)
        self.key_capacity, self.kernel_nodes, self.n_batches = cap.value, nodes.value, nb.value

    def launch(self, stream=None):
        check(lib().gc_batch_graph_launch(self.handle, _stream(stream)), self.renderer.ctx)

    def check(self, stream=None):
        check(lib().gc_batch_graph_check(self.handle, _stream(stream)), self.renderer.ctx)

    def close(self):
        if getattr(self, "handle", None):
            lib().gc_batch_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, layer_offsets, sh_degree, layer_mask, camera, means, log_scales, quats,
                opacity_logits, sh, group_id, group_q, group_t):
        gs = GaussianSet(layer_offsets, sh_degree, _abi.GC_PREC_FP32, means=means.contiguous(),
                         log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                         opacity_logits=opacity_logits.contiguous(), sh=sh.contiguous(),
                         group_id=group_id)
        mo = MotionFrame(group_q, group_t) if group_q is not None else None
        saved = Saved(renderer)
        img = renderer.forward(gs, mo, layer_mask, camera, saved)
        ctx.renderer, ctx.gs, ctx.mo, ctx.saved = renderer, gs, mo, saved
        return img

    @staticmethod
    def backward(ctx, dimg):
        g = ctx.renderer.backward(ctx.saved, ctx.gs, ctx.mo, dimg.contiguous())
        return (None, None, None, None, None, g["means"], g["log_scales"], g["quats"],
                g["opacity_logits"], g["sh"], None, g.get("group_q"), g.get("group_t"))


def render(renderer: Renderer, layer_offsets, sh_degree: int, layer_mask: int, camera, means,
           log_scales, quats, opacity_logits, sh, group_id=None, group_q=None, group_t=None):
    """Differentiable render of one frame (image 3 x H x W)."""
    return _RenderFn.apply(renderer, layer_offsets, sh_degree, layer_mask, camera, means,
                           log_scales, quats, opacity_logits, sh, group_id, group_q, group_t)
