"""FP64 CPU oracle of the hierarchical 4D Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA product path never imports it.  It shares
no code with the CUDA library: the C source ``gc_oracle.c`` next to this file
is compiled with gcc (``-ffp-contract=off``, OpenMP) into ``libgc_oracle.so``.

Functions (each follows the paper, 4DGCPro):

* :func:`bin_f32`      the FP32 binning mirror: visibility, depth, pixel and
                       tile footprint of each selected Gaussian, taken in the
                       op order of the written binning specification.
* :func:`render`       FP64 per-pixel brute-force compositing (Eq. 2, Eq. 4)
                       over the selected layers, after per-group rigid motion
                       (Sec. 3.2) and EWA projection of Sigma = R s s^T R^T
                       (Sec. 3.1).  Full frame or a list of sampled pixels.
* :func:`grad`         FP64 reverse mode of a linear functional of the image.
* :func:`tile_lists`   the per-tile (depth, index)-ordered Gaussian lists the
                       binning mirror implies.

Parity: the FP32 mirror's integer decisions are the same decisions an FP32
renderer takes; the FP64 render consumes them.  Pins live in
``tests/test_oracle_*.py``.  The reading of the paper's silent points (near
plane 0.2, dilation 0.3, frustum clamp 1.3, SH offset +0.5) is "parity
unpinned": the paper prints no code, so these are readings, each an option.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gc_oracle.c")
_LIB = os.path.join(_HERE, "libgc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``libgc_oracle.so`` (in-tree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("campos", C.c_float * 3)]


class Options(C.Structure):
    _fields_ = [("near_plane", C.c_float), ("dilation", C.c_float), ("frustum_clamp", C.c_float),
                ("bg", C.c_float * 3), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("membership", C.c_int32), ("alpha_cull", C.c_int32)]


class SceneS(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p),
                ("log_scales", C.c_void_p), ("quats", C.c_void_p), ("opacity_logits", C.c_void_p),
                ("sh", C.c_void_p), ("group_id", C.c_void_p)]


class MotionS(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("q", C.c_void_p), ("t", C.c_void_p),
                ("res_ls", C.c_void_p), ("res_logit", C.c_void_p), ("res_sh", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            L.gco_bin_f32.argtypes = [P] * 5 + [C.c_int64] + [P] * 8
            L.gco_bin_rows.argtypes = [P, P, C.c_int64] + [P] * 9
            L.gco_render_f64.argtypes = [P] * 5 + [C.c_int64] + [P] * 5 + [C.c_int64] + [P] * 5
            L.gco_render_f64.restype = C.c_int
            L.gco_grad_f64.argtypes = [P] * 5 + [C.c_int64] + [P] * 5 + [P] * 8
            L.gco_grad_f64.restype = C.c_int
            L.gco_quat_to_rot.argtypes = [P, P]
            L.gco_quat_mul.argtypes = [P, P, P]
            L.gco_sh_eval.argtypes = [C.c_int, P, C.c_int64, P, P]
            L.gco_geom_f64.argtypes = [P] * 4 + [C.c_int64, P]
            L.gco_num_threads.restype = C.c_int
            L.gco_decode_bf16.argtypes = [P, C.c_int64, P]
            L.gco_decode_e4m3.argtypes = [P, C.c_int64, P]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Pack:
    """Keeps contiguous copies alive while the C call runs."""

    def __init__(self):
        self.keep = []

    def f32(self, a):
        a = np.ascontiguousarray(a, np.float32)
        self.keep.append(a)
        return a

    def i32(self, a):
        a = np.ascontiguousarray(a, np.int32)
        self.keep.append(a)
        return a


def default_options(tile=(16, 16), bg=(0.0, 0.0, 0.0), near=0.2, dilation=0.3, clamp=1.3,
                    membership=0, alpha_cull=1) -> dict:
    return {"tile": tuple(tile), "bg": tuple(bg), "near": near, "dilation": dilation,
            "clamp": clamp, "membership": membership, "alpha_cull": alpha_cull}


def _options(o: dict) -> Options:
    op = Options()
    op.near_plane = o.get("near", 0.2)
    op.dilation = o.get("dilation", 0.3)
    op.frustum_clamp = o.get("clamp", 1.3)
    bg = o.get("bg", (0.0, 0.0, 0.0))
    for k in range(3):
        op.bg[k] = bg[k]
    op.tile_w, op.tile_h = o.get("tile", (16, 16))
    op.membership = o.get("membership", 0)
    op.alpha_cull = o.get("alpha_cull", 1)
    return op


def _camera(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    R = np.asarray(cam.R, np.float32).reshape(-1)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(np.float32(cam.t[k]))
        c.campos[k] = float(np.float32(cam.campos[k]))
    return c


def _scene(pk: _Pack, scene) -> SceneS:
    s = SceneS()
    s.n = scene.means.shape[0]
    s.sh_degree = scene.sh_degree
    s.means = _ptr(pk.f32(scene.means))
    s.log_scales = _ptr(pk.f32(scene.log_scales))
    s.quats = _ptr(pk.f32(scene.quats))
    s.opacity_logits = _ptr(pk.f32(scene.opacity_logits))
    s.sh = _ptr(pk.f32(scene.sh))
    s.group_id = _ptr(pk.i32(scene.group_id)) if scene.group_id is not None else None
    return s


def _motion(pk: _Pack, motion, frame: int, residual=None):
    """Frame `frame` of the group motion (None: keyframe, identity) and, optionally, that
    frame's residual deformation (an object with ls (n,3), logit (n,) and sh (n,K,3)
    arrays, any of them None; Sec. 3.2, Eq. 7)."""
    m = MotionS()
    if motion is None:
        m.n_groups = 1
        m.q = None
        m.t = None
    else:
        m.n_groups = motion.q.shape[1]
        m.q = _ptr(pk.f32(motion.q[frame]))
        m.t = _ptr(pk.f32(motion.t[frame]))
    if residual is not None:
        m.res_ls = _ptr(pk.f32(residual.ls)) if residual.ls is not None else None
        m.res_logit = _ptr(pk.f32(residual.logit)) if residual.logit is not None else None
        m.res_sh = _ptr(pk.f32(residual.sh)) if residual.sh is not None else None
    return m


def selection(scene, layer_mask: int) -> np.ndarray:
    parts = [np.arange(scene.layer_offsets[l], scene.layer_offsets[l + 1], dtype=np.int64)
             for l in range(len(scene.layer_offsets) - 1) if (layer_mask >> l) & 1]
    return np.concatenate(parts) if parts else np.zeros(0, np.int64)


def bin_f32(scene, motion, frame, cam, opts: dict, layer_mask: int = 1, residual=None) -> dict:
    """FP32 binning mirror over the selected Gaussians (arrays by selected position).
    ``residual``: the frame's residual deformation (see ``_motion``), or None.

    ``row_off`` / ``row_a`` / ``row_b``: for visible position j, its tile rows
    trect[j, 2] .. trect[j, 3] are entries row_off[j] .. row_off[j+1]-1, each the
    inclusive tile-column interval [a, b] of that row (a > b: empty)."""
    L = lib()
    pk = _Pack()
    sel = np.ascontiguousarray(selection(scene, layer_mask))
    n = sel.shape[0]
    out = {"sel": sel,
           "visible": np.zeros(n, np.int32), "depth": np.zeros(n, np.float32),
           "rect": np.zeros((n, 4), np.int32), "trect": np.zeros((n, 4), np.int32),
           "radius": np.zeros(n, np.int32), "uv": np.zeros((n, 2), np.float32),
           "conic": np.zeros((n, 3), np.float32), "tc": np.zeros(n, np.float32)}
    sc, mo, ca, op = _scene(pk, scene), _motion(pk, motion, frame, residual), _camera(cam), _options(opts)
    L.gco_bin_f32(C.byref(sc), C.byref(mo), C.byref(ca), C.byref(op), _ptr(sel), n,
                  _ptr(out["visible"]), _ptr(out["depth"]), _ptr(out["rect"]), _ptr(out["trect"]),
                  _ptr(out["radius"]), _ptr(out["uv"]), _ptr(out["conic"]), _ptr(out["tc"]))
    rows = np.where(out["visible"] != 0, out["trect"][:, 3] - out["trect"][:, 2] + 1, 0).astype(np.int64)
    row_off = np.zeros(n + 1, np.int64)
    np.cumsum(rows, out=row_off[1:])
    out["row_off"] = row_off
    out["row_a"] = np.ones(int(row_off[-1]), np.int32)
    out["row_b"] = np.zeros(int(row_off[-1]), np.int32)
    L.gco_bin_rows(C.byref(ca), C.byref(op), n, _ptr(out["visible"]), _ptr(out["rect"]), _ptr(out["trect"]),
                   _ptr(out["uv"]), _ptr(out["conic"]), _ptr(out["tc"]), _ptr(row_off), _ptr(out["row_a"]),
                   _ptr(out["row_b"]))
    return out


def render(scene, motion, frame, cam, opts: dict, layer_mask: int = 1, pixels=None,
           bins: dict | None = None, residual=None) -> dict:
    """FP64 render.  ``pixels``: optional (n, 2) int (x, y) sample list.

    Returns ``image`` (3, H, W) or (n, 3) for samples, ``T`` (final
    transmittance), ``n_blended``, ``ambiguous`` (a decision within the FP32
    margin), ``signature`` and the binning mirror output ``bins``.
    ``bins`` may be given to freeze the discrete decisions.  ``residual``: the frame's
    residual deformation (Sec. 3.2, Eq. 7), or None.
    """
    L = lib()
    pk = _Pack()
    if bins is None:
        bins = bin_f32(scene, motion, frame, cam, opts, layer_mask, residual)
    sel = bins["sel"]
    sc, mo, ca, op = _scene(pk, scene), _motion(pk, motion, frame, residual), _camera(cam), _options(opts)
    W, H = int(cam.width), int(cam.height)
    if pixels is None:
        npx = 0
        pix = None
        rgb = np.zeros((3, H, W), np.float64)
        T = np.zeros((H, W), np.float64)
        nb = np.zeros((H, W), np.int32)
        amb = np.zeros((H, W), np.int32)
        sig = np.zeros((H, W), np.float64)
    else:
        pix = np.ascontiguousarray(pixels, np.int32)
        npx = pix.shape[0]
        rgb = np.zeros((npx, 3), np.float64)
        T = np.zeros(npx, np.float64)
        nb = np.zeros(npx, np.int32)
        amb = np.zeros(npx, np.int32)
        sig = np.zeros(npx, np.float64)
        if npx == 0:
            return {"image": rgb, "T": T, "n_blended": nb, "ambiguous": amb, "signature": sig,
                    "bins": bins}
    vis = np.ascontiguousarray(bins["visible"], np.int32)
    dep = np.ascontiguousarray(bins["depth"], np.float32)
    rect = np.ascontiguousarray(bins["rect"], np.int32)
    trect = np.ascontiguousarray(bins["trect"], np.int32)
    rc = L.gco_render_f64(C.byref(sc), C.byref(mo), C.byref(ca), C.byref(op), _ptr(sel),
                          sel.shape[0], _ptr(vis), _ptr(dep), _ptr(rect), _ptr(trect),
                          _ptr(pix), npx, _ptr(rgb), _ptr(T), _ptr(nb), _ptr(amb), _ptr(sig))
    if rc != 0:
        raise MemoryError("oracle render failed")
    return {"image": rgb, "T": T, "n_blended": nb, "ambiguous": amb.astype(bool),
            "signature": sig, "bins": bins}


def grad(scene, motion, frame, cam, opts: dict, dL_dimage, layer_mask: int = 1,
         bins: dict | None = None, residual=None) -> dict:
    """FP64 gradient of L = sum(dL_dimage * image) w.r.t. every input.

    Gradients are returned for the full scene arrays (zero outside the
    selection and for culled Gaussians) plus the group motion table of the
    frame, and the per-Gaussian 2D gradient ``d2d`` (du, dv, dconic a/b/c,
    dopacity, drgb) by selected position.  With a ``residual`` (Sec. 3.2, Eq. 7) the
    log-scale, logit and SH gradients are those of the deformed attributes, which are
    also the gradients of the residuals (they enter additively).
    """
    L = lib()
    pk = _Pack()
    if bins is None:
        bins = bin_f32(scene, motion, frame, cam, opts, layer_mask, residual)
    sel = bins["sel"]
    n_sel = sel.shape[0]
    sc, mo, ca, op = _scene(pk, scene), _motion(pk, motion, frame, residual), _camera(cam), _options(opts)
    K = (scene.sh_degree + 1) ** 2
    G = motion.q.shape[1] if motion is not None else 1
    g = np.ascontiguousarray(dL_dimage, np.float64).reshape(3, cam.height, cam.width)
    dm = np.zeros((n_sel, 3)); dls = np.zeros((n_sel, 3)); dq = np.zeros((n_sel, 4))
    dlo = np.zeros(n_sel); dsh = np.zeros((n_sel, K, 3)); d2d = np.zeros((n_sel, 9))
    dgq = np.zeros((G, 4)); dgt = np.zeros((G, 3))
    vis = np.ascontiguousarray(bins["visible"], np.int32)
    dep = np.ascontiguousarray(bins["depth"], np.float32)
    rect = np.ascontiguousarray(bins["rect"], np.int32)
    trect = np.ascontiguousarray(bins["trect"], np.int32)
    rc = L.gco_grad_f64(C.byref(sc), C.byref(mo), C.byref(ca), C.byref(op), _ptr(sel), n_sel,
                        _ptr(vis), _ptr(dep), _ptr(rect), _ptr(trect), _ptr(g),
                        _ptr(dm), _ptr(dls), _ptr(dq), _ptr(dlo), _ptr(dsh), _ptr(dgq), _ptr(dgt),
                        _ptr(d2d))
    if rc != 0:
        raise MemoryError("oracle grad failed")
    N = scene.means.shape[0]
    full = {"means": np.zeros((N, 3)), "log_scales": np.zeros((N, 3)), "quats": np.zeros((N, 4)),
            "opacity_logits": np.zeros(N), "sh": np.zeros((N, K, 3))}
    full["means"][sel] = dm
    full["log_scales"][sel] = dls
    full["quats"][sel] = dq
    full["opacity_logits"][sel] = dlo
    full["sh"][sel] = dsh
    full["group_q"] = dgq
    full["group_t"] = dgt
    full["d2d"] = d2d
    full["bins"] = bins
    return full


def tile_lists(bins: dict, cam, tile=(16, 16)) -> dict:
    """Per-tile lists of global Gaussian ids ordered by (depth, index).

    Every visible Gaussian contributes one entry per tile of each row interval of
    its tile rectangle.  Returns ``gauss_of_entry`` / ``tile_of_entry`` sorted by
    (tile, depth, index) with numpy's lexsort, and ``ranges`` (n_tiles, 2).
    """
    tw, th = tile
    ntx = (cam.width + tw - 1) // tw
    nty = (cam.height + th - 1) // th
    off = bins["row_off"]
    n_rows = int(off[-1])
    row_owner = np.repeat(np.arange(len(off) - 1), np.diff(off))  # selected position of each row
    row_ty = bins["trect"][row_owner, 2].astype(np.int64) + (np.arange(n_rows) - off[row_owner])
    a = bins["row_a"].astype(np.int64)
    cnt = np.maximum(bins["row_b"].astype(np.int64) - a + 1, 0)
    owner = np.repeat(row_owner, cnt)
    start = np.concatenate([[0], np.cumsum(cnt)[:-1]]) if len(cnt) else np.zeros(0, np.int64)
    k = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(start, cnt)
    tx = np.repeat(a, cnt) + k
    ty = np.repeat(row_ty, cnt)
    t = ty * ntx + tx
    g = bins["sel"][owner]
    d = bins["depth"][owner]
    order = np.lexsort((g, d, t))
    t, g = t[order], g[order]
    n_tiles = ntx * nty
    starts = np.searchsorted(t, np.arange(n_tiles), side="left")
    ends = np.searchsorted(t, np.arange(n_tiles), side="right")
    return {"tile_of_entry": t, "gauss_of_entry": g, "ranges": np.stack([starts, ends], 1),
            "n_tiles": n_tiles}


def tile_list(bins: dict, cam, tile_id: int, tile=(16, 16)) -> np.ndarray:
    """The (depth, index)-ordered global ids of one tile's list (cheap for big scenes)."""
    tw, th = tile
    ntx = (cam.width + tw - 1) // tw
    tx, ty = tile_id % ntx, tile_id // ntx
    tr = bins["trect"]
    m = (bins["visible"] == 1) & (tr[:, 2] <= ty) & (tr[:, 3] >= ty)
    j = np.nonzero(m)[0]
    row = bins["row_off"][j] + (ty - tr[j, 2])
    j = j[(bins["row_a"][row] <= tx) & (bins["row_b"][row] >= tx)]
    order = np.lexsort((bins["sel"][j], bins["depth"][j]))
    return bins["sel"][j][order]


def quat_to_rot(q) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9)
    lib().gco_quat_to_rot(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def quat_mul(a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    o = np.zeros(4)
    lib().gco_quat_mul(_ptr(a), _ptr(b), _ptr(o))
    return o


def sh_eval(deg: int, dirs, with_grad: bool = False):
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    Y = np.zeros((dirs.shape[0], K))
    dY = np.zeros((dirs.shape[0], K, 3)) if with_grad else None
    lib().gco_sh_eval(deg, _ptr(dirs), dirs.shape[0], _ptr(Y), _ptr(dY))
    return (Y, dY) if with_grad else Y


def geom(scene, motion, frame, cam, opts: dict, i: int, residual=None) -> dict:
    pk = _Pack()
    sc, mo, ca, op = _scene(pk, scene), _motion(pk, motion, frame, residual), _camera(cam), _options(opts)
    out = np.zeros(28)
    lib().gco_geom_f64(C.byref(sc), C.byref(mo), C.byref(ca), C.byref(op), int(i), _ptr(out))
    return {"u": out[0], "v": out[1], "sigma2": np.array([[out[2], out[3]], [out[3], out[4]]]),
            "conic": out[5:8].copy(), "J": out[8:12].copy(), "opacity": out[12],
            "rgb": out[13:16].copy(), "cam_point": out[16:19].copy(),
            "sigma3": out[19:28].reshape(3, 3).copy()}


def decode_bf16(a) -> np.ndarray:
    a = np.ascontiguousarray(a, np.uint16)
    out = np.zeros(a.shape, np.float32)
    lib().gco_decode_bf16(_ptr(a), a.size, _ptr(out))
    return out


def decode_e4m3(a) -> np.ndarray:
    a = np.ascontiguousarray(a, np.uint8)
    out = np.zeros(a.shape, np.float32)
    lib().gco_decode_e4m3(_ptr(a), a.size, _ptr(out))
    return out


def dequantize(q: dict, scene_template):
    """Scene whose attributes are the FP32 dequantised values of ``q``.

    value = fl32(decode(stored) * scale), one FP32 multiply per element.
    """
    import copy
    s = copy.copy(scene_template)

    def deq(raw, scale, dec):
        v = dec(raw).reshape(raw.shape[0], -1)
        return (v * np.asarray(scale, np.float32)[None, :]).astype(np.float32).reshape(raw.shape)

    s.means = deq(q["means"], q["means_scale"], decode_bf16)
    s.log_scales = deq(q["log_scales"], q["log_scales_scale"], decode_bf16)
    s.quats = deq(q["quats"], q["quats_scale"], decode_bf16)
    s.opacity_logits = deq(q["opacity_logits"][:, None], q["opacity_scale"], decode_bf16).reshape(-1)
    s.sh = deq(q["sh"], q["sh_scale"], decode_e4m3)
    return s


def dequantize_planes(planes: dict, scene_template):
    """Scene whose attributes are the FP32 values of the paper's decoded planes (Sec. 3.4; the
    layout of ``synth.scenes.quantize_planes``): Gaussian j of layer l is read at row
    j // plane_width, column j % plane_width of each of its layer's channel planes, and
    value = fl32(fl32(float(code) * step) + lo) with the channel's (lo, step) - the min / max
    affine map, one FP32 multiply and one FP32 add.  Group ids come from the template."""
    import copy
    s = copy.copy(scene_template)
    W = int(planes["plane_width"])
    dq = np.asarray(planes["dequant"], np.float32)
    n_ch = dq.shape[1]
    out = np.zeros((scene_template.n, n_ch), np.float32)
    for l in range(len(scene_template.layer_offsets) - 1):
        a, b = int(scene_template.layer_offsets[l]), int(scene_template.layer_offsets[l + 1])
        row, col = np.divmod(np.arange(b - a), W)   # Gaussian j of the layer
        for ch in range(n_ch):
            code = planes["pos"][l][ch, row, col] if ch < 3 else planes["u8"][l][ch - 3, row, col]
            lo, step = dq[l, ch]
            out[a:b, ch] = (code.astype(np.float32) * step).astype(np.float32) + lo
    K3 = n_ch - 11
    s.means = out[:, 0:3].copy()
    s.quats = out[:, 3:7].copy()
    s.log_scales = out[:, 7:10].copy()
    s.opacity_logits = out[:, 10].copy()
    s.sh = out[:, 11:].reshape(-1, K3 // 3, 3).copy()
    return s


def num_threads() -> int:
    return int(lib().gco_num_threads())
