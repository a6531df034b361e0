"""Seeded synthetic workloads for the hierarchical 4D Gaussian rasterizer.

This module only draws random inputs and arranges them into arrays: the keyframe
Gaussians, the per-group motion tables, the camera poses and the render
requests.  It holds none of the rasterizer's arithmetic (no projection, no
compositing, no spherical harmonics); both the FP64 oracle and the CUDA path
consume what it produces, and neither is imported here.

Workloads stand in for the paper's captured datasets, which are not available:

* ``tiny``      2,000 Gaussians, one layer, no motion, SH degree 0, 128x128.
* ``hier1080``  300k Gaussians in 6 layers of 50k, SH degree 3, 64 motion
                groups over a 30-frame group of pictures, 1920x1080, every
                frame at every level L1..L6.
* ``diff``      200k Gaussians, SH degree 3, 32 groups, 1352x1014, an L1 loss
                against a target rendered from a perturbed copy.
* ``batch``     500k Gaussians, SH degree 3, 128 groups, 16 views x 8 frames,
                each request at its own level and resolution.
* ``prec4k``    1M Gaussians in 6 layers, SH degree 3, 256 groups, 3840x2160.

Layering follows the paper's significance ordering (Sec. 3.1, Eq. 3): the
generator sorts Gaussians by Psi = opacity + lambda_Psi * (4/3) pi a b c in
descending order and cuts the sorted array into L contiguous layers, so that
level l is the prefix made of layers 1..l (Eq. 4).  Motion follows Sec. 3.2
(rigid transformation): each group carries a cumulative keyframe-to-frame
translation and rotation, composed here with ``scipy.spatial.transform``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

LAMBDA_PSI = 1.0e5  # significance weight, Sec. A (implementation details)


@dataclass
class Scene:
    """Keyframe Gaussians, all float32 row-major, index order = layer order."""

    means: np.ndarray           # (N, 3)
    log_scales: np.ndarray      # (N, 3)
    quats: np.ndarray           # (N, 4) Hamilton (w, x, y, z), not necessarily unit
    opacity_logits: np.ndarray  # (N,)
    sh: np.ndarray              # (N, (d+1)^2, 3)
    group_id: np.ndarray        # (N,) int32 in [0, n_groups)
    layer_offsets: np.ndarray   # (L+1,) int64, layer l = [off[l], off[l+1])
    sh_degree: int
    n_groups: int = 1

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_layers(self) -> int:
        return int(self.layer_offsets.shape[0] - 1)

    def subset(self, idx) -> "Scene":
        """Gaussians ``idx`` (sorted index array) as a one-layer scene."""
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.group_id[idx].copy(),
                     np.array([0, len(idx)], np.int64), self.sh_degree,
                     self.n_groups)


@dataclass
class Motion:
    """Cumulative per-group rigid motion, keyframe (frame 0) = identity."""

    q: np.ndarray  # (F, G, 4) float32 unit Hamilton quaternions (w, x, y, z)
    t: np.ndarray  # (F, G, 3) float32 translations

    @property
    def n_frames(self) -> int:
        return int(self.q.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.q.shape[1])

    def frame(self, f: int) -> "Motion":
        return Motion(self.q[f:f + 1].copy(), self.t[f:f + 1].copy())


@dataclass
class Residual:
    """Residual deformation of one frame (Sec. 3.2, Eq. 7), cumulative from the keyframe:
    offsets added to the log-scales, opacity logits and SH coefficients before activation.
    Any field may be None (no residual for that attribute)."""

    ls: np.ndarray | None      # (n, 3) float32
    logit: np.ndarray | None   # (n,) float32
    sh: np.ndarray | None      # (n, K, 3) float32


def random_residual(seed: int, n: int, sh_degree: int, frame: int, ls_sigma=0.01, logit_sigma=0.05,
                    sh_sigma=0.01) -> Residual:
    """Residuals of frame `frame` of a random walk with independent N(0, sigma^2) steps per
    frame (the paper observes Gaussian-distributed residual attributes, Sec. 3.3): the
    cumulative offset is N(0, frame sigma^2) per attribute; the keyframe (frame 0) has none."""
    rng = np.random.default_rng([seed, frame])
    k = _sh_count(sh_degree)
    sd = np.sqrt(max(frame, 0))
    return Residual(ls=(rng.normal(0.0, ls_sigma * sd, (n, 3))).astype(np.float32),
                    logit=(rng.normal(0.0, logit_sigma * sd, n)).astype(np.float32),
                    sh=(rng.normal(0.0, sh_sigma * sd, (n, k, 3))).astype(np.float32))


def apply_residual(scene: "Scene", res: Residual) -> "Scene":
    """The scene with the residuals added in FP32 (one rounding per attribute)."""
    import dataclasses
    out = dataclasses.replace(scene)
    if res.ls is not None:
        out.log_scales = (scene.log_scales + res.ls).astype(np.float32)
    if res.logit is not None:
        out.opacity_logits = (scene.opacity_logits + res.logit).astype(np.float32)
    if res.sh is not None:
        out.sh = (scene.sh + res.sh).astype(np.float32)
    return out


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    A world point X maps to camera coordinates R @ X + t; pixel (i, j) covers
    [i, i+1) x [j, j+1) and has its centre at (i + 0.5, j + 0.5).
    """

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray       # (3, 3) float32, world -> camera
    t: np.ndarray       # (3,) float32
    campos: np.ndarray  # (3,) float32, camera centre in world coordinates


@dataclass
class Request:
    """One render of a batch: a camera, a motion frame and a layer mask."""

    camera: Camera
    frame: int
    layer_mask: int


@dataclass
class Workload:
    name: str
    scene: Scene
    motion: Motion | None
    cameras: list = field(default_factory=list)
    requests: list = field(default_factory=list)
    extra: dict = field(default_factory=dict)


def level_mask(level: int) -> int:
    """Layer mask of quality level ``level`` (1-based): layers 1..level."""
    return (1 << level) - 1


def look_at_camera(eye, target, width, height, vfov_deg=60.0) -> Camera:
    """Camera at ``eye`` looking at ``target`` with world up (0, 1, 0).

    Rows of R are the camera's x (right), y (down) and z (forward) axes in
    world coordinates; the vertical field of view fixes fy, and fx = fy.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(np.array([0.0, 1.0, 0.0]), fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float64)
    t = -R @ eye
    fy = (height / 2.0) / math.tan(math.radians(vfov_deg) / 2.0)
    return Camera(int(width), int(height), float(np.float32(fy)), float(np.float32(fy)),
                  float(width) / 2.0, float(height) / 2.0,
                  R.astype(np.float32), t.astype(np.float32), eye.astype(np.float32))


def orbit_camera(theta, radius, width, height) -> Camera:
    """Camera on a circle of ``radius`` in the y = 0 plane looking at the origin.

    theta = 0 puts the eye at (0, 0, -radius), so that R is the identity.
    """
    eye = (radius * math.sin(theta), 0.0, -radius * math.cos(theta))
    return look_at_camera(eye, (0.0, 0.0, 0.0), width, height)


def _sh_count(deg: int) -> int:
    return (deg + 1) * (deg + 1)


def random_gaussians(rng: np.random.Generator, n: int, sh_degree: int,
                     rgb_dc: bool = False):
    """Draw the keyframe attributes in a fixed order (the recipe's order).

    means ~ U[-1,1]^3, log-scales ~ N(-3, 0.5), quaternions = normalised
    N(0, I4), opacity logits ~ N(0, 1).  Colour: with ``rgb_dc`` (SH degree 0)
    the colour is drawn U[0,1] and stored as the DC coefficient that decodes
    to it (DC = (rgb - 0.5) / Y00, Y00 = 1 / (2 sqrt(pi))); otherwise the DC
    coefficient is U[0,1] and the higher coefficients are N(0, 0.1).
    """
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32)
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = q.astype(np.float32)
    logits = rng.normal(0.0, 1.0, n).astype(np.float32)
    k = _sh_count(sh_degree)
    sh = np.zeros((n, k, 3), np.float32)
    if rgb_dc:
        rgb = rng.uniform(0.0, 1.0, (n, 3))
        y00 = 0.5 / math.sqrt(math.pi)
        sh[:, 0, :] = ((rgb - 0.5) / y00).astype(np.float32)
    else:
        sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
        if k > 1:
            sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, k - 1, 3)).astype(np.float32)
    return means, log_scales, quats, logits, sh


def significance_order(log_scales, logits) -> np.ndarray:
    """Indices sorting Gaussians by the significance Psi, descending (Eq. 3)."""
    opacity = 1.0 / (1.0 + np.exp(-logits.astype(np.float64)))
    volume = (4.0 / 3.0) * math.pi * np.exp(log_scales.astype(np.float64).sum(axis=1))
    psi = opacity + LAMBDA_PSI * volume
    return np.argsort(-psi, kind="stable")


def layer_offsets_even(n: int, n_layers: int) -> np.ndarray:
    return np.array([(n * k) // n_layers for k in range(n_layers + 1)], np.int64)


def voronoi_groups(rng, means, n_groups) -> np.ndarray:
    """Group id = index of the nearest of ``n_groups`` seeds ~ U[-1,1]^3."""
    seeds = rng.uniform(-1.0, 1.0, (n_groups, 3))
    gid = np.empty(means.shape[0], np.int32)
    m = means.astype(np.float64)
    step = 65536
    for s in range(0, m.shape[0], step):
        d2 = ((m[s:s + step, None, :] - seeds[None, :, :]) ** 2).sum(-1)
        gid[s:s + step] = np.argmin(d2, axis=1)
    return gid


def random_motion(rng, n_groups, n_frames, trans_sigma=0.02, angle_sigma_deg=2.0) -> Motion:
    """Cumulative per-group rigid motion over ``n_frames`` (frame 0 = identity).

    Each frame after the keyframe draws, per group, a translation increment
    ~ N(0, trans_sigma^2 I3) and a rotation increment by an angle
    ~ N(0, angle_sigma_deg) about a uniformly random axis; the table stores
    t_{g,f} = sum of increments and R_{g,f} = dR_f ... dR_1 (the paper's
    mu_t = mu_{t-1} + dmu_t and R_t = dR_t R_{t-1}, Sec. 3.2).
    """
    q = np.zeros((n_frames, n_groups, 4), np.float64)
    t = np.zeros((n_frames, n_groups, 3), np.float64)
    q[0, :, 0] = 1.0
    cur = Rotation.identity(n_groups)
    cur_t = np.zeros((n_groups, 3))
    for f in range(1, n_frames):
        dt = rng.normal(0.0, trans_sigma, (n_groups, 3))
        axis = rng.normal(0.0, 1.0, (n_groups, 3))
        axis /= np.linalg.norm(axis, axis=1, keepdims=True)
        ang = np.radians(rng.normal(0.0, angle_sigma_deg, n_groups))
        dR = Rotation.from_rotvec(axis * ang[:, None])
        cur = dR * cur
        cur_t = cur_t + dt
        q[f] = cur.as_quat(scalar_first=True)
        t[f] = cur_t
    # canonical sign (w >= 0); q and -q are the same rotation
    sgn = np.where(q[..., :1] < 0, -1.0, 1.0)
    q *= sgn
    return Motion(q.astype(np.float32), t.astype(np.float32))


def identity_motion(n_groups=1, n_frames=1) -> Motion:
    q = np.zeros((n_frames, n_groups, 4), np.float32)
    q[..., 0] = 1.0
    return Motion(q, np.zeros((n_frames, n_groups, 3), np.float32))


def make_hier_scene(rng, n, n_layers, sh_degree, n_groups) -> Scene:
    means, ls, quats, logits, sh = random_gaussians(rng, n, sh_degree)
    order = significance_order(ls, logits)
    means, ls, quats, logits, sh = (a[order] for a in (means, ls, quats, logits, sh))
    gid = voronoi_groups(rng, means, n_groups) if n_groups > 1 else np.zeros(n, np.int32)
    return Scene(np.ascontiguousarray(means), np.ascontiguousarray(ls),
                 np.ascontiguousarray(quats), np.ascontiguousarray(logits),
                 np.ascontiguousarray(sh), gid, layer_offsets_even(n, n_layers),
                 sh_degree, n_groups)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

def tiny(seed: int = 0, n: int = 2000, size: int = 128) -> Workload:
    """2,000 Gaussians, one layer, one frame, no motion, SH degree 0, 128x128."""
    rng = np.random.default_rng(seed)
    means, ls, quats, logits, sh = random_gaussians(rng, n, 0, rgb_dc=True)
    scene = Scene(means, ls, quats, logits, sh, np.zeros(n, np.int32),
                  np.array([0, n], np.int64), 0, 1)
    cam = look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), size, size)
    return Workload("tiny", scene, None, [cam],
                    [Request(cam, 0, 1)], {"tile": (16, 16), "bg": (0.0, 0.0, 0.0)})


def hier1080(seed: int = 2, n: int = 300_000, n_frames: int = 30, width: int = 1920,
             height: int = 1080) -> Workload:
    """300k Gaussians in 6 nested layers, 64 groups, 30 frames, 1080p, L1..L6."""
    rng = np.random.default_rng(seed)
    scene = make_hier_scene(rng, n, 6, 3, 64)
    motion = random_motion(rng, 64, n_frames)
    cams = [orbit_camera(2.0 * math.pi * f / n_frames, 4.0, width, height)
            for f in range(n_frames)]
    reqs = [Request(cams[f], f, level_mask(lv)) for f in range(n_frames) for lv in range(1, 7)]
    return Workload("hier1080", scene, motion, cams, reqs, {"tile": (16, 16)})


def diff(seed: int = 3, n: int = 200_000, width: int = 1352, height: int = 1014) -> Workload:
    """200k Gaussians, 32 groups, 1352x1014; target from means + N(0, 0.01^2)."""
    rng = np.random.default_rng(seed)
    scene = make_hier_scene(rng, n, 6, 3, 32)
    motion = random_motion(rng, 32, 2)
    cam = orbit_camera(0.0, 4.0, width, height)
    target_means = (scene.means.astype(np.float64)
                    + rng.normal(0.0, 0.01, scene.means.shape)).astype(np.float32)
    return Workload("diff", scene, motion, [cam], [Request(cam, 1, level_mask(6))],
                    {"target_means": target_means})


def diff_subscene(seed: int = 3, n_sub: int = 500, size: int = 64, n: int = 200_000) -> Workload:
    """The first ``n_sub`` Gaussians (by significance) of ``diff`` at size x size."""
    w = diff(seed, n)
    sub = w.scene.subset(np.arange(n_sub))
    cam = orbit_camera(0.0, 4.0, size, size)
    return Workload("diff_sub", sub, w.motion, [cam], [Request(cam, 1, 1)],
                    {"target_means": w.extra["target_means"][:n_sub].copy()})


RESOLUTIONS = [(960, 540), (1280, 720), (1920, 1080)]


def batch(seed: int = 4, n: int = 500_000, n_views: int = 16, n_frames: int = 8) -> Workload:
    """16 views x 8 frames, each at its own level (U{1..6}) and resolution."""
    rng = np.random.default_rng(seed)
    scene = make_hier_scene(rng, n, 6, 3, 128)
    motion = random_motion(rng, 128, n_frames)
    reqs = []
    cams = []
    for v in range(n_views):
        for f in range(n_frames):
            lv = int(rng.integers(1, 7))
            w_, h_ = RESOLUTIONS[int(rng.integers(0, 3))]
            cam = orbit_camera(2.0 * math.pi * v / n_views, 4.0, w_, h_)
            cams.append(cam)
            reqs.append(Request(cam, f, level_mask(lv)))
    return Workload("batch", scene, motion, cams, reqs, {})


def prec4k(seed: int = 5, n: int = 1_000_000, width: int = 3840, height: int = 2160) -> Workload:
    """1M Gaussians in 6 layers, 256 groups, 3840x2160."""
    rng = np.random.default_rng(seed)
    scene = make_hier_scene(rng, n, 6, 3, 256)
    motion = random_motion(rng, 256, 2)
    cam = orbit_camera(0.0, 4.0, width, height)
    return Workload("prec4k", scene, motion, [cam], [Request(cam, 1, level_mask(6))], {})


def sample_pixels(rng_or_seed, width, height, count) -> np.ndarray:
    """``count`` distinct pixel coordinates (x, y) drawn uniformly, int32 (count, 2)."""
    rng = np.random.default_rng(rng_or_seed) if not isinstance(rng_or_seed, np.random.Generator) \
        else rng_or_seed
    count = min(count, width * height)
    flat = rng.choice(width * height, size=count, replace=False)
    flat.sort()
    return np.stack([flat % width, flat // width], axis=1).astype(np.int32)


def selected_indices(layer_offsets, layer_mask: int) -> np.ndarray:
    """Global indices of the Gaussians of every layer whose bit is set, ascending."""
    parts = [np.arange(layer_offsets[l], layer_offsets[l + 1], dtype=np.int64)
             for l in range(len(layer_offsets) - 1) if (layer_mask >> l) & 1]
    return np.concatenate(parts) if parts else np.zeros(0, np.int64)


def quantize_scene(scene: Scene):
    """Reduced-precision storage of a scene, with per-channel FP32 scales.

    Positions, log-scales, quaternions and opacity logits are stored as
    bfloat16 of value / scale and SH coefficients as float8 e4m3 of
    value / scale, where each channel's scale is its absolute maximum divided
    by the format's largest finite value (bf16: 3.3895e38 is never reached, so
    its scale is absmax / 1 - a plain normalisation; e4m3: 448).  Returns the
    raw 16- and 8-bit planes as uint16 / uint8 arrays plus the scales.
    Dequantised value = float(stored) * scale (one FP32 multiply).
    """
    import torch  # library casts (round to nearest even)

    def bf16_plane(a):
        a = np.asarray(a, np.float32)
        flat = a.reshape(a.shape[0], -1)
        amax = np.abs(flat).max(axis=0).astype(np.float32)
        scale = np.where(amax > 0, amax, np.float32(1.0)).astype(np.float32)
        v = torch.from_numpy(flat / scale).to(torch.bfloat16)
        return v.view(torch.int16).numpy().view(np.uint16).reshape(a.shape), scale

    def e4m3_plane(a):
        a = np.asarray(a, np.float32)
        flat = a.reshape(a.shape[0], -1)
        amax = np.abs(flat).max(axis=0).astype(np.float32)
        scale = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
        v = torch.from_numpy(flat / scale).to(torch.float8_e4m3fn)
        return v.view(torch.uint8).numpy().reshape(a.shape), scale

    q = {}
    q["means"], q["means_scale"] = bf16_plane(scene.means)
    q["log_scales"], q["log_scales_scale"] = bf16_plane(scene.log_scales)
    q["quats"], q["quats_scale"] = bf16_plane(scene.quats)
    q["opacity_logits"], q["opacity_scale"] = bf16_plane(scene.opacity_logits[:, None])
    q["opacity_logits"] = q["opacity_logits"].reshape(-1)
    q["sh"], q["sh_scale"] = e4m3_plane(scene.sh)
    return q


PLANE_CHANNELS_FIXED = 11  # x, y, z | quaternion w, x, y, z | log-scales 3 | opacity logit


def quantize_planes(scene: Scene, plane_width: int = 512, pos_bits: int = 16, pitch_align: int = 256) -> dict:
    """The paper's decoded attribute format (Sec. 3.4): per layer, each attribute channel is
    quantised with its own min / max affine map - positions to uint16 (or uint32), every other
    channel to uint8 - and laid out as a 2D single-channel plane in which Gaussian j of the
    layer sits at row j // plane_width, column j % plane_width.  A layer's channel planes are
    stacked in one buffer (channel c in rows [c * rows, (c + 1) * rows), rows = ceil(n_l /
    plane_width)) whose rows are `pitch` bytes apart (the row size rounded up to `pitch_align`,
    like a video decoder's frame pitch); padding is zero.  This is the encoder side: it only
    produces inputs.  Channel order: x, y, z | quaternion w, x, y, z | log-scales 3 | opacity
    logit | SH (coefficient-major, then r, g, b).

    Returns plane_width, pos_bits, pitch (bytes of the uint8 planes), pos_pitch (bytes of the
    position planes), u8 (per layer a uint8 array (C - 3, rows, pitch)), pos (per layer a
    uint16/uint32 array (3, rows, pos_pitch / (pos_bits / 8))) and dequant, float32 (L, C, 2)
    = (lo, step) per layer and channel, step = (hi - lo) / (2^bits - 1)."""
    assert pos_bits in (16, 32)
    n_ch = PLANE_CHANNELS_FIXED + 3 * _sh_count(scene.sh_degree)
    attrs = np.concatenate([scene.means, scene.quats, scene.log_scales, scene.opacity_logits[:, None],
                            scene.sh.reshape(scene.n, -1)], axis=1).astype(np.float32)
    assert attrs.shape[1] == n_ch
    L = scene.n_layers
    pb = pos_bits // 8
    pitch = -(-plane_width // pitch_align) * pitch_align
    pos_pitch = -(-(plane_width * pb) // pitch_align) * pitch_align
    pos_dtype = np.uint16 if pos_bits == 16 else np.uint32
    dequant = np.zeros((L, n_ch, 2), np.float32)
    u8, pos = [], []
    for l in range(L):
        a, b = int(scene.layer_offsets[l]), int(scene.layer_offsets[l + 1])
        n_l = b - a
        rows = -(-n_l // plane_width)
        pl8 = np.zeros((n_ch - 3, rows, pitch), np.uint8)
        plp = np.zeros((3, rows, pos_pitch // pb), pos_dtype)
        j = np.arange(n_l)
        r, c = j // plane_width, j % plane_width
        for ch in range(n_ch):
            x = attrs[a:b, ch].astype(np.float64)
            bits = pos_bits if ch < 3 else 8
            top = float(2 ** bits - 1)
            lo = np.float32(x.min()) if n_l else np.float32(0.0)
            hi = np.float32(x.max()) if n_l else np.float32(0.0)
            step = np.float32((float(hi) - float(lo)) / top)
            dequant[l, ch] = (lo, step)
            if n_l == 0:
                continue
            code = np.zeros(n_l) if step == 0 else np.clip(np.rint((x - float(lo)) / float(step)), 0, top)
            if ch < 3:
                plp[ch, r, c] = code.astype(pos_dtype)
            else:
                pl8[ch - 3, r, c] = code.astype(np.uint8)
        u8.append(pl8)
        pos.append(plp)
    return {"plane_width": plane_width, "pos_bits": pos_bits, "pitch": pitch, "pos_pitch": pos_pitch,
            "u8": u8, "pos": pos, "dequant": dequant}


def motion_field_params(rng, n_levels=16, log2_T=15, n_min=16, n_max=512, lo=(-1.5,) * 3, hi=(1.5,) * 3,
                        table_sigma=1e-2, w_sigma=None, hidden=64) -> dict:
    """Seeded parameters of a per-Gaussian motion source (Sec. 3.2: a multi-resolution hash grid
    of n_levels levels, 2 features each, 2^log2_T entries per level, resolutions
    floor(n_min b^l) growing geometrically to n_max, and two MLPs of one hidden layer):
    table ~ U(-table_sigma, table_sigma), first-layer weights ~ N(0, 1/fan_in), output weights
    scaled by 0.05 so that the motion is small."""
    growth = float(np.exp((np.log(n_max) - np.log(n_min)) / max(n_levels - 1, 1)))
    T = 1 << log2_T
    d_in = n_levels * 2
    HIDDEN, FEAT = hidden, 2

    def w(o, i):
        s = (1.0 / np.sqrt(i)) if w_sigma is None else w_sigma
        return rng.normal(0, s, (o, i)).astype(np.float32)

    return {"table": rng.uniform(-table_sigma, table_sigma, (n_levels, T, FEAT)).astype(np.float32),
            "lo": np.asarray(lo, np.float32), "hi": np.asarray(hi, np.float32),
            "res": np.array([int(np.floor(n_min * growth ** l)) for l in range(n_levels)], np.int32),
            "w1t": w(HIDDEN, d_in), "b1t": rng.normal(0, 0.01, HIDDEN).astype(np.float32),
            "w2t": (w(3, HIDDEN) * 0.05).astype(np.float32), "b2t": np.zeros(3, np.float32),
            "w1r": w(HIDDEN, d_in), "b1r": rng.normal(0, 0.01, HIDDEN).astype(np.float32),
            "w2r": (w(4, HIDDEN) * 0.05).astype(np.float32), "b2r": np.zeros(4, np.float32)}
