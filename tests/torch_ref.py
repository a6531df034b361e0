"""A second, independent FP64 formulation of the rasterizer in PyTorch autograd.

Test-only.  It pins the oracle's hand-written reverse mode: it shares no code
with the C oracle and formulates every step differently - spherical harmonics
by the associated-Legendre recurrence in spherical angles, compositing as a
masked cumulative product over a dense (pixel x Gaussian) matrix - and lets
autograd produce the gradient.  Discrete decisions (visibility, depth order,
footprint rectangle) come from the oracle's FP32 binning mirror, as they do
for the oracle itself; per-pixel skip/stop decisions are taken here in FP64.
"""
import math

import numpy as np
import torch


def _assoc_legendre(l, m, z):
    """P_l^m(z) with the Condon-Shortley phase, by the standard recurrence."""
    pmm = torch.ones_like(z)
    if m > 0:
        somx2 = torch.sqrt(torch.clamp(1 - z * z, min=0))
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * somx2
            fact += 2.0
    if l == m:
        return pmm
    pmmp1 = z * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = None
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * z * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def real_sh(deg, d):
    """(n, (deg+1)^2) real SH of unit directions d (n, 3)."""
    z = d[:, 2]
    phi = torch.atan2(d[:, 1], d[:, 0])
    cols = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = _assoc_legendre(l, am, z)
            if m == 0:
                cols.append(K * P)
            elif m > 0:
                cols.append(math.sqrt(2) * K * P * torch.cos(m * phi))
            else:
                cols.append(math.sqrt(2) * K * P * torch.sin(am * phi))
    return torch.stack(cols, 1)


def _quat_rot(q):
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z], -1),
    ], -2)


def _hamilton(a, b):
    a0, a1, a2, a3 = a.unbind(-1)
    b0, b1, b2, b3 = b.unbind(-1)
    return torch.stack([a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3,
                        a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2,
                        a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1,
                        a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0], -1)


def render_and_grad(scene, motion, frame, cam, opts, bins, dL_dimage):
    """Returns (image (3,H,W) float64, dict of gradients) for L = sum(dL_dimage * image)."""
    dt = torch.float64
    sel = torch.from_numpy(bins["sel"])
    vis = torch.from_numpy(bins["visible"].astype(bool))
    order = np.lexsort((bins["sel"], bins["depth"]))
    order = order[bins["visible"][order] != 0]
    P = {k: torch.tensor(np.asarray(getattr(scene, k), np.float64), dtype=dt, requires_grad=True)
         for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    if motion is not None:
        gq = torch.tensor(motion.q[frame].astype(np.float64), requires_grad=True)
        gt = torch.tensor(motion.t[frame].astype(np.float64), requires_grad=True)
    else:
        gq = torch.tensor([[1.0, 0, 0, 0]], dtype=dt, requires_grad=True)
        gt = torch.zeros((1, 3), dtype=dt, requires_grad=True)
    gid = torch.from_numpy(scene.group_id.astype(np.int64)) if motion is not None else \
        torch.zeros(scene.n, dtype=torch.long)
    idx = sel[torch.from_numpy(order)]
    g = gid[idx]
    mu = P["means"][idx] + gt[g]
    p = _hamilton(gq[g], P["quats"][idx])
    qn = p / p.norm(dim=-1, keepdim=True)
    R = _quat_rot(qn)
    s = torch.exp(P["log_scales"][idx])
    M = R * s[:, None, :]
    Sig = M @ M.transpose(1, 2)
    Wc = torch.tensor(np.asarray(cam.R, np.float64).reshape(3, 3), dtype=dt)
    tc = torch.tensor(np.asarray(cam.t, np.float64), dtype=dt)
    c = mu @ Wc.T + tc
    x, y, z = c.unbind(-1)
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    cx, cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    clampk = float(np.float32(opts.get("clamp", 1.3)))
    limx = clampk * (0.5 * cam.width / fx)
    limy = clampk * (0.5 * cam.height / fy)
    xt = torch.clamp(x / z, -limx, limx)
    yt = torch.clamp(y / z, -limy, limy)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * xt / z], -1),
                     torch.stack([zero, fy / z, -fy * yt / z], -1)], -2)
    T = J @ Wc
    S2 = T @ Sig @ T.transpose(1, 2)
    dil = float(np.float32(opts.get("dilation", 0.3)))
    A = S2[:, 0, 0] + dil
    B = S2[:, 0, 1]
    Cc = S2[:, 1, 1] + dil
    det = A * Cc - B * B
    ca, cb, cc = Cc / det, -B / det, A / det
    u = fx * (x / z) + cx
    v = fy * (y / z) + cy
    o = torch.sigmoid(P["opacity_logits"][idx])
    campos = torch.tensor(np.asarray(cam.campos, np.float64), dtype=dt)
    dv = mu - campos
    dirs = dv / dv.norm(dim=-1, keepdim=True)
    Y = real_sh(scene.sh_degree, dirs)
    rgb = torch.clamp(torch.einsum("nk,nkc->nc", Y, P["sh"][idx]) + 0.5, min=0)

    H, W = cam.height, cam.width
    py, px = torch.meshgrid(torch.arange(H, dtype=dt), torch.arange(W, dtype=dt), indexing="ij")
    pcx = (px + 0.5).reshape(-1, 1)
    pcy = (py + 0.5).reshape(-1, 1)
    rect = torch.from_numpy(bins["rect"][order].astype(np.int64))
    pxi = px.reshape(-1, 1).long()
    pyi = py.reshape(-1, 1).long()
    inside = (pxi >= rect[None, :, 0]) & (pxi <= rect[None, :, 1]) & \
             (pyi >= rect[None, :, 2]) & (pyi <= rect[None, :, 3])
    dx = pcx - u[None, :]
    dy = pcy - v[None, :]
    power = -0.5 * (ca[None] * dx * dx + cc[None] * dy * dy) - cb[None] * dx * dy
    alpha = torch.clamp(o[None] * torch.exp(power), max=0.99)
    with torch.no_grad():
        use = inside & (power <= 0) & (alpha >= 1.0 / 255.0)
        a_use = torch.where(use, alpha, torch.zeros_like(alpha))
        Tafter = torch.cumprod(1 - a_use, dim=1)
        stop = use & (Tafter < 1e-4)
        stopped = torch.cumsum(stop.to(torch.int64), dim=1) > 0
        use = use & ~stopped
    a = torch.where(use, alpha, torch.zeros_like(alpha))
    Tcum = torch.cumprod(1 - a, dim=1)
    Tex = torch.cat([torch.ones_like(Tcum[:, :1]), Tcum[:, :-1]], 1)
    wgt = a * Tex
    bg = torch.tensor(np.asarray(opts.get("bg", (0.0, 0.0, 0.0)), np.float32).astype(np.float64), dtype=dt)
    img = wgt @ rgb + Tcum[:, -1:] * bg[None] if a.shape[1] > 0 else bg[None].expand(H * W, 3)
    img = img.T.reshape(3, H, W)
    L = (img * torch.from_numpy(np.asarray(dL_dimage, np.float64))).sum()
    L.backward()
    grads = {k: P[k].grad.numpy() for k in P}
    grads["group_q"] = gq.grad.numpy()
    grads["group_t"] = gt.grad.numpy()
    return img.detach().numpy(), grads
