"""Oracle of the per-Gaussian motion source (Sec. 3.2, rigid transformation): the positions of
frame t-1 are encoded by a multi-resolution hash grid (trilinear interpolation of per-level
feature tables) and two small MLPs map the features to the translation and the rotation of
each Gaussian.  TEST INFRASTRUCTURE ONLY (tests, the smoke check and the CPU baseline use it).

The paper fixes none of the sizes; the readings (the multiresolution hash encoding of
Mueller et al. 2022, which the paper's hash grid refers to, and the lightweight MLPs of the
3DGStream line it builds on):

* L_h levels (<= 16), F = 2 features per level, T = 2^log2_T entries per level; level l has
  resolution N_l (given with the parameters; the generator uses floor(N_min b^l));
* x = (mu - lo) / (hi - lo) per axis, clamped to [0, 1]; p = x * N_l; cell = floor(p)
  clamped to [0, N_l - 1]; w = p - cell.  These are evaluated in FP32 (they decide the cell,
  an integer), the rest in FP64;
* vertex (i, j, k) of level l is entry i + (N_l + 1) (j + (N_l + 1) k) when (N_l + 1)^3 <= T,
  else (i * 1 xor j * 2654435761 xor k * 805459861) mod 2^32 mod T (the spatial hash);
* h = concatenation over levels of the trilinear blend of the 8 cell vertices' features;
* translation = W2t relu(W1t h + b1t) + b2t (3 outputs), rotation quaternion =
  W2r relu(W1r h + b1r) + b2r + (1, 0, 0, 0) (4 outputs, not normalised: the renderer
  normalises q_g (x) q, and |q_g (x) q| = |q_g| |q|); hidden width 64.
"""
import numpy as np

HIDDEN = 64
FEAT = 2
PRIMES = (1, 2654435761, 805459861)


def cells_f32(means, lo, hi, res):
    """Per level: the cell (int, (n, 3)) and the weights (FP32 lifted to float64, (n, 3))."""
    m = np.asarray(means, np.float32)
    lo32, hi32 = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    x = (m - lo32) / (hi32 - lo32)
    x = np.minimum(np.maximum(x, np.float32(0.0)), np.float32(1.0)).astype(np.float32)
    out = []
    for n_l in res:
        p = (x * np.float32(n_l)).astype(np.float32)
        c = np.floor(p).astype(np.int64)
        c = np.minimum(np.maximum(c, 0), int(n_l) - 1)
        w = (p - c.astype(np.float32)).astype(np.float32)
        out.append((c, w.astype(np.float64)))
    return out


def vertex_index(c, n_l: int, table_size: int) -> np.ndarray:
    """Table entry of integer vertices c (n, 3) of a level of resolution n_l."""
    c = np.asarray(c, np.int64)
    if (n_l + 1) ** 3 <= table_size:
        return c[:, 0] + (n_l + 1) * (c[:, 1] + (n_l + 1) * c[:, 2])
    h = np.zeros(c.shape[0], np.uint64)
    for a in range(3):
        h ^= (c[:, a].astype(np.uint64) * np.uint64(PRIMES[a])) & np.uint64(0xFFFFFFFF)
    return (h % np.uint64(table_size)).astype(np.int64)


def encode(means, table, lo, hi, res):
    """Hash-grid features h (n, L_h * F) and, for the backward, the corners and weights."""
    L, T, F = table.shape
    cells = cells_f32(means, lo, hi, res)
    n = np.asarray(means).shape[0]
    h = np.zeros((n, L * F))
    parts = []
    for l in range(L):
        c, w = cells[l]
        corners = []
        for corner in range(8):
            o = np.array([(corner >> a) & 1 for a in range(3)], np.int64)
            idx = vertex_index(c + o, int(res[l]), T)
            wt = np.prod(np.where(o[None, :] == 1, w, 1.0 - w), axis=1)
            h[:, l * F:(l + 1) * F] += wt[:, None] * table[l, idx, :].astype(np.float64)
            corners.append((idx, wt))
        parts.append(corners)
    return h, parts


def forward(means, params: dict):
    """Per-Gaussian translation (n, 3) and rotation quaternion (n, 4), FP64."""
    h, _ = encode(means, params["table"], params["lo"], params["hi"], params["res"])
    zt = h @ params["w1t"].T.astype(np.float64) + params["b1t"]
    t = np.maximum(zt, 0.0) @ params["w2t"].T.astype(np.float64) + params["b2t"]
    zr = h @ params["w1r"].T.astype(np.float64) + params["b1r"]
    q = np.maximum(zr, 0.0) @ params["w2r"].T.astype(np.float64) + params["b2r"]
    q[:, 0] += 1.0
    return t, q


def backward(means, params: dict, d_t, d_q) -> dict:
    """Gradients of L = sum(d_t * t) + sum(d_q * q) w.r.t. the table and the MLP weights."""
    table = params["table"]
    h, parts = encode(means, table, params["lo"], params["hi"], params["res"])
    d_t = np.asarray(d_t, np.float64)
    d_q = np.asarray(d_q, np.float64)
    g = {}
    dh = np.zeros_like(h)
    for net, d_out in (("t", d_t), ("r", d_q)):
        w1 = params["w1" + net].astype(np.float64)
        w2 = params["w2" + net].astype(np.float64)
        z = h @ w1.T + params["b1" + net]
        a = np.maximum(z, 0.0)
        g["w2" + net] = d_out.T @ a
        g["b2" + net] = d_out.sum(0)
        dz = (d_out @ w2) * (z > 0)
        g["w1" + net] = dz.T @ h
        g["b1" + net] = dz.sum(0)
        dh += dz @ w1
    L, T, F = table.shape
    dtab = np.zeros((L, T, F))
    for l in range(L):
        for idx, wt in parts[l]:
            np.add.at(dtab[l], idx, wt[:, None] * dh[:, l * F:(l + 1) * F])
    g["table"] = dtab
    return g
