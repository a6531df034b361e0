"""Pins of the oracle's per-Gaussian motion source (Sec. 3.2, rigid transformation: a
multi-resolution hash grid interpolated at the frame t-1 positions, then two small MLPs for the
translation and the rotation).

* a Gaussian exactly on a grid vertex reads that vertex's table entry (weights 1 / 0);
* a level whose table holds an affine function of the vertex coordinates interpolates it
  exactly (pins the trilinear weights, the corner order and the dense index order);
* the spatial hash of two vertices, worked out by hand (uint32 wrap-around, xor, mod T);
* zero parameters give the identity motion (t = 0, q = (1, 0, 0, 0));
* the MLP forward, the MLP backward and the table's scatter backward against PyTorch FP64
  autograd of an independent formulation (torch.nn.functional.linear / relu on gathered
  features).
"""
import numpy as np
import pytest
import torch

from oracle import motion_net as mn
from synth import scenes


def _params(rng, res, log2_T=15, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    p = scenes.motion_field_params(rng, n_levels=len(res), log2_T=log2_T, lo=lo, hi=hi)
    p["res"] = np.asarray(res, np.int32)
    return p


def test_vertex_reads_its_entry():
    rng = np.random.default_rng(0)
    p = _params(rng, [16, 8])
    mu = np.array([[3 / 16, 5 / 16, 7 / 16]], np.float32)
    h, _ = mn.encode(mu, p["table"], p["lo"], p["hi"], p["res"])
    assert np.array_equal(h[0, 0:2], p["table"][0, 3 + 17 * (5 + 17 * 7)].astype(np.float64))
    # level 1 (resolution 8): p = (1.5, 2.5, 3.5), the cell's centre: the mean of its 8 vertices
    idx = [(1 + a) + 9 * ((2 + b) + 9 * (3 + c)) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    want = p["table"][1, idx].astype(np.float64).mean(axis=0)
    assert np.allclose(h[0, 2:4], want, rtol=0, atol=1e-15)


def test_affine_table_is_interpolated_exactly():
    rng = np.random.default_rng(1)
    p = _params(rng, [8])
    n = 9
    coef = np.array([[0.25, 0.5, -0.75, 1.0], [-1.0, 0.125, 0.25, -0.5]])  # per feature: a + b i + c j + d k
    for k in range(n):
        for j in range(n):
            for i in range(n):
                p["table"][0, i + n * (j + n * k)] = coef[:, 0] + coef[:, 1] * i + coef[:, 2] * j + coef[:, 3] * k
    mu = rng.uniform(0, 1, (200, 3)).astype(np.float32)
    h, _ = mn.encode(mu, p["table"], p["lo"], p["hi"], p["res"])
    pos = (mu.astype(np.float32) * np.float32(8)).astype(np.float64)   # lo = 0, hi = 1: x = mu
    want = coef[:, 0][None] + pos @ coef[:, 1:].T
    assert np.allclose(h, want, rtol=0, atol=1e-12)


def test_spatial_hash_by_hand():
    # (1, 2, 3) and (7, 11, 13) at T = 2^15: (i ^ (2654435761 j mod 2^32) ^ (805459861 k mod 2^32)) mod T
    got = mn.vertex_index(np.array([[1, 2, 3], [7, 11, 13]]), 100, 1 << 15)
    assert list(got) == [30172, 18445]
    # a dense level indexes i + (N+1) (j + (N+1) k)
    assert list(mn.vertex_index(np.array([[1, 2, 3]]), 4, 1 << 15)) == [1 + 5 * (2 + 5 * 3)]


def test_zero_parameters_give_identity_motion():
    rng = np.random.default_rng(2)
    p = _params(rng, [16, 32, 64])
    for k in list(p):
        if isinstance(p[k], np.ndarray) and p[k].dtype == np.float32 and k not in ("lo", "hi"):
            p[k] = np.zeros_like(p[k])
    t, q = mn.forward(rng.uniform(-1, 1, (50, 3)).astype(np.float32), p)
    assert np.array_equal(t, np.zeros_like(t))
    assert np.array_equal(q, np.tile([1.0, 0.0, 0.0, 0.0], (50, 1)))


def test_forward_backward_against_torch_autograd():
    rng = np.random.default_rng(3)
    p = _params(rng, [16, 23, 40, 70, 128], log2_T=12, lo=(-1.2, -1.1, -1.3), hi=(1.1, 1.2, 1.0))
    mu = rng.uniform(-1.1, 1.1, (300, 3)).astype(np.float32)
    t, q = mn.forward(mu, p)
    d_t = rng.normal(0, 1, t.shape)
    d_q = rng.normal(0, 1, q.shape)
    g = mn.backward(mu, p, d_t, d_q)
    # independent formulation: gather the corner features with torch, MLPs with F.linear
    _, parts = mn.encode(mu, p["table"], p["lo"], p["hi"], p["res"])
    tab = torch.tensor(p["table"], dtype=torch.float64, requires_grad=True)
    feats = []
    for l, corners in enumerate(parts):
        acc = 0
        for idx, wt in corners:
            acc = acc + torch.tensor(wt)[:, None] * tab[l][torch.tensor(idx)]
        feats.append(acc)
    h = torch.cat(feats, dim=1)
    W = {k: torch.tensor(p[k], dtype=torch.float64, requires_grad=True)
         for k in ("w1t", "b1t", "w2t", "b2t", "w1r", "b1r", "w2r", "b2r")}
    tt = torch.nn.functional.linear(torch.relu(torch.nn.functional.linear(h, W["w1t"], W["b1t"])), W["w2t"], W["b2t"])
    qq = torch.nn.functional.linear(torch.relu(torch.nn.functional.linear(h, W["w1r"], W["b1r"])), W["w2r"], W["b2r"])
    qq = qq + torch.tensor([1.0, 0.0, 0.0, 0.0], dtype=torch.float64)
    assert np.allclose(tt.detach().numpy(), t, rtol=0, atol=1e-13)
    assert np.allclose(qq.detach().numpy(), q, rtol=0, atol=1e-13)
    loss = (tt * torch.tensor(d_t)).sum() + (qq * torch.tensor(d_q)).sum()
    loss.backward()
    for k, v in W.items():
        assert np.allclose(g[k], v.grad.numpy(), rtol=1e-12, atol=1e-12), k
    assert np.allclose(g["table"], tab.grad.numpy(), rtol=1e-12, atol=1e-12)
    assert np.abs(g["table"]).max() > 0
