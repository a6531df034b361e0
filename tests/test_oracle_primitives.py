"""Pins of the oracle's building blocks against mathematics and library routines.

Each check fixes a part of the oracle by something other than the oracle:
textbook identities of rotations, scipy's rotation composition and complex
spherical harmonics, quadrature, numpy's symmetric eigensolver and finite
differences.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

from synth import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_quats(n, seed=0):
    q = np.random.default_rng(seed).normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# ---------------------------------------------------------------- rotations

def test_quat_to_rot_orthonormal(oracle_lib):
    for q in _rand_quats(64):
        R = oracle_lib.quat_to_rot(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14, rtol=0)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
        assert np.allclose(oracle_lib.quat_to_rot(-q), R, atol=0, rtol=0)


def test_quat_to_rot_quarter_turns(oracle_lib):
    c = math.cos(math.pi / 4)
    # +90 degrees about x maps e_y -> e_z, about y maps e_z -> e_x, about z maps e_x -> e_y
    Rx = oracle_lib.quat_to_rot([c, c, 0, 0])
    Ry = oracle_lib.quat_to_rot([c, 0, c, 0])
    Rz = oracle_lib.quat_to_rot([c, 0, 0, c])
    assert np.allclose(Rx @ [0, 1, 0], [0, 0, 1], atol=1e-15, rtol=0)
    assert np.allclose(Ry @ [0, 0, 1], [1, 0, 0], atol=1e-15, rtol=0)
    assert np.allclose(Rz @ [1, 0, 0], [0, 1, 0], atol=1e-15, rtol=0)


def test_quat_to_rot_matches_scipy(oracle_lib):
    for q in _rand_quats(32, 1):
        ref = Rotation.from_quat(q, scalar_first=True).as_matrix()
        assert np.allclose(oracle_lib.quat_to_rot(q), ref, atol=1e-14, rtol=0)


def test_quat_mul_is_rotation_composition(oracle_lib):
    qs = _rand_quats(40, 2)
    for a, b in zip(qs[:20], qs[20:]):
        ab = oracle_lib.quat_mul(a, b)
        ref = (Rotation.from_quat(a, scalar_first=True) * Rotation.from_quat(b, scalar_first=True))
        assert np.allclose(oracle_lib.quat_to_rot(ab), ref.as_matrix(), atol=1e-14, rtol=0)
    assert np.allclose(oracle_lib.quat_mul([1, 0, 0, 0], qs[0]), qs[0], atol=0, rtol=0)


# ---------------------------------------------------------------- spherical harmonics

def _real_sh_scipy(deg, dirs):
    """Real SH from scipy's complex Y_l^m (Condon-Shortley phase included)."""
    x, y, z = dirs.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    out = np.zeros((dirs.shape[0], (deg + 1) ** 2))
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            if m == 0:
                out[:, k] = sph_harm_y(l, 0, theta, phi).real
            elif m > 0:
                out[:, k] = math.sqrt(2) * sph_harm_y(l, m, theta, phi).real
            else:
                out[:, k] = math.sqrt(2) * sph_harm_y(l, -m, theta, phi).imag
    return out


def _rand_dirs(n, seed=3):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy(oracle_lib):
    dirs = _rand_dirs(200)
    Y = oracle_lib.sh_eval(3, dirs)
    assert np.allclose(Y, _real_sh_scipy(3, dirs), atol=1e-12, rtol=0)


def test_sh_closed_forms_golden(oracle_lib):
    rows = np.loadtxt(os.path.join(GOLDEN, "sh_closed_forms.txt"))
    for x, y, z, k, val in rows:
        Y = oracle_lib.sh_eval(3, np.array([[x, y, z]]))[0]
        assert abs(Y[int(k)] - val) < 1e-14, (x, y, z, k)


def test_sh_orthonormal_by_quadrature(oracle_lib):
    # Gauss-Legendre in cos(theta) x uniform phi: exact for polynomials of degree <= 6
    nz, nphi = 12, 24
    zs, wz = np.polynomial.legendre.leggauss(nz)
    phis = 2 * np.pi * np.arange(nphi) / nphi
    Z, P = np.meshgrid(zs, phis, indexing="ij")
    st = np.sqrt(1 - Z ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle_lib.sh_eval(3, dirs)
    gram = (Y * w[:, None]).T @ Y
    assert np.allclose(gram, np.eye(16), atol=1e-12, rtol=0)


def test_sh_degree0_constant(oracle_lib):
    Y = oracle_lib.sh_eval(0, _rand_dirs(10))
    assert np.allclose(Y, 0.5 / math.sqrt(math.pi), atol=0, rtol=1e-15)


def test_sh_gradient_tangential_matches_fd(oracle_lib):
    dirs = _rand_dirs(20, 5)
    Y, dY = oracle_lib.sh_eval(3, dirs, with_grad=True)
    eps = 1e-6
    for i in range(dirs.shape[0]):
        d = dirs[i]
        for a in range(3):
            e = np.zeros(3); e[a] = eps
            fd = (oracle_lib.sh_eval(3, (d + e)[None])[0] - oracle_lib.sh_eval(3, (d - e)[None])[0]) / (2 * eps)
            assert np.allclose(dY[i, :, a], fd, atol=1e-7, rtol=0)


# ---------------------------------------------------------------- geometry

def _one_gaussian_scene(mu, log_s, q, logit=0.0, rgb=(0.8, 0.5, 0.2)):
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = (np.asarray(rgb) - 0.5) / (0.5 / math.sqrt(math.pi))
    return scenes.Scene(np.array([mu], np.float32), np.array([log_s], np.float32),
                        np.array([q], np.float32), np.array([logit], np.float32), sh,
                        np.zeros(1, np.int32), np.array([0, 1], np.int64), 0, 1)


def test_isotropic_covariance_any_rotation(oracle_lib):
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64)
    opts = oracle_lib.default_options()
    s = math.exp(-2.0)
    for q in _rand_quats(8, 7):
        sc = _one_gaussian_scene([0.1, -0.2, 0.3], [-2.0, -2.0, -2.0], q)
        g = oracle_lib.geom(sc, None, 0, cam, opts, 0)
        assert np.allclose(g["sigma3"], s * s * np.eye(3), atol=1e-12, rtol=0)


def test_covariance_eigenvalues(oracle_lib):
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64)
    opts = oracle_lib.default_options()
    ls = np.array([-2.0, -2.7, -3.1], np.float32)
    for q in _rand_quats(8, 8):
        sc = _one_gaussian_scene([0.0, 0.0, 0.0], ls, q)
        g = oracle_lib.geom(sc, None, 0, cam, opts, 0)
        ev = np.linalg.eigh(g["sigma3"])[0]
        assert np.allclose(np.sort(ev), np.sort(np.exp(2 * ls.astype(np.float64))), rtol=1e-10)


def test_on_axis_projection_and_isotropic_ewa(oracle_lib):
    W, H = 96, 64
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), W, H)
    opts = oracle_lib.default_options()
    ls = -2.5
    sc = _one_gaussian_scene([0, 0, 0], [ls] * 3, [1, 0, 0, 0])
    g = oracle_lib.geom(sc, None, 0, cam, opts, 0)
    assert abs(g["u"] - W / 2) < 1e-12 and abs(g["v"] - H / 2) < 1e-12
    s = math.exp(ls)
    z = 3.0
    dil = float(np.float32(0.3))  # options are FP32 values on both sides
    expect = (cam.fx * s / z) ** 2 + dil
    assert np.allclose(g["sigma2"], np.diag([expect, (cam.fy * s / z) ** 2 + dil]), rtol=1e-12, atol=1e-12)


def test_off_axis_projection_hand_computed(oracle_lib):
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 128, 128)
    opts = oracle_lib.default_options()
    sc = _one_gaussian_scene([0.5, -0.25, 1.0], [-3, -3, -3], [1, 0, 0, 0])
    g = oracle_lib.geom(sc, None, 0, cam, opts, 0)
    # camera point (0.5, -0.25, 4): u = fx * 0.125 + 64, v = fy * (-0.0625) + 64
    assert abs(g["u"] - (cam.fx * 0.125 + 64)) < 1e-9
    assert abs(g["v"] - (cam.fy * -0.0625 + 64)) < 1e-9


def test_jacobian_is_projection_derivative(oracle_lib):
    cam = scenes.look_at_camera((0.3, 0.2, -3), (0, 0, 0), 128, 96)
    opts = oracle_lib.default_options()
    rng = np.random.default_rng(9)
    for _ in range(8):
        mu = rng.uniform(-0.5, 0.5, 3)
        sc = _one_gaussian_scene(mu, [-3, -3, -3], [1, 0, 0, 0])
        g = oracle_lib.geom(sc, None, 0, cam, opts, 0)
        c = g["cam_point"]

        def proj(p):
            return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

        eps = 1e-6
        Jfd = np.stack([(proj(c + e) - proj(c - e)) / (2 * eps) for e in np.eye(3) * eps], 1)
        J = g["J"]
        assert np.allclose([J[0], J[1], J[2], J[3]], [Jfd[0, 0], Jfd[0, 2], Jfd[1, 1], Jfd[1, 2]],
                           rtol=1e-7)


def test_radius_from_eigenvalues(oracle_lib):
    w = scenes.tiny()
    cam = w.cameras[0]
    opts = oracle_lib.default_options()
    b = oracle_lib.bin_f32(w.scene, None, 0, cam, opts, 1)
    checked = 0
    for j in range(0, w.scene.n, 37):
        if not b["visible"][j]:
            continue
        g = oracle_lib.geom(w.scene, None, 0, cam, opts, j)
        lam = np.linalg.eigvalsh(g["sigma2"]).max()
        r = 3 * math.sqrt(lam)
        if abs(r - round(r)) < 1e-4:
            continue
        assert b["radius"][j] == math.ceil(r)
        checked += 1
    assert checked > 40


def test_mirror_agrees_with_fp64_geometry(oracle_lib):
    w = scenes.tiny()
    cam = w.cameras[0]
    opts = oracle_lib.default_options()
    b = oracle_lib.bin_f32(w.scene, None, 0, cam, opts, 1)
    for j in range(0, w.scene.n, 53):
        g = oracle_lib.geom(w.scene, None, 0, cam, opts, j)
        assert abs(b["uv"][j, 0] - g["u"]) < 1e-4 and abs(b["uv"][j, 1] - g["v"]) < 1e-4
        assert np.allclose(b["conic"][j], g["conic"], rtol=1e-4, atol=1e-7)
        assert abs(b["depth"][j] - g["cam_point"][2]) < 1e-6


def test_mirror_rect_is_pixel_square(oracle_lib):
    """Without the alpha cull, every pixel of the rectangle has its centre within r of
    (u, v), and its neighbours do not."""
    w = scenes.tiny()
    cam = w.cameras[0]
    opts = oracle_lib.default_options(alpha_cull=0)
    b = oracle_lib.bin_f32(w.scene, None, 0, cam, opts, 1)
    for j in range(0, w.scene.n, 11):
        if not b["visible"][j]:
            continue
        u, v = b["uv"][j].astype(np.float64)
        r = b["radius"][j]
        x0, x1, y0, y1 = b["rect"][j]
        assert abs(x0 + 0.5 - u) <= r + 1e-3 and abs(x1 + 0.5 - u) <= r + 1e-3
        if x0 > 0:
            assert abs(x0 - 0.5 - u) >= r - 1e-3
        if x1 < cam.width - 1:
            assert abs(x1 + 1.5 - u) >= r - 1e-3
        assert abs(y0 + 0.5 - v) <= r + 1e-3 and abs(y1 + 0.5 - v) <= r + 1e-3


# ---------------------------------------------------------------- reduced-precision formats

def test_decoders_match_torch_casts(oracle_lib):
    import torch
    x = torch.linspace(-500, 500, 4001, dtype=torch.float32)
    x = torch.cat([x, torch.tensor([0.0, -0.0, 1e-3, 2.0 ** -9, 448.0, -448.0])])
    b = x.to(torch.bfloat16)
    raw = b.view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle_lib.decode_bf16(raw), b.float().numpy())
    e = x.clamp(-448, 448).to(torch.float8_e4m3fn)
    raw8 = e.view(torch.uint8).numpy()
    assert np.array_equal(oracle_lib.decode_e4m3(raw8), e.float().numpy())
    allcodes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(allcodes).view(torch.float8_e4m3fn).float().numpy()
    got = oracle_lib.decode_e4m3(allcodes)
    finite = np.isfinite(ref)
    assert np.array_equal(got[finite], ref[finite]) and np.all(np.isnan(got[~finite]))
