"""Pins of the oracle's residual deformation (Sec. 3.2, Eq. 7): the log-scales, opacity
logits and SH coefficients of frame t are the keyframe's plus the frame's residuals,
before activation (reading: additive in log-scale, logit and SH-coefficient space).

* zero residuals change nothing, bit for bit;
* with attributes and residuals on a 2^-12 grid (their FP32 and FP64 sums are exact), the
  render and the binning mirror with a residual on ONE attribute equal those of the scene
  with that residual added beforehand, bit for bit (the gradients to 1e-12), and differ from the
  undeformed scene - so a residual that is dropped, applied to the wrong attribute or
  applied with the wrong sign fails;
* the render's gradient w.r.t. a residual equals central finite differences in the residual.
"""
import numpy as np
import pytest

from synth import scenes


def _grid(x, step=2.0 ** -12):
    return (np.round(np.asarray(x, np.float64) / step) * step).astype(np.float32)


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(31)
    sc = scenes.make_hier_scene(rng, 3000, 3, 3, 8)
    sc.log_scales = _grid(sc.log_scales)
    sc.opacity_logits = _grid(sc.opacity_logits)
    sc.sh = _grid(sc.sh)
    motion = scenes.random_motion(rng, 8, 3)
    res = scenes.random_residual(5, sc.n, 3, frame=2, ls_sigma=0.05, logit_sigma=0.3, sh_sigma=0.05)
    res = scenes.Residual(_grid(res.ls), _grid(res.logit), _grid(res.sh))
    cam = scenes.orbit_camera(0.7, 4.0, 96, 72)
    return sc, motion, res, cam


def _only(res, name):
    return scenes.Residual(res.ls if name == "ls" else None, res.logit if name == "logit" else None,
                           res.sh if name == "sh" else None)


def test_zero_residual_changes_nothing(oracle_lib, case):
    sc, motion, res, cam = case
    opts = oracle_lib.default_options(tile=(8, 32))
    zero = scenes.Residual(np.zeros_like(res.ls), np.zeros_like(res.logit), np.zeros_like(res.sh))
    a = oracle_lib.render(sc, motion, 1, cam, opts, scenes.level_mask(3))
    b = oracle_lib.render(sc, motion, 1, cam, opts, scenes.level_mask(3), residual=zero)
    assert np.array_equal(a["image"], b["image"])
    for k in ("visible", "depth", "rect", "trect", "tc"):
        assert np.array_equal(a["bins"][k], b["bins"][k]), k


@pytest.mark.parametrize("name", ["ls", "logit", "sh"])
def test_residual_equals_pre_added_scene(oracle_lib, case, name):
    sc, motion, res, cam = case
    opts = oracle_lib.default_options(tile=(8, 32))
    r1 = _only(res, name)
    pre = scenes.apply_residual(sc, r1)
    # the grid makes the FP32 sums exact
    if name == "ls":
        assert np.array_equal(pre.log_scales.astype(np.float64), sc.log_scales.astype(np.float64) + r1.ls)
    mask = scenes.level_mask(3)
    a = oracle_lib.render(sc, motion, 1, cam, opts, mask, residual=r1)
    b = oracle_lib.render(pre, motion, 1, cam, opts, mask)
    plain = oracle_lib.render(sc, motion, 1, cam, opts, mask)
    assert np.array_equal(a["image"], b["image"]), name
    assert np.abs(a["image"] - plain["image"]).max() > 1e-3, name
    for k in ("visible", "depth", "rect", "trect", "tc", "uv", "conic"):
        assert np.array_equal(a["bins"][k], b["bins"][k]), (name, k)
    up = np.random.default_rng(4).normal(0, 1, (3, cam.height, cam.width))
    ga = oracle_lib.grad(sc, motion, 1, cam, opts, up, mask, residual=r1)
    gb = oracle_lib.grad(pre, motion, 1, cam, opts, up, mask)
    # the oracle's per-thread partial sums make its gradients reproducible to ~1e-15 only
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "group_q", "group_t"):
        assert np.abs(ga[k] - gb[k]).max() <= 1e-12 * np.abs(gb[k]).max(), (name, k)


def test_residual_gradient_matches_central_differences(oracle_lib):
    w = scenes.diff_subscene()
    sc, motion, cam = w.scene, w.motion, w.cameras[0]
    res = scenes.random_residual(9, sc.n, sc.sh_degree, frame=3)
    opts = oracle_lib.default_options()
    up = np.random.default_rng(1).normal(0, 1, (3, cam.height, cam.width))
    g = oracle_lib.grad(sc, motion, 1, cam, opts, up, residual=res)
    bins = g["bins"]

    def loss():
        r = oracle_lib.render(sc, motion, 1, cam, opts, bins=bins, residual=res)
        return float((r["image"] * up).sum()), r["signature"]

    _, sig0 = loss()
    rng = np.random.default_rng(8)
    vis = np.nonzero(bins["visible"])[0]
    eps = 1e-4
    checked = total = 0
    for field, gname, ncomp in (("ls", "log_scales", 3), ("logit", "opacity_logits", 1), ("sh", "sh", 48)):
        arr = getattr(res, field).reshape(sc.n, -1)
        for j in rng.choice(vis, 10, replace=False):
            comp = int(rng.integers(ncomp))
            total += 1
            orig = arr[j, comp]
            hi, lo = np.float32(orig + eps), np.float32(orig - eps)
            arr[j, comp] = hi
            lp, sp = loss()
            arr[j, comp] = lo
            lm, sm = loss()
            arr[j, comp] = orig
            if not (np.array_equal(sp, sig0) and np.array_equal(sm, sig0)):
                continue  # a skip / stop decision changed inside the step
            fd = (lp - lm) / (float(hi) - float(lo))
            an = g[gname].reshape(sc.n, -1)[j, comp]
            tol = 1e-4 * max(abs(an), 1e-3 * np.abs(g[gname]).max()) + 1e-9
            assert abs(fd - an) <= tol, (field, j, comp, fd, an)
            checked += 1
    assert checked >= 0.8 * total, (checked, total)
