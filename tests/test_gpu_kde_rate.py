"""The KDE rate estimate on the GPU (Sec. 3.3) against the FP64 oracle (oracle.kde_rate):
several channel shapes in one call (narrow and wide normals, a skewed gamma, a constant and a
negative-valued channel, a ragged length), the unsupported cases (a symbol span above 8192, a
non-finite value) reported as NaN, and the paper's setting: every quantised attribute channel
of a layer of 50k Gaussians (uint8 symbols).  The training form (noise-injected values, the
symbols' density held fixed, gradient through the values) against the oracle's training form,
equal to the symbol rate on integer inputs, with NaN rows for unsupported channels."""
import numpy as np
import pytest
import torch

from oracle import kde_rate as kr
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gc():
    import paper_2509_17513_b300 as gc
    return gc


def test_kde_rate_matches_oracle(gc):
    rng = np.random.default_rng(4)
    n = 20011
    chans = [rng.normal(0, 0.3, n), rng.normal(5, 3.0, n), rng.normal(-100, 40.0, n),
             rng.gamma(1.5, 12.0, n), np.full(n, 3.7), rng.uniform(-300, -250, n)]
    y = np.stack(chans).astype(np.float32)
    r = gc.Renderer(0)
    got = r.kde_rate(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    want = np.array([kr.rate(c) for c in y])
    assert np.all(np.abs(got - want) <= 2e-5 * np.maximum(np.abs(want), 1.0)), (got, want)


def test_kde_rate_unsupported_channels(gc):
    rng = np.random.default_rng(5)
    y = np.stack([rng.uniform(0, 20000, 1000), rng.normal(0, 1, 1000), rng.normal(0, 1, 1000)]).astype(np.float32)
    y[2, 17] = np.inf
    r = gc.Renderer(0)
    got = r.kde_rate(torch.from_numpy(y).cuda()).cpu().numpy()
    assert np.isnan(got[0]) and np.isnan(got[2])
    assert abs(float(got[1]) - kr.rate(y[1])) <= 2e-5 * max(kr.rate(y[1]), 1.0)


def test_kde_rate_of_quantised_attribute_planes(gc):
    rng = np.random.default_rng(6)
    scene = scenes.make_hier_scene(rng, 12000, 2, 3, 4)
    planes = scenes.quantize_planes(scene, plane_width=128)
    n0 = int(scene.layer_offsets[1])
    u8 = planes["u8"][0]
    # Gaussian j of the layer sits at (j // width, j % width): drop the row padding
    y = u8[:, :, :128].reshape(u8.shape[0], -1)[:, :n0].astype(np.float32)
    r = gc.Renderer(0)
    got = r.kde_rate(torch.from_numpy(np.ascontiguousarray(y)).cuda()).cpu().numpy().astype(np.float64)
    want = np.array([kr.rate(c) for c in y])
    assert np.all(np.abs(got - want) <= 2e-5 * np.maximum(np.abs(want), 1.0))
    assert np.all((got > 0) & (got < 8.5))   # uint8 symbols: at most about 8 bits


# ---- training form (noise-injected values, symbol density held fixed) and its gradient

def _noisy(rng, base):
    return (np.rint(base) + rng.uniform(-0.5, 0.5, base.shape)).astype(np.float32)


def test_kde_rate_grad_matches_oracle(gc):
    rng = np.random.default_rng(14)
    n = 8011
    chans = [rng.normal(0, 0.3, n), rng.normal(5, 3.0, n), rng.normal(-100, 40.0, n),
             rng.gamma(1.5, 12.0, n), np.full(n, 3.0), rng.uniform(-300, -250, n)]
    y = np.stack([_noisy(rng, c) for c in chans])
    d_rate = np.array([1.0, 2.0, -0.5, 1.0, 3.0, 0.25], np.float32)
    r = gc.Renderer(0)
    rate, dy = r.kde_rate_grad(torch.from_numpy(y).cuda(), torch.from_numpy(d_rate).cuda())
    rate, dy = rate.cpu().numpy().astype(np.float64), dy.cpu().numpy().astype(np.float64)
    for c in range(len(chans)):
        yc = y[c].astype(np.float64)
        want_r = kr.rate_continuous(yc)
        want_g = d_rate[c] * kr.rate_continuous_grad(yc)
        assert abs(rate[c] - want_r) <= 2e-5 * max(abs(want_r), 1.0), (c, rate[c], want_r)
        scale = np.abs(want_g).max()
        assert np.abs(dy[c] - want_g).max() <= 1e-4 * scale, (c, np.abs(dy[c] - want_g).max(), scale)


def test_kde_rate_grad_on_integers_equals_symbol_rate(gc):
    rng = np.random.default_rng(15)
    y = np.stack([np.rint(rng.normal(0, s, 6007)) for s in (0.8, 7.0, 60.0)]).astype(np.float32)
    r = gc.Renderer(0)
    yd = torch.from_numpy(y).cuda()
    rate, dy = r.kde_rate_grad(yd)
    plain = r.kde_rate(yd)
    torch.cuda.synchronize()
    assert torch.allclose(rate, plain, rtol=2e-5, atol=2e-5)
    for c in range(3):
        want = kr.rate_continuous_grad(y[c].astype(np.float64))
        assert np.abs(dy[c].cpu().numpy() - want).max() <= 1e-4 * np.abs(want).max()


def test_kde_rate_grad_unsupported_and_rate_only(gc):
    rng = np.random.default_rng(16)
    y = np.stack([rng.uniform(0, 20000, 1000), rng.normal(0, 1, 1000), rng.normal(0, 1, 1000)]).astype(np.float32)
    y[2, 17] = np.nan
    r = gc.Renderer(0)
    rate, dy = r.kde_rate_grad(torch.from_numpy(y).cuda())
    rate, dy = rate.cpu().numpy(), dy.cpu().numpy()
    assert np.isnan(rate[0]) and np.isnan(rate[2])
    assert np.isnan(dy[0]).all() and np.isnan(dy[2]).all() and np.isfinite(dy[1]).all()
    r_only, none = r.kde_rate_grad(torch.from_numpy(y).cuda(), grad=False)
    assert none is None and float(r_only[1].cpu()) == float(rate[1])


def test_kde_rate_grad_of_noisy_attribute_planes(gc):
    """The paper's setting: uint8 attribute channels of a layer with injected noise."""
    rng = np.random.default_rng(17)
    scene = scenes.make_hier_scene(rng, 8000, 2, 3, 4)
    planes = scenes.quantize_planes(scene, plane_width=128)
    n0 = int(scene.layer_offsets[1])
    u8 = planes["u8"][0]
    base = u8[:, :, :128].reshape(u8.shape[0], -1)[:, :n0].astype(np.float64)[:6]
    y = (base + rng.uniform(-0.5, 0.5, base.shape)).astype(np.float32)
    r = gc.Renderer(0)
    rate, dy = r.kde_rate_grad(torch.from_numpy(np.ascontiguousarray(y)).cuda())
    rate, dy = rate.cpu().numpy().astype(np.float64), dy.cpu().numpy().astype(np.float64)
    for c in range(y.shape[0]):
        yc = y[c].astype(np.float64)
        assert abs(rate[c] - kr.rate_continuous(yc)) <= 2e-5 * max(kr.rate_continuous(yc), 1.0)
        want = kr.rate_continuous_grad(yc)
        assert np.abs(dy[c] - want).max() <= 1e-4 * np.abs(want).max()


@pytest.mark.parametrize("n", [1, 2, 2049])
def test_kde_rate_grad_edge_lengths(gc, n):
    """One value (h = 1), two values, and one value past a chunk of 2048."""
    rng = np.random.default_rng(100 + n)
    y = (np.rint(rng.normal(3.0, 4.0, (2, n))) + rng.uniform(-0.5, 0.5, (2, n))).astype(np.float32)
    r = gc.Renderer(0)
    rate, dy = r.kde_rate_grad(torch.from_numpy(y).cuda())
    rate, dy = rate.cpu().numpy().astype(np.float64), dy.cpu().numpy().astype(np.float64)
    for c in range(2):
        yc = y[c].astype(np.float64)
        want_r = kr.rate_continuous(yc)
        assert abs(rate[c] - want_r) <= 2e-5 * max(abs(want_r), 1.0), (n, c, rate[c], want_r)
        want_g = kr.rate_continuous_grad(yc)
        assert np.abs(dy[c] - want_g).max() <= 1e-4 * max(np.abs(want_g).max(), 1e-30), (n, c)
