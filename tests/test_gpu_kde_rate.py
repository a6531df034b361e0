"""The KDE rate estimate on the GPU (Sec. 3.3) against the FP64 oracle (oracle.kde_rate):
several channel shapes in one call (narrow and wide normals, a skewed gamma, a constant and a
negative-valued channel, a ragged length), the unsupported cases (a symbol span above 8192, a
non-finite value) reported as NaN, and the paper's setting: every quantised attribute channel
of a layer of 50k Gaussians (uint8 symbols)."""
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
