"""The L1 photometric loss of the differentiation workload (gc_l1_loss): against the plain
definition in FP64 - loss = scale * sum |image - target|, gradient scale * sign(image -
target) with sign(0) = 0 - on an aligned 1352x1014 image, a ragged length with
unaligned pointers, exact ties and the empty case; the sum is deterministic."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r():
    import paper_2509_17513_b300 as gc
    rr = gc.Renderer(0)
    yield rr
    rr.close()


def _check(r, img, tgt, scale):
    loss, grad = r.l1_loss(img, tgt, scale=scale)
    torch.cuda.synchronize()
    a = img.double().cpu().numpy()
    b = tgt.double().cpu().numpy()
    d = img.cpu().numpy() - tgt.cpu().numpy()      # the FP32 difference the kernel takes
    want = scale * np.abs(d.astype(np.float64)).sum()
    assert abs(float(loss) - want) <= 1e-6 * max(abs(want), 1e-30), (float(loss), want)
    g = grad.cpu().numpy()
    assert np.array_equal(g, (np.float32(scale) * np.sign(d)).astype(np.float32))
    assert not np.any(g[a == b])                    # sign(0) = 0
    return loss, grad


def test_l1_loss_matches_definition(r):
    gen = torch.Generator(device="cuda").manual_seed(1)
    img = torch.rand((3, 1014, 1352), generator=gen, device="cuda")
    tgt = torch.rand((3, 1014, 1352), generator=gen, device="cuda")
    tgt[:, ::7, ::5] = img[:, ::7, ::5]            # exact ties
    l1, g1 = _check(r, img, tgt, 1.0 / img.numel())
    l2, g2 = _check(r, img, tgt, 1.0 / img.numel())
    assert torch.equal(l1, l2) and torch.equal(g1, g2)  # deterministic


def test_l1_loss_ragged_unaligned_and_empty(r):
    gen = torch.Generator(device="cuda").manual_seed(2)
    base = torch.rand(100003, generator=gen, device="cuda")
    other = torch.rand(100003, generator=gen, device="cuda")
    img, tgt = base[1:], other[1:]                 # 4-byte offset: the scalar path
    _check(r, img, tgt, 0.5)
    _check(r, base[:13], other[:13], 2.0)
    e = torch.empty(0, device="cuda")
    loss, grad = r.l1_loss(e, e, scale=1.0)
    torch.cuda.synchronize()
    assert float(loss) == 0.0 and grad.numel() == 0
