"""Pins of the oracle's reading of the paper's decoded attribute format (Sec. 3.4: uint16 /
uint32 positions, uint8 for every other attribute, each channel a 2D single-channel plane;
dequantised here by the per-layer, per-channel min / max affine map value = lo + code * step
in FP32).

* a hand-built two-layer example: codes placed by hand at (row, column) = (j // width,
  j % width) of each channel's plane, expected values worked out by hand;
* the end points of the map (code 0 is lo exactly; the top code is hi to FP32 rounding);
* quantising with the input generator and dequantising with the oracle (two independent
  implementations of the same affine map) reproduces every attribute within half a step;
* the row pitch of the planes (padding) does not change the result.
"""
import numpy as np

from synth import scenes


def _hand_scene():
    # 2 layers: 5 + 3 Gaussians, SH degree 0 (14 channels)
    n = 8
    return scenes.Scene(np.zeros((n, 3), np.float32), np.zeros((n, 3), np.float32), np.zeros((n, 4), np.float32),
                        np.zeros(n, np.float32), np.zeros((n, 1, 3), np.float32), np.zeros(n, np.int32),
                        np.array([0, 5, 8], np.int64), 0, 1)


def test_hand_built_planes(oracle_lib):
    sc = _hand_scene()
    W = 2
    rows = [3, 2]                     # ceil(5 / 2), ceil(3 / 2)
    pos = [np.zeros((3, r, 4), np.uint16) for r in rows]       # pitch 8 bytes = 4 uint16
    u8 = [np.zeros((11, r, 8), np.uint8) for r in rows]        # pitch 8 bytes
    dq = np.zeros((2, 14, 2), np.float32)
    dq[:, :, 1] = 1.0                                          # step 1, lo 0 unless set below
    # layer 0, Gaussian 3 -> row 1, column 1; Gaussian 4 -> row 2, column 0
    pos[0][0, 1, 1] = 7            # x of Gaussian 3
    dq[0, 0] = (1.0, 0.5)          # x = 1 + 7 * 0.5 = 4.5
    pos[0][2, 2, 0] = 65535        # z of Gaussian 4
    dq[0, 2] = (-2.0, 0.25)        # z = -2 + 65535 / 4 = 16381.75
    u8[0][10 - 3, 2, 0] = 200      # opacity logit of Gaussian 4 (channel 10)
    dq[0, 10] = (-4.0, 0.03125)    # -4 + 200 / 32 = 2.25
    # layer 1, Gaussian 2 (global 7) -> row 1, column 0
    u8[1][3 - 3, 1, 0] = 9         # quaternion w (channel 3)
    dq[1, 3] = (0.0, 0.125)        # 1.125
    u8[1][12 - 3, 1, 0] = 255      # SH coefficient 0, green (channel 11 + 1)
    dq[1, 12] = (-1.0, 0.0078125)  # -1 + 255 / 128 = 0.9921875
    # layer 1, Gaussian 1 (global 6) -> row 0, column 1: a log-scale
    u8[1][8 - 3, 0, 1] = 3         # log-scale y (channel 8)
    dq[1, 8] = (-5.0, 0.5)         # -3.5
    planes = {"plane_width": W, "pos_bits": 16, "pos": pos, "u8": u8, "dequant": dq}
    d = oracle_lib.dequantize_planes(planes, sc)
    assert d.means[3, 0] == np.float32(4.5)
    assert d.means[4, 2] == np.float32(16381.75)
    assert d.opacity_logits[4] == np.float32(2.25)
    assert d.quats[7, 0] == np.float32(1.125)
    assert d.sh[7, 0, 1] == np.float32(0.9921875)
    assert d.log_scales[6, 1] == np.float32(-3.5)
    # every other value is its channel's lo (code 0): 0 where lo was not set
    assert d.means[0, 0] == np.float32(1.0) and d.means[3, 1] == 0.0
    assert d.opacity_logits[0] == np.float32(-4.0) and d.opacity_logits[5] == 0.0


def test_end_points_and_round_trip(oracle_lib):
    rng = np.random.default_rng(3)
    sc = scenes.make_hier_scene(rng, 5000, 4, 3, 8)
    for bits in (16, 32):
        q = scenes.quantize_planes(sc, plane_width=96, pos_bits=bits)
        d = oracle_lib.dequantize_planes(q, sc)
        attrs = np.concatenate([sc.means, sc.quats, sc.log_scales, sc.opacity_logits[:, None],
                                sc.sh.reshape(sc.n, -1)], 1).astype(np.float64)
        deq = np.concatenate([d.means, d.quats, d.log_scales, d.opacity_logits[:, None],
                              d.sh.reshape(sc.n, -1)], 1).astype(np.float64)
        for l in range(sc.n_layers):
            a, b = sc.layer_offsets[l], sc.layer_offsets[l + 1]
            lo, step = q["dequant"][l, :, 0].astype(np.float64), q["dequant"][l, :, 1].astype(np.float64)
            # within half a step (+ the FP32 rounding of the product and the sum)
            slack = 0.5 * step + 4 * np.spacing(np.abs(attrs[a:b]).max(0).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(deq[a:b] - attrs[a:b]) <= slack[None, :]), (bits, l)
            # code 0 is lo exactly: the channel minimum is reproduced exactly
            assert np.all(deq[a:b].min(0) == lo), (bits, l)
            hi = attrs[a:b].max(0)
            assert np.all(np.abs(deq[a:b].max(0) - hi) <= 4 * np.spacing(np.abs(hi).astype(np.float32))), (bits, l)


def test_pitch_does_not_matter(oracle_lib):
    rng = np.random.default_rng(5)
    sc = scenes.make_hier_scene(rng, 2000, 3, 1, 4)
    a = oracle_lib.dequantize_planes(scenes.quantize_planes(sc, plane_width=50, pitch_align=1), sc)
    b = oracle_lib.dequantize_planes(scenes.quantize_planes(sc, plane_width=50, pitch_align=256), sc)
    for k in ("means", "quats", "log_scales", "opacity_logits", "sh"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
