"""Pins of the oracle's colour path (Sec. 2.3): the 4:4:4 planes of the
reversible colour transform of JPEG2000 and the inverse transform of the
decoder's output.

Independent anchors:
* the forward transform, written here from its definition
  (Y = floor((R + 2G + B)/4), U = B - G, V = R - G), composed with the
  oracle's inverse is the identity on every corner of the RGB cube and on
  random colours;
* half-up rounding of the reconstructed planes before the transform and
  clamping of out-of-gamut results;
* the 4:4:4 decoder: chroma moves with the luma flow itself, U and V clamp
  at -255, zero flow and zero residual keep the reference.
"""
import numpy as np

import oracle
from workload import make_gop
from workload.synth import PFrame, empty_residual


def _forward(R, G, B):
    R, G, B = (np.asarray(x, np.int64) for x in (R, G, B))
    return np.floor_divide(R + 2 * G + B, 4), B - G, R - G


def test_inverse_rct_is_exact():
    rng = np.random.default_rng(0)
    corners = np.array([[r, g, b] for r in (0, 255) for g in (0, 255) for b in (0, 255)])
    rgb = np.concatenate([corners, rng.integers(0, 256, (200000, 3))]).T
    Y, U, V = _forward(*rgb)
    assert Y.min() >= 0 and Y.max() <= 255 and U.min() >= -255 and V.max() <= 255
    out = oracle.inverse_rct(*(x.reshape(1, -1).astype(np.float64) for x in (Y, U, V)))
    for k in range(3):
        assert np.array_equal(out[k].reshape(-1), rgb[k])


def test_inverse_rct_rounding_and_clamping():
    y = np.array([[10.5, 10.49, 0.0, 255.0]])
    u = np.array([[0.0, 0.0, 255.0, -255.0]])
    v = np.array([[-0.5, 0.49, 255.0, -255.0]])
    R, G, B = oracle.inverse_rct(y, u, v)
    # (11, 0, 0): G = 11 - floor(0/4) = 11;  (10, 0, 0): 10
    assert (G[0, 0], R[0, 0], B[0, 0]) == (11, 11, 11)
    assert (G[0, 1], R[0, 1], B[0, 1]) == (10, 10, 10)
    # Y 0, U = V = 255: G = -127 -> 0, R = B = 128
    assert (R[0, 2], G[0, 2], B[0, 2]) == (128, 0, 128)
    # Y 255, U = V = -255: G = 255 + 128 -> 255, R = B = 128
    assert (R[0, 3], G[0, 3], B[0, 3]) == (128, 255, 128)


def test_rct_decoder_moves_chroma_with_the_luma_flow():
    W, H = 48, 32
    gop = make_gop(3, W, H, n_frames=2, rct=True)
    dec = oracle.OracleDecoder(W, H, True, rct=True)
    rec0, _ = dec.decode_iframe(gop.iframe)
    flow = np.zeros((H, W, 2), np.float32)
    flow[..., 0] = 2.0  # pred(x, y) = ref(x + 2, y)
    zero = [empty_residual(W, H, 16) for _ in range(3)]
    rec1, rgb = dec.decode_pframe(PFrame(flow, zero))
    for p in range(3):
        assert rec1[p].shape == (H, W)
        assert np.array_equal(rec1[p][:, :W - 2], rec0[p][:, 2:])
    assert [x.shape for x in rgb] == [(H, W)] * 3
    assert np.array_equal(np.stack(rgb), np.stack(oracle.inverse_rct(*rec1)))
    # zero flow keeps the reference
    rec2, _ = dec.decode_pframe(PFrame(np.zeros((H, W, 2), np.float32), zero))
    for p in range(3):
        assert np.array_equal(rec2[p], rec1[p])


def test_rct_chroma_clamps_at_minus_255():
    W, H = 32, 16
    gop = make_gop(4, W, H, n_frames=2, rct=True)
    dec = oracle.OracleDecoder(W, H, True, rct=True)
    rec0, _ = dec.decode_iframe(gop.iframe)
    # one point per block at -255 below the prediction pulls U under -255
    res = [empty_residual(W, H, 16) for _ in range(3)]
    from workload import Residual
    bp = np.array([0, 1, 2], np.uint32)
    res[1] = Residual(W, H, 16, bp, np.array([0, 0], np.uint8), np.array([-32000, -32000], np.int16))
    rec1, _ = dec.decode_pframe(PFrame(np.zeros((H, W, 2), np.float32), res))
    assert rec1[1].min() == -255.0 and rec1[0].min() >= 0.0
