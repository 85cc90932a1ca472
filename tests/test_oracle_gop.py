"""Pins of the oracle's frame/GOP composition (Sec. 2: one intra frame, then
inter frames predicted from the previous reconstruction, each corrected by
its block residual)."""
import numpy as np
import pytest

from workload import IFrame, PFrame, make_config1, make_gop
from workload.synth import empty_residual


def test_zero_flow_zero_residual_repeats_intra(oracle_lib):
    src, ifr, pfr = make_config1(0, 64, 48)
    dec = oracle_lib.OracleDecoder(64, 48, False)
    rec0, out0 = dec.decode_iframe(ifr)
    zero = PFrame(np.zeros((48, 64, 2), np.float32), [empty_residual(64, 48, 16)])
    for _ in range(3):
        rec, out = dec.decode_pframe(zero)
        assert np.array_equal(rec[0], rec0[0]) and np.array_equal(out[0], out0[0])


def test_integer_flow_chain_shifts(oracle_lib):
    src, ifr, _ = make_config1(1, 48, 32)
    dec = oracle_lib.OracleDecoder(48, 32, False)
    rec0, _ = dec.decode_iframe(ifr)
    flow = np.zeros((32, 48, 2), np.float32)
    flow[..., 0] = 2.0
    rec1, _ = dec.decode_pframe(PFrame(flow, [empty_residual(48, 32, 16)]))
    xs = np.minimum(np.arange(48) + 2, 47)
    assert np.array_equal(rec1[0], rec0[0][:, xs])


def test_constant_intra_plus_residual(oracle_lib):
    """A constant intra frame reconstructs exactly; a residual on top of a
    zero-flow prediction adds the block inpainting of the residual data."""
    W, H = 40, 24
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(W * H, 30, replace=False)).astype(np.uint32)
    ifr = IFrame(W, H, False, idx, np.full(30, 100, np.uint8))
    dec = oracle_lib.OracleDecoder(W, H, False)
    rec, out = dec.decode_iframe(ifr)
    assert np.all(rec[0] == 100.0) and np.all(out[0] == 100)
    from workload import make_residual
    res = make_residual(rng, W, H, 16, 6.0, 64)
    rec, out = dec.decode_pframe(PFrame(np.zeros((H, W, 2), np.float32), [res]))
    expect = np.clip(100.0 + oracle_lib.block_residual(res), 0, 255)
    assert np.abs(rec[0] - expect).max() == 0.0


def test_rounding_rule():
    import oracle

    x = np.array([-3.0, 0.49999, 0.5, 1.5, 254.5, 254.49, 300.0])
    assert list(oracle.to_uint8(x)) == [0, 0, 1, 2, 255, 254, 255]


def test_pframe_before_iframe_rejected(oracle_lib):
    dec = oracle_lib.OracleDecoder(16, 16, False)
    with pytest.raises(RuntimeError):
        dec.decode_pframe(PFrame(np.zeros((16, 16, 2), np.float32), [empty_residual(16, 16, 16)]))


def test_small_color_gop_runs(oracle_lib):
    gop = make_gop(0, 96, 54, n_frames=3, lam_y=4, lam_c=2)
    frames = oracle_lib.decode_gop(gop)
    assert len(frames) == 3
    for rec, out in frames:
        assert [p.shape for p in rec] == [(54, 96), (27, 48), (27, 48)]
        for p in rec:
            assert p.min() >= 0.0 and p.max() <= 255.0
    # intra mask pixels are reproduced exactly (Eq. 1)
    rec0 = frames[0][0]
    assert np.array_equal(rec0[0].reshape(-1)[gop.iframe.y_idx], gop.iframe.y_val.astype(float))
    assert np.array_equal(rec0[1].reshape(-1)[gop.iframe.c_idx], gop.iframe.cb_val.astype(float))
