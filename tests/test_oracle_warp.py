"""Pins of the oracle's inter prediction: backward warping along a dense
backward optic flow field (Sec. 2, Sec. 2.3), read as bilinear interpolation
with the sample position clamped to the plane, and the 4:2:0 chroma flow.
"""
import numpy as np
import pytest

from conftest import read_golden


def test_golden_bilinear_samples(oracle_lib):
    _, tags = read_golden("bilinear_2x2.txt")
    ref = np.array(tags["row"])
    for X, Y, expect in tags["sample"]:
        flow = np.zeros((2, 2, 2))
        flow[0, 0] = (X, Y)  # sample for output pixel (0, 0)
        pred = oracle_lib.warp(ref, flow)
        assert abs(pred[0, 0] - expect) < 1e-14


def test_zero_flow_is_identity(oracle_lib):
    rng = np.random.default_rng(0)
    ref = rng.uniform(0, 255, (19, 31))
    assert np.array_equal(oracle_lib.warp(ref, np.zeros((19, 31, 2))), ref)


@pytest.mark.parametrize("dx,dy", [(3, -2), (-5, 4), (0, 7), (40, 0)])
def test_integer_flow_is_clamped_shift(oracle_lib, dx, dy):
    rng = np.random.default_rng(1)
    H, W = 17, 23
    ref = rng.uniform(0, 255, (H, W))
    flow = np.zeros((H, W, 2))
    flow[..., 0], flow[..., 1] = dx, dy
    ys, xs = np.mgrid[0:H, 0:W]
    expect = ref[np.clip(ys + dy, 0, H - 1), np.clip(xs + dx, 0, W - 1)]
    assert np.abs(oracle_lib.warp(ref, flow) - expect).max() < 1e-12


def test_constant_and_linear_reference(oracle_lib):
    rng = np.random.default_rng(2)
    H, W = 15, 21
    flow = rng.uniform(-6, 6, (H, W, 2))
    assert np.abs(oracle_lib.warp(np.full((H, W), 42.5), flow) - 42.5).max() < 1e-12
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    ref = 3.0 + 2.0 * xs - 1.5 * ys
    X = np.clip(xs + flow[..., 0], 0, W - 1)
    Y = np.clip(ys + flow[..., 1], 0, H - 1)
    assert np.abs(oracle_lib.warp(ref, flow) - (3.0 + 2.0 * X - 1.5 * Y)).max() < 1e-11


def test_half_pixel_shift_is_mean(oracle_lib):
    rng = np.random.default_rng(3)
    ref = rng.uniform(0, 255, (9, 12))
    flow = np.zeros((9, 12, 2))
    flow[..., 0] = 0.5
    pred = oracle_lib.warp(ref, flow)
    assert np.abs(pred[:, :-1] - 0.5 * (ref[:, :-1] + ref[:, 1:])).max() < 1e-12
    assert np.abs(pred[:, -1] - ref[:, -1]).max() < 1e-12  # clamped at the right edge


def test_degenerate_sizes(oracle_lib):
    ref = np.arange(7, dtype=np.float64).reshape(1, 7)
    flow = np.zeros((1, 7, 2))
    flow[..., 0] = 1.25
    flow[..., 1] = 3.0
    pred = oracle_lib.warp(ref, flow)
    assert np.abs(pred[0] - np.minimum(np.arange(7) + 1.25, 6)).max() < 1e-12
    one = oracle_lib.warp(np.array([[9.0]]), np.full((1, 1, 2), -4.0))
    assert one[0, 0] == 9.0


@pytest.mark.parametrize("W,H", [(8, 6), (9, 7), (1, 1), (5, 2)])
def test_chroma_flow(oracle_lib, W, H):
    cw, ch = (W + 1) // 2, (H + 1) // 2
    flow = np.zeros((H, W, 2), np.float32)
    flow[..., 0], flow[..., 1] = 3.0, -1.0
    cf = oracle_lib.chroma_flow(flow, cw, ch)
    assert np.allclose(cf[..., 0], 1.5) and np.allclose(cf[..., 1], -0.5)
    rng = np.random.default_rng(W * 10 + H)
    flow = rng.uniform(-4, 4, (H, W, 2)).astype(np.float32)
    cf = oracle_lib.chroma_flow(flow, cw, ch)
    for j in range(ch):
        for i in range(cw):
            blk = flow[2 * j: 2 * j + 2, 2 * i: 2 * i + 2].reshape(-1, 2).astype(np.float64)
            assert np.allclose(cf[j, i], 0.5 * blk.mean(axis=0), atol=1e-12)
