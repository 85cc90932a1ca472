"""GPU parity of the single steps (C-ABI step entry points) against the FP64
oracle on the same seeded inputs: the backward warp (Sec. 2, 2.3) and the
block residual (Sec. 2.2, Eqs. 2-4)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_BLOCK, TOL_WARP, hivc_module, to_np, torch_cuda
from workload import make_config1, make_flow_sinusoids, make_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _warp_case(hv, W, H, flow, chroma=False, seed=0):
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    ref = rng.uniform(0, 255, (H, W)).astype(np.float32)
    r_d = torch.from_numpy(ref).cuda()
    f_d = torch.from_numpy(np.ascontiguousarray(flow, np.float32)).cuda()
    pred = torch.empty((H, W), dtype=torch.float32, device="cuda")
    hv.warp(r_d, f_d, pred, chroma_flow=chroma)
    torch.cuda.synchronize()
    if chroma:
        cf = oracle.chroma_flow(flow, W, H)
        expect = oracle.warp(ref.astype(np.float64), cf)
    else:
        expect = oracle.warp(ref.astype(np.float64), flow.astype(np.float64))
    return to_np(pred).astype(np.float64), expect, ref


def test_warp_zero_flow_is_bit_identity(hv):
    got, _, ref = _warp_case(hv, 203, 77, np.zeros((77, 203, 2), np.float32))
    assert np.array_equal(got, ref.astype(np.float64))


@pytest.mark.parametrize("W,H,vmax,seed", [(256, 144, 4.0, 0), (203, 77, 9.5, 1), (1, 9, 3.0, 2), (17, 1, 3.0, 3),
                                           (33, 31, 40.0, 4), (1920, 1080, 6.0, 5)])
def test_warp_vs_oracle(hv, W, H, vmax, seed):
    rng = np.random.default_rng(seed)
    flow = make_flow_sinusoids(rng, W, H, 3, vmax) if W > 1 and H > 1 else rng.uniform(-vmax, vmax, (H, W, 2))
    got, expect, _ = _warp_case(hv, W, H, flow.astype(np.float32), seed=seed)
    assert np.abs(got - expect).max() <= TOL_WARP


@pytest.mark.parametrize("LW,LH", [(256, 144), (203, 77), (9, 1), (1920, 1080)])
def test_warp_chroma_flow_vs_oracle(hv, LW, LH):
    rng = np.random.default_rng(LW)
    flow = (make_flow_sinusoids(rng, LW, LH, 3, 5.0) if LH > 1 else rng.uniform(-5, 5, (LH, LW, 2))).astype(np.float32)
    torch = torch_cuda()
    W, H = (LW + 1) // 2, (LH + 1) // 2
    ref = rng.uniform(0, 255, (H, W)).astype(np.float32)
    pred = torch.empty((H, W), dtype=torch.float32, device="cuda")
    hv.warp(torch.from_numpy(ref).cuda(), torch.from_numpy(flow).cuda(), pred, chroma_flow=True)
    torch.cuda.synchronize()
    expect = oracle.warp(ref.astype(np.float64), oracle.chroma_flow(flow, W, H))
    assert np.abs(to_np(pred) - expect).max() <= TOL_WARP


def _block_case(hv, res, pitch_extra=3):
    torch = torch_cuda()
    W, H = res.width, res.height
    r = torch.full((H, W + pitch_extra), float("nan"), dtype=torch.float32, device="cuda")
    rv = r[:, :W]
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    bp, pos, val = hv.device_residual(res)
    need = hv.lib().hivc_block_residual_workspace_bytes(W, H, res.block, res.n_points)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = hv.lib().hivc_block_residual(W, H, res.block, hv.ctypes.byref(hv.residual_struct(bp, pos, val)),
                                      rv.data_ptr(), r.stride(0), ws.data_ptr(), need, flags.data_ptr(), None)
    assert st == hv.HIVC_OK
    torch.cuda.synchronize()
    return to_np(rv).astype(np.float64), int(flags.item())


@pytest.mark.parametrize("W,H,B,lam,kmax,seed", [
    (256, 144, 16, 6.0, None, 0),    # tiny config
    (203, 77, 16, 8.0, None, 1),     # ragged edge blocks (11 x 16, 16 x 13, 11 x 13)
    (37, 21, 16, 5.0, None, 2),
    (120, 72, 8, 4.0, None, 3),      # the paper's 8 x 8 blocks
    (61, 29, 5, 3.0, None, 4),       # an odd block edge
    (160, 96, 16, 30.0, 48, 5),      # K up to 48: warp and CTA paths
])
def test_block_residual_vs_oracle(hv, W, H, B, lam, kmax, seed):
    rng = np.random.default_rng(seed)
    res = make_residual(rng, W, H, B, lam, 64 if B == 16 else 32, kmax=kmax, empty_frac=0.1)
    got, flags = _block_case(hv, res)
    assert flags == 0
    expect = oracle.block_residual(res)
    assert np.abs(got - expect).max() <= TOL_BLOCK
    # the data at the points, bit-exact
    nbx = -(-W // B)
    for b in range(res.n_blocks):
        lo, hi = res.block_ptr[b], res.block_ptr[b + 1]
        w = min(B, W - (b % nbx) * B)
        for j in range(lo, hi):
            y = (b // nbx) * B + res.pos[j] // w
            x = (b % nbx) * B + res.pos[j] % w
            assert got[y, x] == float(res.val[j])


def test_block_residual_dense_blocks(hv):
    """K up to w*h - 1 (255 on 16 x 16): the CTA path.  Near K = N the
    saddle matrix has condition ~ 1e5 (lambda_min >= (1 - K/N)/8), so FP32
    keeps ~0.1 grey level; the benchmark spec's bound 0.5 applies."""
    rng = np.random.default_rng(7)
    W, H = 64, 48
    res = make_residual(rng, W, H, 16, 400.0, 64)  # Poisson(400) clipped to w*h - 1
    got, flags = _block_case(hv, res)
    assert flags == 0
    assert np.abs(got - oracle.block_residual(res)).max() <= 0.5


def test_block_residual_bad_data_is_flagged_not_faulted(hv):
    torch = torch_cuda()
    rng = np.random.default_rng(8)
    res = make_residual(rng, 64, 32, 16, 6.0, 64)
    bad = res.pos.copy()
    k = np.diff(res.block_ptr.astype(np.int64))
    b = int(np.flatnonzero(k >= 2)[0])
    j = int(res.block_ptr[b])
    bad[j], bad[j + 1] = bad[j + 1], bad[j]  # positions no longer increasing
    res.pos = bad
    got, flags = _block_case(hv, res)
    assert flags != 0
    assert np.all(np.isfinite(got))
