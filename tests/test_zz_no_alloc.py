"""hivc_block_residual_static: the residual plane without any device
allocation, for callers that cannot allocate device memory when they need it
(a host whose memory budget is fully reserved at start-up, or a latency-bound
loop in which an allocation could synchronise the device).  It must give the
same plane as hivc_block_residual, which uses a caller workspace, on calls
made one after another (the second call reuses the library's scratch array
that the first one left behind), with or without a caller error word, and
on a call exactly at its limits; and calls after the first leave the
device's free memory unchanged.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from gpu_util import TOL_BLOCK, hivc_module, to_np, torch_cuda
from workload import make_residual

pytestmark = pytest.mark.gpu


def _with_workspace(hv, res):
    torch = torch_cuda()
    r = torch.zeros((res.height, res.width), dtype=torch.float32, device="cuda")
    bp, pos, val = hv.device_residual(res)
    hv.block_residual(res.width, res.height, res.block, bp, pos, val, r)
    torch.cuda.synchronize()
    return to_np(r)


def _without_allocation(hv, res, flags):
    torch = torch_cuda()
    r = torch.full((res.height, res.width), float("nan"), dtype=torch.float32, device="cuda")
    bp, pos, val = hv.device_residual(res)
    hv.block_residual_static(res.width, res.height, res.block, bp, pos, val, r, flags=flags)
    torch.cuda.synchronize()
    return to_np(r)


def test_matches_workspace_entry_point_on_consecutive_calls():
    hv = hivc_module()
    torch = torch_cuda()
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(21)
    first = make_residual(rng, 203, 77, 16, 8.0, 64, empty_frac=0.1)
    # the second call has blocks with K > 32 (solved by a whole CTA in its
    # range's scratch slot) on a different plane size
    second = make_residual(rng, 160, 96, 16, 30.0, 64, kmax=60)
    for res in (first, second):
        got = _without_allocation(hv, res, flags)
        ref = _with_workspace(hv, res)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_BLOCK
    assert int(flags.item()) == 0


def test_without_a_caller_error_word():
    """flags = NULL: the entry point clears its own error word inside the
    scratch array before its kernels run (two calls in a row, the first of
    them with bad block data that leaves bits in that word)."""
    hv = hivc_module()
    rng = np.random.default_rng(22)
    good = make_residual(rng, 131, 67, 16, 6.0, 64)
    bad = make_residual(rng, 131, 67, 16, 6.0, 64)
    bad.pos = bad.pos.copy()
    b = int(np.argmax(np.diff(bad.block_ptr.astype(np.int64)) >= 2))
    s = int(bad.block_ptr[b])
    bad.pos[s], bad.pos[s + 1] = bad.pos[s + 1], bad.pos[s]  # not increasing: that block reads as zero
    for res in (bad, good, good):
        got = _without_allocation(hv, res, None)
        ref = _with_workspace(hv, res)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_BLOCK


def test_device_memory_unchanged_around_calls():
    """After a first call (which loads the library's kernels and tables),
    further calls leave the device's free memory unchanged: no allocation
    by the library or by the runtime on its behalf."""
    hv = hivc_module()
    torch = torch_cuda()
    rng = np.random.default_rng(24)
    res = make_residual(rng, 320, 176, 16, 8.0, 64, kmax=48)
    bp, pos, val = hv.device_residual(res)
    r = torch.zeros((res.height, res.width), dtype=torch.float32, device="cuda")
    hv.block_residual_static(res.width, res.height, res.block, bp, pos, val, r)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        hv.block_residual_static(res.width, res.height, res.block, bp, pos, val, r)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.all(np.isfinite(to_np(r)))


def test_at_exactly_its_limits():
    """16384 blocks of 16 x 16 (a 2048 x 2048 plane) with 8 points each:
    131072 points, both limits reached and accepted."""
    hv = hivc_module()
    rng = np.random.default_rng(23)
    W = H = 2048
    nb = (W // 16) * (H // 16)
    keys = rng.random((nb, 256))
    pos = np.sort(np.argsort(keys, axis=1)[:, :8], axis=1).astype(np.uint8).reshape(-1)
    bp = (np.arange(nb + 1) * 8).astype(np.uint32)
    val = rng.integers(-64, 65, size=nb * 8).astype(np.int16)
    from workload.synth import Residual

    res = Residual(W, H, 16, bp, pos, val)
    assert res.n_points == 1 << 17 and res.n_blocks == 1 << 14
    got = _without_allocation(hv, res, None)
    ref = _with_workspace(hv, res)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= TOL_BLOCK


def test_rejects_inputs_beyond_its_limits():
    hv = hivc_module()
    torch = torch_cuda()
    W, H = 2048, 2048  # 16384 blocks of 16 x 16: at the limit
    n = 131073  # one point more than the limit
    bp = torch.zeros(128 * 128 + 1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(n, dtype=torch.uint8, device="cuda")
    val = torch.zeros(n, dtype=torch.int16, device="cuda")
    r = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    with pytest.raises(hv.HivcError) as e:
        hv.block_residual_static(W, H, 16, bp, pos, val, r)
    assert e.value.status == hv.HIVC_E_INVALID
    with pytest.raises(hv.HivcError) as e:
        hv.block_residual_static(W + 16, H, 16, bp, pos[:10], val[:10], r)  # 16512 blocks
    assert e.value.status == hv.HIVC_E_INVALID
