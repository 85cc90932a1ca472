"""GPU decoding of the side information (Sec. 2.3) against the FP64
oracle: the piecewise-constant backward flow of a rectangular subdivision,
the intra mask of a subdivision of the plane and the residual mask points
of one subdivision per block.  Both are
integer and copy work, so the results must be identical; invalid trees are
reported and leave the output unwritten."""
import numpy as np
import pytest

import oracle
from gpu_util import hivc_module, to_np, torch_cuda
from workload.synth import _pack_bits, make_block_trees, make_flow_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


@pytest.mark.parametrize("W,H,n,seed", [(64, 48, 30, 0), (1920, 1080, 400, 1), (203, 77, 2000, 2), (1, 1, 1, 3),
                                        (37, 5, 185, 4)])
def test_flow_from_tree(hv, W, H, n, seed):
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    words, nbits, vals = make_flow_tree(rng, W, H, n)
    want = oracle.flow_from_tree(W, H, words, nbits, vals)
    flow = torch.full((H, W, 2), float("nan"), dtype=torch.float32, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    hv.flow_from_tree(W, H, _dev(torch, words), nbits, _dev(torch, vals), flow, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    assert np.array_equal(to_np(flow), want)


@pytest.mark.parametrize("W,H,B,lam,seed", [(256, 144, 16, 6.0, 0), (203, 77, 16, 8.0, 1), (50, 37, 8, 20.0, 2),
                                            (1920, 1080, 16, 8.0, 3)])
def test_masks_from_trees(hv, W, H, B, lam, seed):
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    words, nbits, tp = make_block_trees(rng, W, H, B, lam)
    bp_want, pos_want = oracle.masks_from_trees(W, H, B, words, tp)
    nb = len(tp) - 1
    bp = torch.zeros(nb + 1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(max(1, W * H), dtype=torch.uint8, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    hv.masks_from_trees(W, H, B, _dev(torch, words), _dev(torch, tp), bp, pos, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    assert np.array_equal(to_np(bp).view(np.uint32), bp_want)
    assert np.array_equal(to_np(pos)[:len(pos_want)], pos_want)


def test_invalid_trees_are_reported(hv):
    torch = torch_cuda()
    W, H = 4, 4
    flow = torch.full((H, W, 2), 7.0, dtype=torch.float32, device="cuda")
    vals = torch.zeros((3, 2), dtype=torch.float32, device="cuda")
    for bits in ([1, 0], [0, 0], [1, 0, 0]):  # too few bits, bits left over, 2 leaves for 3 values
        flags = torch.zeros(1, dtype=torch.int32, device="cuda")
        hv.flow_from_tree(W, H, _dev(torch, _pack_bits(bits)), len(bits), vals, flow, flags=flags)
        torch.cuda.synchronize()
        assert int(flags.item()) & (1 << 8), bits
        assert np.all(to_np(flow) == 7.0)
    # a one-pixel node that splits, in the second block
    words = _pack_bits([0] + [1, 0, 0] + [1, 1, 0, 1, 0, 0, 0])
    tp = np.array([0, 1, 4, 11], np.uint32)
    bp = torch.zeros(4, dtype=torch.int32, device="cuda")
    pos = torch.zeros(64, dtype=torch.uint8, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    hv.masks_from_trees(17, 1, 16, _dev(torch, words), _dev(torch, tp[:3]), bp[:3], pos, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) & (1 << 8)


@pytest.mark.parametrize("W,H,n,seed", [(64, 48, 30, 0), (1920, 1080, 62000, 1), (203, 77, 900, 2), (1, 1, 1, 3)])
def test_intra_mask_from_tree(hv, W, H, n, seed):
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    words, nbits, _ = make_flow_tree(rng, W, H, n)
    want = oracle.intra_mask_from_tree(W, H, words, nbits)
    idx = torch.zeros(W * H, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    hv.intra_mask_from_tree(W, H, _dev(torch, words), nbits, idx, cnt, flags=flags)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0 and int(cnt.item()) == len(want)
    assert np.array_equal(to_np(idx)[:len(want)].view(np.uint32), want)
    # too little room: nothing written, count 0, reported
    small = torch.full((max(1, len(want) - 1),), -1, dtype=torch.int32, device="cuda")
    if len(want) > 1:
        hv.intra_mask_from_tree(W, H, _dev(torch, words), nbits, small, cnt, flags=flags)
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0 and int(flags.item()) & (1 << 8)
        assert np.all(to_np(small) == -1)
