"""Pins of the oracle's side-information decoding (Sec. 2.3): rectangular
subdivision trees give the piecewise-constant backward flow (each region
its value) and the mask points of the residual blocks (leaf centres).

Independent anchors:
* a tree decoded by hand (tests/golden/subdivision_5x3.txt);
* invariants any correct decoder keeps: the leaves tile the rectangle
  exactly, a full binary tree has one more leaf than splits, a split halves
  the longer side;
* invalid streams (a split of a one-pixel node, too few bits) are refused;
* the flow is constant on each leaf and takes that leaf's value; the mask
  points are the leaf centres, increasing within each block.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from workload.synth import _pack_bits, make_block_trees, make_flow_tree


def _golden():
    _, tags = read_golden("subdivision_5x3.txt")
    assert tags["size"] == [[5, 3]]
    bits = [int(x) for x in tags["bits"][0]]
    leaves = np.array(tags["leaf"], np.int64)
    centres = [int(x) for x in tags["centres"][0]]
    return bits, leaves, centres


def test_hand_decoded_tree():
    bits, leaves, centres = _golden()
    got = oracle.tree_leaves(5, 3, _pack_bits(bits), len(bits))
    assert np.array_equal(got, leaves)
    tp = np.array([0, len(bits)], np.uint32)
    bp, pos = oracle.masks_from_trees(5, 3, 16, _pack_bits(bits), tp)
    assert list(bp) == [0, 4] and list(pos) == centres


@pytest.mark.parametrize("w,h,n,seed", [(64, 48, 30, 0), (1920, 1080, 400, 1), (16, 16, 255, 2), (7, 1, 7, 3)])
def test_leaves_tile_the_rectangle(w, h, n, seed):
    rng = np.random.default_rng(seed)
    words, nbits, vals = make_flow_tree(rng, w, h, n)
    leaves = oracle.tree_leaves(w, h, words, nbits)
    bits = [(int(words[i >> 5]) >> (i & 31)) & 1 for i in range(nbits)]
    assert len(leaves) == sum(bits) + 1 == len(vals)
    cover = np.zeros((h, w), np.int32)
    for x0, y0, lw, lh in leaves:
        assert lw >= 1 and lh >= 1
        cover[y0:y0 + lh, x0:x0 + lw] += 1
    assert np.all(cover == 1)
    # a split halves the longer side: every leaf has a sibling-compatible
    # size, i.e. its sides are ceil/floor halvings of the plane's sides
    for x0, y0, lw, lh in leaves:
        assert max(lw, lh) <= max(w, h)


def test_flow_is_the_leaf_value():
    rng = np.random.default_rng(4)
    words, nbits, vals = make_flow_tree(rng, 96, 64, 50)
    flow = oracle.flow_from_tree(96, 64, words, nbits, vals)
    for (x0, y0, lw, lh), v in zip(oracle.tree_leaves(96, 64, words, nbits), vals):
        assert np.all(flow[y0:y0 + lh, x0:x0 + lw] == v)


def test_block_masks_are_leaf_centres():
    rng = np.random.default_rng(5)
    W, H, B = 50, 37, 16
    words, nbits, tp = make_block_trees(rng, W, H, B, 6.0)
    bp, pos = oracle.masks_from_trees(W, H, B, words, tp)
    nbx = -(-W // B)
    for b in range(len(tp) - 1):
        w = min(B, W - (b % nbx) * B)
        h = min(B, H - (b // nbx) * B)
        sub = [(int(words[i >> 5]) >> (i & 31)) & 1 for i in range(int(tp[b]), int(tp[b + 1]))]
        leaves = oracle.tree_leaves(w, h, _pack_bits(sub), len(sub))
        want = sorted((y0 + (lh - 1) // 2) * w + x0 + (lw - 1) // 2 for x0, y0, lw, lh in leaves)
        got = list(pos[bp[b]:bp[b + 1]])
        assert got == want and all(a < c for a, c in zip(got, got[1:]))


def test_invalid_trees_are_refused():
    with pytest.raises(ValueError):  # a one-pixel node may not split
        oracle.tree_leaves(1, 1, _pack_bits([1, 0, 0]), 3)
    with pytest.raises(ValueError):  # bits run out
        oracle.tree_leaves(4, 4, _pack_bits([1, 0]), 2)
    with pytest.raises(ValueError):  # bits left over
        oracle.tree_leaves(4, 4, _pack_bits([0, 0]), 2)


def test_intra_mask_is_the_sorted_leaf_centres():
    """The intra mask of a plane's tree: one point per leaf, inside it, and
    the hand-decoded tree's centres as plane indices."""
    bits, leaves, centres = _golden()
    idx = oracle.intra_mask_from_tree(5, 3, _pack_bits(bits), len(bits))
    assert list(idx) == centres  # a 5-wide plane: block and plane indices agree
    rng = np.random.default_rng(6)
    W, H = 300, 170
    words, nbits, _ = make_flow_tree(rng, W, H, 1500)
    idx = oracle.intra_mask_from_tree(W, H, words, nbits)
    leaves = oracle.tree_leaves(W, H, words, nbits)
    assert len(idx) == len(leaves) and np.all(np.diff(idx.astype(np.int64)) > 0)
    owner = np.full(W * H, -1)
    for k, (x0, y0, lw, lh) in enumerate(leaves):
        owner.reshape(H, W)[y0:y0 + lh, x0:x0 + lw] = k
    assert sorted(owner[idx]) == list(range(len(leaves)))  # one point in every leaf
