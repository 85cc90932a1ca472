"""The seeded input generator: determinism and the structural invariants the
decoder's input contract requires (sorted unique positions, K <= w*h - 1)."""
import numpy as np

from workload import block_grid, make_config1, make_gop, make_residual


def _check_residual(res):
    nbx, nby, w, h = block_grid(res.width, res.height, res.block)
    assert res.block_ptr.shape[0] == nbx * nby + 1 and res.block_ptr[0] == 0
    k = np.diff(res.block_ptr.astype(np.int64))
    assert np.all(k >= 0) and np.all(k <= w * h - 1)
    for b in range(nbx * nby):
        p = res.pos[res.block_ptr[b]: res.block_ptr[b + 1]].astype(int)
        assert np.all(np.diff(p) > 0) and np.all(p < w[b] * h[b])


def test_config1_deterministic():
    a = make_config1(7)
    b = make_config1(7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2].flow, b[2].flow)
    assert np.array_equal(a[2].res[0].pos, b[2].res[0].pos)
    src, ifr, pfr = a
    assert src.shape == (144, 256) and ifr.y_idx.size == round(0.04 * 256 * 144)
    assert np.all(np.diff(ifr.y_idx.astype(np.int64)) > 0)
    assert np.abs(pfr.flow).max() <= 4.0 + 1e-5
    _check_residual(pfr.res[0])


def test_residual_variants():
    rng = np.random.default_rng(0)
    for kw in ({}, {"kmax": 48, "empty_frac": 0.1, "shared_layouts": 8, "shared_frac": 0.3},
               {"clustered_frac": 0.2}):
        res = make_residual(rng, 203, 77, 16, 8.0, 64, **kw)
        _check_residual(res)
        assert res.val.min() >= -64 and res.val.max() <= 64


def test_gop_shapes_and_shared_chroma_layout():
    gop = make_gop(1, 130, 70, n_frames=3)
    assert gop.n_frames == 3
    y, cb, cr = gop.pframes[0].res
    assert (cb.width, cb.height) == (65, 35)
    assert np.array_equal(cb.pos, cr.pos) and np.array_equal(cb.block_ptr, cr.block_ptr)
    for r in (y, cb, cr):
        _check_residual(r)
    assert gop.pframes[0].flow.shape == (70, 130, 2)
