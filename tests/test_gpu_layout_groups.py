"""Layout groups (Sec. 2.2, Eq. 3 for blocks that share one mask layout):
the blocks of a plane with the same points form a group when at least 16 of
them share the layout; one factorisation serves the group, and the residual
planes of all its blocks come from one tensor-core product R = V E^T.  The
result must match the FP64 oracle within the parity bar, agree with the
per-block path within the block tolerance, and stay bit-identical between
batched and per-frame decoding."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_BLOCK, TOL_PSNR_DB, TOL_RECON, hivc_module, psnr, to_np
from workload import make_gop

pytestmark = pytest.mark.gpu

SHARED = {"kmax": 48, "empty_frac": 0.1, "shared_layouts": 8, "shared_frac": 0.3}


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _planes(dec):
    return [to_np(dec.reference(p)).astype(np.float64) for p in range(3)]


def _decode(hv, gop, n, groups):
    W, H = gop.width, gop.height
    dec = hv.Decoder(W, H, chroma=True, layout_groups=groups)
    out = hv.alloc_out(W, H)
    got, stats = [], []
    for t in range(n):
        if t == 0:
            dec.decode_iframe(hv.device_iframe(gop.iframe), out)
        else:
            dec.decode_pframe(hv.device_pframe(gop.pframes[t - 1]), out)
        stats.append(dec.sync())
        got.append((_planes(dec), [to_np(o).copy() for o in out]))
    dec.close()
    return got, stats


@pytest.mark.parametrize("W,H,seed,formed", [(480, 272, 31, True), (203, 150, 32, False)])
def test_groups_against_oracle_and_per_block_path(hv, W, H, seed, formed):
    """480 x 272: about 19 blocks per shared layout, so groups form; 203 x
    150: about 4 per layout (ragged edges), so the blocks stay on their own."""
    n = 3
    gop = make_gop(seed, W, H, n_frames=n, residual_kw=SHARED)
    want = oracle.decode_gop(gop)
    on, st_on = _decode(hv, gop, n, True)
    off, st_off = _decode(hv, gop, n, False)
    # groups on the inter frames (8 shared luma layouts per frame)
    if formed:
        assert all(s.layout_groups > 0 and s.group_blocks >= 16 * s.layout_groups for s in st_on[1:])
    assert all(s.layout_groups == 0 and s.group_blocks == 0 for s in st_off)
    for t in range(n):
        rec, o8 = want[t]
        for p in range(3):
            g = on[t][0][p]
            assert np.abs(g - rec[p]).max() <= TOL_RECON, (t, p)
            assert abs(psnr(g, gop.sources[t][p]) - psnr(rec[p], gop.sources[t][p])) <= TOL_PSNR_DB
            assert np.abs(on[t][1][p].astype(int) - o8[p].astype(int)).max() <= 1
            # the product and the per-block solves differ by FP32 rounding only
            assert np.abs(g - off[t][0][p]).max() <= TOL_BLOCK, (t, p)


def test_groups_batch_equals_per_frame(hv):
    """640 x 352: about 33 luma blocks per shared layout and frame; a
    layout's group is formed per plane of a frame, so batching the frames
    forms the same groups and gives the same bits."""
    W, H, n = 640, 352, 5
    gop = make_gop(33, W, H, n_frames=n, residual_kw=SHARED)
    per, st_per = _decode(hv, gop, n, True)
    assert all(s.layout_groups > 0 for s in st_per[1:])
    dec = hv.Decoder(W, H, chroma=True, layout_groups=True)
    outs = [hv.alloc_out(W, H) for _ in range(n)]
    fr = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(p)) for p in gop.pframes]
    hv.decode_batch([dec] * n, fr, outs)
    st = dec.sync()
    assert st.layout_groups > 0
    for p in range(3):
        assert np.array_equal(_planes(dec)[p], per[-1][0][p]), p
    for t in range(n):
        for p in range(3):
            assert np.array_equal(to_np(outs[t][p]), per[t][1][p]), (t, p)


def test_groups_exact_at_the_points_and_zero_free(hv):
    """A single inter frame whose luma blocks all share one layout, with
    zero flow on a constant reference: the new reference minus the constant
    is the residual plane itself, which must equal the values at the points
    exactly (the unit rows of E) and the oracle's residual elsewhere."""
    W, H = 96, 64  # 24 full luma blocks on one layout
    gop = make_gop(34, W, H, n_frames=2, residual_kw={"shared_layouts": 1, "shared_frac": 1.0, "kmax": 12})
    ifr = gop.iframe
    ifr.y_val = np.full_like(ifr.y_val, 100)
    ifr.cb_val = np.full_like(ifr.cb_val, 100)
    ifr.cr_val = np.full_like(ifr.cr_val, 100)
    pf = gop.pframes[0]
    pf.flow = np.zeros_like(pf.flow)
    dec = hv.Decoder(W, H, chroma=True, layout_groups=True)
    out = hv.alloc_out(W, H)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    dec.decode_pframe(hv.device_pframe(pf), out)
    st = dec.sync()
    assert st.layout_groups >= 1 and st.group_blocks >= 16
    r = _planes(dec)[0] - 100.0
    res = pf.res[0]
    want = oracle.block_residual(res)
    assert np.abs(r - want).max() <= TOL_BLOCK
    bp = res.block_ptr.astype(np.int64)
    nbx = -(-W // 16)
    for b in range(res.n_blocks):
        by, bx = divmod(b, nbx)
        for j in range(bp[b], bp[b + 1]):
            y, x = divmod(int(res.pos[j]), 16)
            assert r[by * 16 + y, bx * 16 + x] == float(res.val[j])
    dec.close()


def test_layouts_the_product_cannot_take_stay_per_block(hv):
    """Layouts with K > 32 points, and blocks with values beyond +-256, are
    never grouped; their residual still matches the oracle."""
    W, H = 256, 160
    gop = make_gop(35, W, H, n_frames=2, lam_y=40.0, vmax=300,
                   residual_kw={"kmax": 48, "shared_layouts": 4, "shared_frac": 0.5})
    want = oracle.decode_gop(gop)
    got, st = _decode(hv, gop, 2, True)
    for p in range(3):
        assert np.abs(got[1][0][p] - want[1][0][p]).max() <= TOL_RECON, p
