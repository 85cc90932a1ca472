"""The fused inter-frame kernel (Sec. 2; Eq. 3 per block): the residual of
each 16 x 16 block is evaluated in shared memory from the block stage's
coefficients, then the block's pixels are warped, added, clamped and packed,
so no residual plane reaches memory.  It is opt-in (fused_residual) and
takes 4:2:0 and grey frames of even size with 16 x 16 blocks; the split
path (evaluation kernel into residual planes, then the pixel kernel) is
the default and takes every shape.  Both must give the same bits, per
frame and batched, and the fused frames must launch no evaluation
kernel."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_PSNR_DB, TOL_RECON, hivc_module, psnr, to_np
from workload import make_gop

pytestmark = pytest.mark.gpu

EVAL = 5  # hivc_stats kernel family of the evaluation kernel
DENSE = {"kmax": 48, "empty_frac": 0.1}


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _decode(hv, gop, chroma, fused, batch, shared_chroma=True, **kw):
    """Reference planes and uint8 outputs after every frame, and the
    evaluation launches of the inter frames."""
    W, H = gop.width, gop.height
    n = len(gop.pframes) + 1
    npl = 3 if chroma else 1
    dec = hv.Decoder(W, H, chroma=chroma, fused_residual=fused, **kw)
    fr = [("i", hv.device_iframe(gop.iframe))] + [
        ("p", hv.device_pframe(p, shared_chroma=shared_chroma)) for p in gop.pframes]
    if batch:
        outs = [hv.alloc_out(W, H, chroma=chroma) for _ in range(n)]
        hv.decode_batch([dec] * n, fr, outs)
        st = dec.sync()
        got = ([to_np(dec.reference(p)).copy() for p in range(npl)],
               [[to_np(o).copy() for o in out] for out in outs])
        dec.close()
        return got, st.kernel_launches[EVAL]
    out = hv.alloc_out(W, H, chroma=chroma)
    refs, outs, evals = [], [], 0
    dec.decode_iframe(fr[0][1], out)
    dec.sync()
    refs.append([to_np(dec.reference(p)).copy() for p in range(npl)])
    outs.append([to_np(o).copy() for o in out])
    for _, f in fr[1:]:
        dec.decode_pframe(f, out)
        evals += dec.sync().kernel_launches[EVAL]
        refs.append([to_np(dec.reference(p)).copy() for p in range(npl)])
        outs.append([to_np(o).copy() for o in out])
    dec.close()
    return (refs, outs), evals


@pytest.mark.parametrize("W,H,n,seed,chroma,kw", [
    (160, 96, 5, 40, True, {}),
    (854, 480, 3, 41, True, {}),       # luma width 2 mod 4, chroma width 427 (odd edge blocks)
    (202, 150, 4, 42, True, DENSE),    # K up to 48 (the coefficient kernel's CTA path), empty blocks
    (96, 64, 6, 43, False, {}),        # grey
    (18, 34, 3, 44, True, {}),         # one 2 x 3 macroblock grid with cropped blocks
])
def test_fused_equals_split(hv, W, H, n, seed, chroma, kw):
    gop = make_gop(seed, W, H, n_frames=n, chroma=chroma, residual_kw=kw or None)
    for batch in (False, True):
        fused, ev_f = _decode(hv, gop, chroma, True, batch)
        split, ev_s = _decode(hv, gop, chroma, False, batch)
        assert ev_f == 0 and ev_s > 0, (batch, ev_f, ev_s)
        if batch:
            for a, b in zip(fused[0], split[0]):
                assert np.array_equal(a, b)
            for fo, so in zip(fused[1], split[1]):
                for a, b in zip(fo, so):
                    assert np.array_equal(a, b)
        else:
            for t in range(n):
                for a, b in zip(fused[0][t], split[0][t]):
                    assert np.array_equal(a, b), (t, "ref")
                for a, b in zip(fused[1][t], split[1][t]):
                    assert np.array_equal(a, b), (t, "out")


def test_fused_against_the_oracle_with_separate_chroma_jobs(hv):
    """Cb and Cr handed over as separate arrays (two chroma jobs, each
    quarter evaluated twice) against the FP64 oracle, and equal to the
    paired jobs bit for bit."""
    W, H, n = 192, 112, 4
    gop = make_gop(45, W, H, n_frames=n)
    want = oracle.decode_gop(gop)
    sep, ev = _decode(hv, gop, True, True, False, shared_chroma=False)
    paired, _ = _decode(hv, gop, True, True, False, shared_chroma=True)
    assert ev == 0
    for t in range(n):
        rec, o8 = want[t]
        for p in range(3):
            g = sep[0][t][p].astype(np.float64)
            assert np.abs(g - rec[p]).max() <= TOL_RECON, (t, p)
            assert abs(psnr(g, gop.sources[t][p]) - psnr(rec[p], gop.sources[t][p])) <= TOL_PSNR_DB
            assert np.abs(sep[1][t][p].astype(int) - o8[p].astype(int)).max() <= 1
            assert np.array_equal(sep[0][t][p], paired[0][t][p])


def test_fused_bad_positions_give_a_zero_block_and_a_flag(hv):
    """A block whose positions are not increasing is reported at sync and
    reconstructs as the prediction alone, as on the split path."""
    W, H = 64, 48
    gop = make_gop(46, W, H, n_frames=2)
    pf = gop.pframes[0]
    r = pf.res[0]
    bp = r.block_ptr.astype(np.int64)
    b = next(k for k in range(len(bp) - 1) if bp[k + 1] - bp[k] >= 3)
    pos = r.pos.copy()
    pos[bp[b]], pos[bp[b] + 1] = pos[bp[b] + 1], pos[bp[b]]
    r.pos = pos
    got = []
    for fused in (True, False):
        dec = hv.Decoder(W, H, chroma=True, fused_residual=fused)
        out = hv.alloc_out(W, H)
        dec.decode_iframe(hv.device_iframe(gop.iframe), out)
        dec.sync()
        dec.decode_pframe(hv.device_pframe(pf), out)
        st = dec.sync(raise_on_error=False)
        assert dec.last_status == hv.HIVC_E_INVALID and st.device_flags != 0
        got.append([to_np(dec.reference(p)).copy() for p in range(3)])
        dec.close()
    for a, b2 in zip(*got):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b2)


def test_layout_groups_and_other_blocks_take_the_split_path(hv):
    """Layout groups need the residual planes, and so do blocks other than
    16 x 16: those frames launch the evaluation kernel even when the fused
    kernel is asked for; so does every frame by default."""
    W, H = 160, 96
    gop = make_gop(47, W, H, n_frames=2, block=8)
    dec = hv.Decoder(W, H, chroma=True, block=8, fused_residual=True)
    out = hv.alloc_out(W, H)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    dec.sync()
    dec.decode_pframe(hv.device_pframe(gop.pframes[0]), out)
    assert dec.sync().kernel_launches[EVAL] == 1
    dec.close()
    gop = make_gop(47, W, H, n_frames=2)
    for kw in ({"layout_groups": True, "fused_residual": True}, {}):
        dec = hv.Decoder(W, H, chroma=True, **kw)
        dec.decode_iframe(hv.device_iframe(gop.iframe), out)
        dec.sync()
        dec.decode_pframe(hv.device_pframe(gop.pframes[0]), out)
        assert dec.sync().kernel_launches[EVAL] == 1
        dec.close()
