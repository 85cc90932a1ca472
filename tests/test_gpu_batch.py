"""Batched decoding (hivc_decode_batch): the inter frames of a batch share
multi-frame coefficient and evaluation launches and run their pixel kernels
one after the other.  Every block is solved by the same arithmetic as in single-frame
decoding, so a batch must reproduce the per-frame path bit for bit, and
with it the FP64 oracle within the parity tolerance."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_PSNR_DB, TOL_RECON, hivc_module, psnr, to_np
from workload import make_gop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _planes(dec):
    return [to_np(dec.reference(p)).astype(np.float64) for p in range(3 if dec.chroma else 1)]


def _per_frame(hv, gop, W, H, chroma, B):
    """Reference planes and uint8 outputs after every frame, one call each."""
    dec = hv.Decoder(W, H, chroma=chroma, block=B)
    out = hv.alloc_out(W, H, chroma=chroma)
    refs, outs = [], []
    for t in range(len(gop.pframes) + 1):
        if t == 0:
            dec.decode_iframe(hv.device_iframe(gop.iframe), out)
        else:
            dec.decode_pframe(hv.device_pframe(gop.pframes[t - 1]), out)
        dec.sync()
        refs.append(_planes(dec))
        outs.append([to_np(o).copy() for o in out])
    return refs, outs


def _batched(hv, gop, W, H, chroma, B):
    """The whole GOP in one hivc_decode_batch call, one output per frame."""
    dec = hv.Decoder(W, H, chroma=chroma, block=B)
    n = len(gop.pframes) + 1
    outs = [hv.alloc_out(W, H, chroma=chroma) for _ in range(n)]
    frames = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(p)) for p in gop.pframes]
    hv.decode_batch([dec] * n, frames, outs)
    dec.sync()
    return dec, [[to_np(o).copy() for o in out] for out in outs]


@pytest.mark.parametrize("W,H,n,seed,B,chroma", [(160, 90, 12, 0, 16, True), (150, 70, 10, 2, 8, True),
                                                 (96, 64, 19, 4, 16, False), (131, 67, 5, 3, 12, True)])
def test_batch_matches_per_frame(hv, W, H, n, seed, B, chroma):
    """More inter frames than one coefficient launch takes (8 with chroma,
    16 grey) for B = 16 and 8; B = 12 decodes frame by frame."""
    gop = make_gop(seed, W, H, n_frames=n, block=B, chroma=chroma)
    refs, outs = _per_frame(hv, gop, W, H, chroma, B)
    dec, bouts = _batched(hv, gop, W, H, chroma, B)
    for t in range(n):
        for p in range(len(outs[t])):
            assert np.array_equal(bouts[t][p], outs[t][p]), (t, p)
    for p, g in enumerate(_planes(dec)):
        assert np.array_equal(g, refs[-1][p]), p
    # and the oracle, for the last frame
    rec, _ = oracle.decode_gop(gop)[-1]
    for p, g in enumerate(_planes(dec)):
        assert np.abs(g - rec[p]).max() <= TOL_RECON, p
        assert abs(psnr(g, gop.sources[-1][p]) - psnr(rec[p], gop.sources[-1][p])) <= TOL_PSNR_DB


@pytest.mark.parametrize("chroma,n", [(False, 6), (True, 11)])
def test_batch_with_large_blocks(hv, chroma, n):
    """Blocks with K > 32 are solved by a whole CTA in the scratch slot of
    their range: every range of a launch gets its own slot (with chroma 8
    frames share a launch)."""
    W, H = 128, 96
    gop = make_gop(5, W, H, n_frames=n, chroma=chroma, lam_y=30.0, lam_c=20.0, residual_kw={"kmax": 60})
    refs, outs = _per_frame(hv, gop, W, H, chroma, 16)
    dec, bouts = _batched(hv, gop, W, H, chroma, 16)
    for t in range(len(outs)):
        for p in range(len(outs[t])):
            assert np.array_equal(bouts[t][p], outs[t][p]), (t, p)
    for p, g in enumerate(_planes(dec)):
        assert np.array_equal(g, refs[-1][p]), p


def test_batch_two_decoders_interleaved(hv):
    """Frames of two decoders of different sizes interleaved in one batch:
    each decoder's frames stay in order and equal its own decoding."""
    ga = make_gop(6, 160, 90, n_frames=4)
    gb = make_gop(7, 96, 64, n_frames=5, chroma=False)
    ra, oa = _per_frame(hv, ga, 160, 90, True, 16)
    rb, ob = _per_frame(hv, gb, 96, 64, False, 16)
    da = hv.Decoder(160, 90, chroma=True)
    db = hv.Decoder(96, 64, chroma=False)
    decs, frames, outs, tags = [], [], [], []
    seq = [("a", 0), ("b", 0)] + [x for t in range(1, 5) for x in (("a", t), ("b", t)) if not (x[0] == "a" and t >= 4)]
    for who, t in seq:
        g, d, ch, (W, H) = (ga, da, True, (160, 90)) if who == "a" else (gb, db, False, (96, 64))
        decs.append(d)
        frames.append(("i", hv.device_iframe(g.iframe)) if t == 0 else ("p", hv.device_pframe(g.pframes[t - 1])))
        outs.append(hv.alloc_out(W, H, chroma=ch))
        tags.append((who, t))
    hv.decode_batch(decs, frames, outs)
    da.sync()
    db.sync()
    for (who, t), out in zip(tags, outs):
        ref = oa if who == "a" else ob
        for p, o in enumerate(out):
            assert np.array_equal(to_np(o), ref[t][p]), (who, t, p)
    for p, g in enumerate(_planes(da)):
        assert np.array_equal(g, ra[-1][p])
    assert np.array_equal(_planes(db)[0], rb[-1][0])


def _frame_list(hv, gops):
    """The frames of consecutive GOPs of one decoder, as (type, device frame)."""
    fr = []
    for g in gops:
        fr.append(("i", hv.device_iframe(g.iframe)))
        fr += [("p", hv.device_pframe(p)) for p in g.pframes]
    return fr


def _per_frame_list(hv, frames, W, H, chroma):
    """uint8 outputs after every frame of the list and the last reference planes,
    one call per frame."""
    dec = hv.Decoder(W, H, chroma=chroma)
    out = hv.alloc_out(W, H, chroma=chroma)
    outs = []
    for kind, f in frames:
        (dec.decode_iframe if kind == "i" else dec.decode_pframe)(f, out)
        dec.sync()
        outs.append([to_np(o).copy() for o in out])
    return outs, _planes(dec)


def test_batch_long_runs_two_decoders(hv):
    """Two GOPs of 13 frames back to back on one 4:2:0 decoder (each run
    needs two evaluation launches: the second waits for its intra frame and
    overlaps the first batch's pixel kernels) interleaved with a grey
    decoder's GOP of 21 frames (two launches of up to 16 jobs), all in one
    call: every output equals the decoder's own frame-by-frame decoding."""
    fa = _frame_list(hv, [make_gop(45, 160, 90, n_frames=13), make_gop(46, 160, 90, n_frames=13)])
    fb = _frame_list(hv, [make_gop(47, 96, 64, n_frames=21, chroma=False)])
    oa, ra = _per_frame_list(hv, fa, 160, 90, True)
    ob, rb = _per_frame_list(hv, fb, 96, 64, False)
    da = hv.Decoder(160, 90, chroma=True)
    db = hv.Decoder(96, 64, chroma=False)
    decs, frames, outs, tags = [], [], [], []
    for t in range(max(len(fa), len(fb))):
        for who, fl, d, ch, (W, H) in (("a", fa, da, True, (160, 90)), ("b", fb, db, False, (96, 64))):
            if t < len(fl):
                decs.append(d)
                frames.append(fl[t])
                outs.append(hv.alloc_out(W, H, chroma=ch))
                tags.append((who, t))
    hv.decode_batch(decs, frames, outs)
    da.sync()
    db.sync()
    for (who, t), out in zip(tags, outs):
        ref = oa if who == "a" else ob
        for p, o in enumerate(out):
            assert np.array_equal(to_np(o), ref[t][p]), (who, t, p)
    for p, g in enumerate(_planes(da)):
        assert np.array_equal(g, ra[p]), p
    assert np.array_equal(_planes(db)[0], rb[0])


def test_batch_rejects_a_bad_frame(hv):
    """An inter run is checked before any of it is launched: an output
    plane narrower than the frame makes the call fail with HIVC_E_INVALID."""
    W, H = 64, 48
    gop = make_gop(8, W, H, n_frames=3, chroma=False)
    dec = hv.Decoder(W, H, chroma=False)
    outs = [hv.alloc_out(W, H, chroma=False) for _ in range(2)] + [hv.alloc_out(W - 8, H, chroma=False)]
    frames = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(p)) for p in gop.pframes]
    with pytest.raises(hv.HivcError) as e:
        hv.decode_batch([dec] * 3, frames, outs)
    assert e.value.status == hv.HIVC_E_INVALID
    dec.sync()


def test_batch_many_decoders_with_intra_frames(hv):
    """Six decoders of mixed sizes, each an intra frame and inter frames, in
    one call: decoders with intra frames run on their own host threads; each
    must match its own per-frame decoding bit for bit."""
    specs = [(160, 90, True, 5), (96, 64, False, 4), (131, 67, True, 3), (64, 48, True, 6), (160, 90, True, 2),
             (150, 70, False, 5)]
    decs, frames, outs, tags, ref = [], [], [], [], []
    per = []
    for i, (W, H, ch, n) in enumerate(specs):
        g = make_gop(40 + i, W, H, n_frames=n, chroma=ch)
        ref.append(_per_frame(hv, g, W, H, ch, 16)[1])
        d = hv.Decoder(W, H, chroma=ch)
        per.append((d, [("i", hv.device_iframe(g.iframe))] + [("p", hv.device_pframe(p)) for p in g.pframes], W, H,
                    ch))
    # interleave the streams' frames (each stream's own order kept)
    t = 0
    while any(t < len(f) for _, f, _, _, _ in per):
        for i, (d, f, W, H, ch) in enumerate(per):
            if t < len(f):
                decs.append(d)
                frames.append(f[t])
                outs.append(hv.alloc_out(W, H, chroma=ch))
                tags.append((i, t))
        t += 1
    hv.decode_batch(decs, frames, outs)
    for d, *_ in per:
        d.sync()
    for (i, t), out in zip(tags, outs):
        for p, o in enumerate(out):
            assert np.array_equal(to_np(o), ref[i][t][p]), (i, t, p)


def test_batch_reference_rules(hv):
    """An inter frame needs a reference: the decoder's own, or an intra frame
    earlier in the same call; hivc_decoder_reset forgets it."""
    W, H = 64, 48
    g = make_gop(9, W, H, n_frames=3, chroma=False)
    fi = ("i", hv.device_iframe(g.iframe))
    fp = [("p", hv.device_pframe(p)) for p in g.pframes]
    o = lambda: hv.alloc_out(W, H, chroma=False)
    d1, d2 = hv.Decoder(W, H, chroma=False), hv.Decoder(W, H, chroma=False)
    with pytest.raises(hv.HivcError) as e:
        hv.decode_batch([d1, d2, d1], [fi, fp[0], fp[0]], [o(), o(), o()])
    assert e.value.status == hv.HIVC_E_NO_REFERENCE
    hv.decode_batch([d2, d1, d2], [fi, fi, fp[0]], [o(), o(), o()])
    hv.decode_batch([d1], [fp[0]], [o()])
    d1.reset()
    with pytest.raises(hv.HivcError) as e:
        hv.decode_batch([d1], [fp[1]], [o()])
    assert e.value.status == hv.HIVC_E_NO_REFERENCE
    with pytest.raises(hv.HivcError) as e:
        d1.decode_pframe(fp[1][1], o())
    assert e.value.status == hv.HIVC_E_NO_REFERENCE
    d1.sync()
    d2.sync()


@pytest.mark.parametrize("k,m", [(3, 6), (6, 2)])
def test_batch_two_gops_in_one_call(hv, k, m):
    """Two GOPs of one decoder in one call, [I P x k I P x m]: the block
    stage of each inter run overlaps its intra frame on a side stream, and the
    second run reuses the batch pool (grown when it is larger) only after the
    first run's pixel kernels.  Equal to decoding frame by frame."""
    W, H = 160, 90
    ga = make_gop(41, W, H, n_frames=k + 1)
    gb = make_gop(42, W, H, n_frames=m + 1)
    frames = []
    for g in (ga, gb):
        frames += [("i", hv.device_iframe(g.iframe))] + [("p", hv.device_pframe(p)) for p in g.pframes]
    dec = hv.Decoder(W, H)
    ref = []
    out = hv.alloc_out(W, H)
    for kind, f in frames:
        (dec.decode_iframe if kind == "i" else dec.decode_pframe)(f, out)
        dec.sync()
        ref.append([to_np(o).copy() for o in out])
    dec2 = hv.Decoder(W, H)
    outs = [hv.alloc_out(W, H) for _ in frames]
    hv.decode_batch([dec2] * len(frames), frames, outs)
    dec2.sync()
    for t, o in enumerate(outs):
        for p in range(3):
            assert np.array_equal(to_np(o[p]), ref[t][p]), (t, p)
