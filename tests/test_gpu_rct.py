"""GPU parity of the paper's colour path (Sec. 2.3): 4:4:4 planes of the
reversible colour transform decoded by the RCT pixel kernel, which also
packs R, G, B.  The FP32 references follow the FP64 oracle within the
parity bar; the packed colours are exactly the inverse RCT of the kernel's
own rounded references (the oracle's inverse applied to them)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_PSNR_DB, TOL_RECON, hivc_module, psnr, to_np
from workload import make_gop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _check(dec, out, rec, srcs):
    g = [to_np(dec.reference(p)).astype(np.float64) for p in range(3)]
    for p in range(3):
        assert np.abs(g[p] - rec[p]).max() <= TOL_RECON, p
        assert abs(psnr(g[p], srcs[p]) - psnr(rec[p], srcs[p])) <= TOL_PSNR_DB, p
    # the pack is the inverse RCT of the kernel's own references
    want = oracle.inverse_rct(*g)
    for p in range(3):
        assert np.array_equal(to_np(out[p]), want[p]), p
    assert g[1].min() >= -255.0 and g[0].min() >= 0.0


def _psnr_src(srcs):
    return [s.astype(np.float64) for s in srcs]


@pytest.mark.parametrize("W,H,B,seed", [(160, 90, 16, 0), (131, 67, 16, 1), (96, 64, 8, 2)])
def test_rct_gop(hv, W, H, B, seed):
    gop = make_gop(80 + seed, W, H, n_frames=5, block=B, rct=True)
    recs = oracle.decode_gop(gop)
    dec = hv.Decoder(W, H, chroma=2, block=B)
    out = hv.alloc_out(W, H, chroma=2)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    dec.sync()
    _check(dec, out, recs[0][0], _psnr_src(gop.sources[0]))
    for t, pf in enumerate(gop.pframes):
        dec.decode_pframe(hv.device_pframe(pf), out)
        dec.sync()
        _check(dec, out, recs[t + 1][0], _psnr_src(gop.sources[t + 1]))


def test_rct_coef_mode_and_batch(hv):
    """Coefficient-mode inter frames on the colour path, and a values-mode
    GOP through hivc_decode_batch equal to its per-frame decoding."""
    W, H = 128, 72
    gop = make_gop(90, W, H, n_frames=4, rct=True, coef_mode=True, coef_kw={"step": 0.1, "kmax": 48})
    recs = oracle.decode_gop(gop)
    dec = hv.Decoder(W, H, chroma=2)
    out = hv.alloc_out(W, H, chroma=2)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    for t, pf in enumerate(gop.pframes):
        dec.decode_pframe_coef(hv.device_pframe_coef(pf), out)
        dec.sync()
        _check(dec, out, recs[t + 1][0], _psnr_src(gop.sources[t + 1]))
    g2 = make_gop(91, W, H, n_frames=4, rct=True)
    frames = [("i", hv.device_iframe(g2.iframe))] + [("p", hv.device_pframe(p)) for p in g2.pframes]
    res = []
    for batched in (False, True):
        d = hv.Decoder(W, H, chroma=2)
        outs = [hv.alloc_out(W, H, chroma=2) for _ in frames]
        if batched:
            hv.decode_batch([d] * len(frames), frames, outs)
        else:
            for (k, f), o in zip(frames, outs):
                (d.decode_iframe if k == "i" else d.decode_pframe)(f, o)
        d.sync()
        res.append([[to_np(p) for p in o] for o in outs])
    for a, b in zip(*res):
        for p in range(3):
            assert np.array_equal(a[p], b[p])
