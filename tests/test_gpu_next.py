"""GPU parity of the next rows against the FP64 oracle: coefficient-mode
residual decoding (Sec. 2.2, 2.3: dequantise, then Eq. 3 without a solve)
and the biharmonic operator (Sec. 2.2: Green's eigenvalues 1/mu^2)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_PSNR_DB, TOL_RECON, hivc_module, psnr, to_np, torch_cuda
from workload import CoefResidual, make_coef_residual, make_gop

pytestmark = pytest.mark.gpu

# FP32 evaluation of Eq. 3 from FP32 Green's rows: each of the K <= 48 terms
# carries a relative rounding of a few 1e-7, so the error stays below 1e-5
# of the plane's largest magnitude
REL_EVAL = 1e-5


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("W,H,B,lam,step,seed", [(256, 144, 16, 8.0, 1.0, 0), (203, 77, 16, 20.0, 0.5, 1),
                                                 (37, 21, 8, 6.0, 2.0, 2), (150, 70, 5, 4.0, 0.25, 3)])
def test_coef_residual_plane(hv, op, W, H, B, lam, step, seed):
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    res = make_coef_residual(rng, W, H, B, lam, step=step, offset=0.375, kmax=48)
    want = oracle.block_residual_coef(res, op)
    r = torch.full((H, W + 3), float("nan"), dtype=torch.float32, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    hv.block_residual_coef(W, H, B, op, hv.device_coef_residual(res), r, flags=flags)  # pitch W + 3
    torch.cuda.synchronize()
    got = to_np(r[:, :W]).astype(np.float64)
    assert int(flags.item()) == 0
    assert np.abs(got - want).max() <= REL_EVAL * max(1.0, np.abs(want).max())
    assert np.isnan(to_np(r[:, W:])).all()  # nothing written beyond the plane


def test_coef_residual_special_cases(hv):
    """K = 0 gives r = a; an index -128 zeroes its block and is reported."""
    torch = torch_cuda()
    W = H = 32
    bp = np.array([0, 0, 2, 3, 3], np.uint32)
    pos = np.array([5, 9, 17], np.uint8)
    q = np.array([3, -128, 0], np.int8)
    a = np.array([1.5, -2.0, 4.0, 0.25], np.float32)
    res = CoefResidual(W, H, 16, bp, pos, q, a, step=1.0, offset=0.5)
    r = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    hv.block_residual_coef(W, H, 16, 0, hv.device_coef_residual(res), r, flags=flags)
    torch.cuda.synchronize()
    got = to_np(r)
    assert np.all(got[:16, :16] == 1.5)  # K = 0
    assert np.all(got[:16, 16:] == 0.0)  # index -128: zero block
    assert np.all(got[16:, 16:] == 0.25)  # K = 0
    assert int(flags.item()) & (1 << 7)
    ok = CoefResidual(W, H, 16, bp, pos, np.array([3, 1, 0], np.int8), a, step=1.0, offset=0.5)
    assert np.abs(got[16:, :16] - oracle.block_residual_coef(ok)[16:, :16]).max() <= 1e-4


@pytest.mark.parametrize("W,H,chroma,B,seed", [(160, 90, True, 16, 0), (131, 67, True, 16, 1), (96, 64, False, 8, 2)])
def test_coef_mode_gop(hv, W, H, chroma, B, seed):
    """A GOP whose inter frames carry coefficient-mode residuals (odd widths
    take the plain warp + add kernel, even ones the staged one)."""
    gop = make_gop(60 + seed, W, H, n_frames=5, chroma=chroma, block=B, coef_mode=True,
                   coef_kw={"step": 0.1, "offset": 0.5, "kmax": 48})
    recs = oracle.decode_gop(gop)
    dec = hv.Decoder(W, H, chroma=chroma, block=B)
    out = hv.alloc_out(W, H, chroma=chroma)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    for t, pf in enumerate(gop.pframes):
        dec.decode_pframe_coef(hv.device_pframe_coef(pf), out)
        dec.sync()
        rec = recs[t + 1][0]
        for p in range(3 if chroma else 1):
            g = to_np(dec.reference(p)).astype(np.float64)
            assert np.abs(g - rec[p]).max() <= TOL_RECON, (t, p)
            src = gop.sources[t + 1][p]
            assert abs(psnr(g, src) - psnr(rec[p], src)) <= TOL_PSNR_DB, (t, p)


@pytest.mark.parametrize("W,H,chroma,B,seed", [(160, 90, True, 16, 0), (96, 64, False, 8, 1)])
def test_biharmonic_gop(hv, W, H, chroma, B, seed):
    """Values-mode residuals with the biharmonic operator: per-frame and
    batched decoding agree bit for bit and follow the oracle."""
    gop = make_gop(70 + seed, W, H, n_frames=5, chroma=chroma, block=B)
    recs = oracle.decode_gop(gop, op=1)
    frames = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(p)) for p in gop.pframes]
    res = []
    for batched in (False, True):
        dec = hv.Decoder(W, H, chroma=chroma, block=B, op=1)
        outs = [hv.alloc_out(W, H, chroma=chroma) for _ in frames]
        if batched:
            hv.decode_batch([dec] * len(frames), frames, outs)
        else:
            for (k, f), o in zip(frames, outs):
                (dec.decode_iframe if k == "i" else dec.decode_pframe)(f, o)
        st = dec.sync()
        assert st.max_cond > 8.0  # the biharmonic bound uses the eigenvalue bound 64
        res.append(([[to_np(p) for p in o] for o in outs], [to_np(dec.reference(p)).astype(np.float64)
                                                           for p in range(3 if chroma else 1)]))
    for a, b in zip(res[0][0], res[1][0]):
        for p in range(len(a)):
            assert np.array_equal(a[p], b[p])
    rec = recs[-1][0]
    for p, g in enumerate(res[0][1]):
        assert np.abs(g - rec[p]).max() <= TOL_RECON, p
        src = gop.sources[-1][p]
        assert abs(psnr(g, src) - psnr(rec[p], src)) <= TOL_PSNR_DB, p
