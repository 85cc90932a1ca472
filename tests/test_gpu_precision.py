"""Precision workloads: intra frames solved to max |Lu| <= 1e-10 at 1%, 3%
and 8% masks (FP32 sweeps, float-float outer correction), and block
residuals on the clustered stress set (points of a block inside a 5 x 5
window), each against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_BLOCK, TOL_RECON, hivc_module, to_np, torch_cuda
from workload import make_gop, make_iframe_only, make_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


@pytest.mark.parametrize("frac", [0.01, 0.03, 0.08])
def test_intra_to_1e10(hv, frac):
    W, H = 480, 270
    _, ifr = make_iframe_only(11, W, H, frac, chroma=True)
    dec = hv.Decoder(W, H, chroma=True, iframe_tol=1e-10)
    out = hv.alloc_out(W, H)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    st = dec.sync()
    assert all(r <= 1e-10 for r in st.resid)
    rec, _ = oracle.OracleDecoder(W, H, True, iframe_tol=1e-10).decode_iframe(ifr)
    for p in range(3):
        g = to_np(dec.reference(p)).astype(np.float64)
        # the reference plane is FP32: the solve is as exact as the storage
        assert np.abs(g - rec[p]).max() <= 1e-4, p
        assert np.abs(g - rec[p]).max() <= TOL_RECON


@pytest.mark.parametrize("frac,seed", [(0.2, 12), (1.0, 13)])
def test_clustered_blocks(hv, frac, seed):
    """K <= 25 points inside a 5 x 5 window: G_PP stays far from singular
    (lambda_min >= (1 - K/N) / 8), so FP32 keeps the block bound."""
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    W, H = 256, 192
    res = make_residual(rng, W, H, 16, 8.0, 64, clustered_frac=frac, cluster_window=5, cluster_kmax=25)
    r = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    bp, pos, val = hv.device_residual(res)
    hv.block_residual(W, H, 16, bp, pos, val, r)
    torch.cuda.synchronize()
    assert np.abs(to_np(r).astype(np.float64) - oracle.block_residual(res)).max() <= TOL_BLOCK


def _block_stats(res_list, G_of):
    """Per-plane blocks: (non-empty count, K > 32 count, max cond_2, max
    bound 8 tr / (1 - K/N)) from the FP64 oracle's Green's matrices.  Cb and
    Cr share positions, so the chroma pair counts once."""
    n = large = 0
    cmax = bmax = 0.0
    for r in res_list:
        bp = r.block_ptr.astype(np.int64)
        nbx = -(-r.width // r.block)
        for b in range(len(bp) - 1):
            K = int(bp[b + 1] - bp[b])
            if K == 0:
                continue
            bx, by = b % nbx, b // nbx
            w = min(r.block, r.width - bx * r.block)
            h = min(r.block, r.height - by * r.block)
            P = r.pos[bp[b]:bp[b + 1]].astype(np.int64)
            A = G_of(w, h)[np.ix_(P, P)]
            ev = np.linalg.eigvalsh(A)
            n += 1
            large += K > 32
            cmax = max(cmax, ev[-1] / ev[0])
            bmax = max(bmax, 8 * np.trace(A) / (1 - K / (w * h)))
    return n, large, cmax, bmax


@pytest.mark.parametrize("residual_kw,lam", [({"clustered_frac": 0.2}, 8.0), ({"kmax": 60}, 30.0)])
def test_fp64_resolve(hv, residual_kw, lam):
    """cond_threshold = 0 re-solves every residual block in FP64 (shared
    memory for K <= 12, the range's slot otherwise); the default 1e6 none.
    Both stay within the parity bound, the statistics count the blocks, and
    the reported bound is at least every block's true condition number."""
    W, H = 128, 96
    gop = make_gop(31, W, H, n_frames=3, chroma=True, lam_y=lam, lam_c=lam / 2, residual_kw=residual_kw)
    recs = oracle.decode_gop(gop)
    cache = {}
    G_of = lambda w, h: cache.setdefault((w, h), oracle.green_matrix(w, h))
    outs = {}
    for thr in (1e6, 0.0):
        dec = hv.Decoder(W, H, chroma=True, cond_threshold=thr)
        out = hv.alloc_out(W, H)
        dec.decode_iframe(hv.device_iframe(gop.iframe), out)
        dec.sync()
        for t, pf in enumerate(gop.pframes):
            dec.decode_pframe(hv.device_pframe(pf), out)
            st = dec.sync()
            n, large, cmax, bmax = _block_stats(pf.res[:2], G_of)
            assert st.fp64_blocks == (n if thr == 0.0 else 0), (thr, t)
            assert st.large_blocks == large
            assert cmax * (1 - 1e-4) <= st.max_cond <= bmax * (1 + 1e-4), (cmax, st.max_cond, bmax)
            assert st.max_cond < 4e5
            rec = recs[t + 1][0]
            for p in range(3):
                g = to_np(dec.reference(p)).astype(np.float64)
                assert np.abs(g - rec[p]).max() <= TOL_RECON, (thr, t, p)
        outs[thr] = [to_np(dec.reference(p)).astype(np.float64) for p in range(3)]
    # the two precisions agree far inside the tolerance
    for p in range(3):
        assert np.abs(outs[0.0][p] - outs[1e6][p]).max() <= 1e-2


def test_fp64_resolve_batch_matches_per_frame(hv):
    """The batch path takes the same FP64 re-solves as per-frame decoding."""
    W, H = 96, 64
    gop = make_gop(32, W, H, n_frames=5, chroma=True, lam_y=20.0, lam_c=10.0, residual_kw={"kmax": 40})
    frames = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(p)) for p in gop.pframes]
    res = []
    for batched in (False, True):
        dec = hv.Decoder(W, H, chroma=True, cond_threshold=0.0)
        outs = [hv.alloc_out(W, H) for _ in frames]
        if batched:
            hv.decode_batch([dec] * len(frames), frames, outs)
        else:
            for (k, f), o in zip(frames, outs):
                (dec.decode_iframe if k == "i" else dec.decode_pframe)(f, o)
        st = dec.sync()
        assert st.fp64_blocks > 0
        res.append([[to_np(p) for p in o] for o in outs])
    for a, b in zip(*res):
        for p in range(3):
            assert np.array_equal(a[p], b[p])


def test_fullhd_precision_report():
    """The precision report at FullHD: every result within the parity bar
    (0.5 grey levels, 0.01 dB), intra residuals at 1e-10, mask pixels exact,
    no FP64 re-solve at the default threshold and all of them at 0."""
    from precision_report import precision_report

    hivc_module()
    rep = precision_report()
    for r in rep["intra"]:
        assert all(x <= 1e-10 for x in r["resid"]), r
        assert max(r["max_abs_err"]) <= TOL_RECON, r
        assert max(abs(d) for d in r["dpsnr_db"]) <= 0.01, r
        assert r["mask_exact"], r
    d, f = rep["blocks"]
    assert d["fp64_blocks"] == 0 and f["fp64_blocks"] > 0
    for r in rep["blocks"]:
        assert max(r["max_abs_err"]) <= TOL_RECON, r
        assert max(abs(x) for x in r["dpsnr_db"]) <= 0.01, r
