"""GPU decoder parity against the FP64 oracle through the C ABI: intra
frames (Sec. 2.1), inter frames (Sec. 2, 2.3), GOPs with the closed
prediction loop, and the error paths (host-side and device-side)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_INTRA, TOL_PSNR_DB, TOL_RECON, hivc_module, psnr, to_np, torch_cuda
from workload import IFrame, PFrame, make_config1, make_gop, make_iframe_only, make_residual
from workload.synth import empty_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _planes(dec):
    return [to_np(dec.reference(p)).astype(np.float64) for p in range(3 if dec.chroma else 1)]


def test_iframe_config1(hv):
    src, ifr, _ = make_config1(0)
    dec = hv.Decoder(256, 144, chroma=False, iframe_tol=1e-8)
    out = hv.alloc_out(256, 144, chroma=False)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    st = dec.sync()
    assert st.resid[0] <= 1e-8
    gpu = _planes(dec)[0]
    u, _, _, _ = oracle.inpaint(256, 144, ifr.y_idx, ifr.y_val, 1e-12)
    assert np.abs(gpu - u).max() <= TOL_INTRA
    # mask pixels bit-exact, in the FP32 reference and in the uint8 output
    assert np.array_equal(gpu.reshape(-1)[ifr.y_idx], ifr.y_val.astype(np.float64))
    assert np.array_equal(to_np(out[0]).reshape(-1)[ifr.y_idx], ifr.y_val)
    assert np.array_equal(to_np(out[0]), oracle.to_uint8(u)) or np.abs(
        to_np(out[0]).astype(int) - oracle.to_uint8(u).astype(int)).max() <= 1


@pytest.mark.parametrize("W,H,frac,seed", [(203, 77, 0.05, 1), (64, 48, 0.01, 2), (1, 40, 0.2, 3), (37, 1, 0.2, 4)])
def test_iframe_color_ragged(hv, W, H, frac, seed):
    srcs, ifr = make_iframe_only(seed, W, H, frac, chroma=True)
    dec = hv.Decoder(W, H, chroma=True, iframe_tol=1e-9, max_cycles=200)
    out = hv.alloc_out(W, H)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    dec.sync()
    gpu = _planes(dec)
    od = oracle.OracleDecoder(W, H, True)
    rec, _ = od.decode_iframe(ifr)
    for p in range(3):
        assert np.abs(gpu[p] - rec[p]).max() <= TOL_INTRA, p
    assert np.array_equal(gpu[1].reshape(-1)[ifr.c_idx], ifr.cb_val.astype(np.float64))
    assert np.array_equal(gpu[2].reshape(-1)[ifr.c_idx], ifr.cr_val.astype(np.float64))


@pytest.mark.parametrize("W,H,cfrac,seed", [
    (480, 272, 0.0075, 11),  # chroma mask at a quarter of luma's: a long chroma phase
    (480, 272, 0.06, 12),    # chroma denser than luma: luma sweeps longest, the chroma loop stays empty
    (202, 150, 0.015, 13),   # ragged planes with chroma regions cut by the edges
])
def test_iframe_chroma_phase(hv, W, H, cfrac, seed):
    """4:2:0 solves run the launches that sweep only the chroma planes on
    regions of their own.  Whatever the split between the all-plane and the
    chroma phase, the result matches the oracle, and the graph the device
    steers gives the same bits as the same launches sent one by one from
    the host (per-kernel timing mode)."""
    srcs, ifr = make_iframe_only(seed, W, H, 0.03, chroma=True, chroma_mask_frac=cfrac)
    got = []
    for timing in (False, True):
        dec = hv.Decoder(W, H, chroma=True, iframe_tol=1e-9, timing=timing)
        out = hv.alloc_out(W, H)
        dec.decode_iframe(hv.device_iframe(ifr), out)
        st = dec.sync()
        got.append((_planes(dec), st.sweeps, st.cycles))
        dec.close()
    assert got[0][1:] == got[1][1:]
    for a, b in zip(got[0][0], got[1][0]):
        assert np.array_equal(a, b)
    od = oracle.OracleDecoder(W, H, True)
    rec, _ = od.decode_iframe(ifr)
    for p in range(3):
        assert np.abs(got[0][0][p] - rec[p]).max() <= TOL_INTRA, p


@pytest.mark.parametrize("W,H,chroma,seed", [(480, 272, True, 21), (202, 150, True, 22), (333, 97, False, 23)])
def test_coarse_start(hv, W, H, chroma, seed):
    """The default solve starts from a half-size solution prolonged to the
    unknown pixels; flat_start = 1 starts from the mean of the mask values.
    Only the start differs: both reach the tolerance and the oracle's
    solution, and the graph and the launches sent one by one from the host
    give the same bits with the coarse start."""
    srcs, ifr = make_iframe_only(seed, W, H, 0.03, chroma=chroma)
    rec, _ = oracle.OracleDecoder(W, H, chroma).decode_iframe(ifr)
    got = {}
    for flat, timing in ((0, False), (0, True), (1, False)):
        dec = hv.Decoder(W, H, chroma=chroma, iframe_tol=1e-9, flat_start=flat, timing=timing)
        out = hv.alloc_out(W, H, chroma=chroma)
        dec.decode_iframe(hv.device_iframe(ifr), out)
        st = dec.sync()
        assert max(st.resid) <= 1e-9
        got[(flat, timing)] = (_planes(dec), st.sweeps, st.cycles, st.kernel_launches[0], st.kernel_launches[7])
        dec.close()
    a, b = got[(0, False)], got[(0, True)]
    assert a[1:3] == b[1:3]
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    # the setup family holds the restriction and the prolongation
    assert got[(0, False)][3] == got[(1, False)][3] + 2
    # and the coarse sweeps are counted in a family of their own
    assert got[(0, False)][4] > 0 and got[(1, False)][4] == 0
    for flat in (0, 1):
        for p, g in enumerate(got[(flat, False)][0]):
            assert np.abs(g - rec[p]).max() <= TOL_INTRA, (flat, p)


def test_iframe_with_residual(hv):
    srcs, ifr = make_iframe_only(5, 160, 96, 0.03, chroma=True, residual={"lam_y": 8.0, "lam_c": 4.0})
    dec = hv.Decoder(160, 96, chroma=True)
    out = hv.alloc_out(160, 96)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    dec.sync()
    rec, _ = oracle.OracleDecoder(160, 96, True).decode_iframe(ifr)
    for p, g in enumerate(_planes(dec)):
        assert np.abs(g - rec[p]).max() <= TOL_RECON


def test_constant_intra_is_exact(hv):
    W, H = 50, 30
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(W * H, 20, replace=False)).astype(np.uint32)
    ifr = IFrame(W, H, False, idx, np.full(20, 131, np.uint8))
    dec = hv.Decoder(W, H, chroma=False)
    out = hv.alloc_out(W, H, chroma=False)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    st = dec.sync()
    assert st.cycles == 0
    assert np.all(_planes(dec)[0] == 131.0)


def test_grey_gop_with_large_blocks(hv):
    """Grey decoder, K up to 60 per block: warp and CTA coefficient paths."""
    gop = make_gop(4, 96, 64, n_frames=3, chroma=False, lam_y=30.0, residual_kw={"kmax": 60})
    dec = hv.Decoder(96, 64, chroma=False)
    out = hv.alloc_out(96, 64, chroma=False)
    frames = oracle.decode_gop(gop)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    for t in range(1, 3):
        dec.decode_pframe(hv.device_pframe(gop.pframes[t - 1]), out)
        dec.sync()
        assert np.abs(_planes(dec)[0] - frames[t][0][0]).max() <= TOL_RECON


def test_pframe_config1(hv):
    src, ifr, pfr = make_config1(0)
    dec = hv.Decoder(256, 144, chroma=False)
    out = hv.alloc_out(256, 144, chroma=False)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    dec.decode_pframe(hv.device_pframe(pfr), out)
    dec.sync()
    od = oracle.OracleDecoder(256, 144, False)
    od.decode_iframe(ifr)
    rec, o8 = od.decode_pframe(pfr)
    gpu = _planes(dec)[0]
    assert np.abs(gpu - rec[0]).max() <= TOL_RECON
    assert abs(psnr(gpu, src) - psnr(rec[0], src)) <= TOL_PSNR_DB
    assert np.abs(to_np(out[0]).astype(int) - o8[0].astype(int)).max() <= 1


def test_zero_flow_zero_residual_keeps_reference(hv):
    src, ifr, _ = make_config1(3, 64, 40)
    dec = hv.Decoder(64, 40, chroma=False)
    out = hv.alloc_out(64, 40, chroma=False)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    dec.sync()
    before = _planes(dec)[0]
    pfr = PFrame(np.zeros((40, 64, 2), np.float32), [empty_residual(64, 40, 16)])
    dec.decode_pframe(hv.device_pframe(pfr), out)
    dec.sync()
    assert np.array_equal(_planes(dec)[0], before)


@pytest.mark.parametrize("W,H,n,seed,B", [(160, 90, 8, 0, 16), (203, 77, 5, 1, 16), (150, 70, 4, 2, 8),
                                           (131, 67, 4, 3, 12)])
def test_small_color_gop(hv, W, H, n, seed, B):
    """Block sizes 16, 8 and 12 (edge blocks of every partial shape)."""
    gop = make_gop(seed, W, H, n_frames=n, block=B)
    dec = hv.Decoder(W, H, chroma=True, block=B)
    out = hv.alloc_out(W, H)
    frames = oracle.decode_gop(gop)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    for t in range(n):
        if t > 0:
            dec.decode_pframe(hv.device_pframe(gop.pframes[t - 1]), out)
        dec.sync()
        rec, o8 = frames[t]
        gpu = _planes(dec)
        for p in range(3):
            assert np.abs(gpu[p] - rec[p]).max() <= TOL_RECON, (t, p)
            assert abs(psnr(gpu[p], gop.sources[t][p]) - psnr(rec[p], gop.sources[t][p])) <= TOL_PSNR_DB
            assert np.abs(to_np(out[p]).astype(int) - o8[p].astype(int)).max() <= 1


@pytest.mark.parametrize("W,H", [(1, 40), (37, 1), (1, 1), (3, 3), (2, 5)])
def test_tiny_color_gop(hv, W, H):
    """Degenerate planes through the inter path: one pixel wide or tall
    (chroma 1 x 20, 19 x 1), a single pixel, odd 3 x 3 and 2 x 5 (chroma
    quads cut by the edge).  Per-frame decoding against the oracle, and the
    same GOP in one batch call equal to it bit for bit."""
    n = 3
    gop = make_gop(7, W, H, n_frames=n)
    frames = oracle.decode_gop(gop)
    dec = hv.Decoder(W, H, chroma=True)
    out = hv.alloc_out(W, H)
    per = []
    for t in range(n):
        if t == 0:
            dec.decode_iframe(hv.device_iframe(gop.iframe), out)
        else:
            dec.decode_pframe(hv.device_pframe(gop.pframes[t - 1]), out)
        dec.sync()
        rec, o8 = frames[t]
        gpu = _planes(dec)
        for p in range(3):
            assert np.abs(gpu[p] - rec[p]).max() <= TOL_RECON, (t, p)
            assert np.abs(to_np(out[p]).astype(int) - o8[p].astype(int)).max() <= 1, (t, p)
        per.append([to_np(o).copy() for o in out])
    dec2 = hv.Decoder(W, H, chroma=True)
    outs = [hv.alloc_out(W, H) for _ in range(n)]
    fr = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(pf)) for pf in gop.pframes]
    hv.decode_batch([dec2] * n, fr, outs)
    dec2.sync()
    for t in range(n):
        for p in range(3):
            assert np.array_equal(to_np(outs[t][p]), per[t][p]), (t, p)


@pytest.mark.parametrize("pre", [2, 6])
def test_batch_pool_sized_at_creation(hv, pre):
    """A decoder created with room for `pre` inter frames in its batch pool
    gives the same bits as one that grows its pool on demand: with 2 the
    4-frame batch outgrows it (stream-ordered growth), with 6 it fits."""
    W, H, n = 160, 96, 5
    gop = make_gop(8, W, H, n_frames=n)
    fr = [("i", hv.device_iframe(gop.iframe))] + [("p", hv.device_pframe(pf)) for pf in gop.pframes]
    got = []
    for kw in ({}, {"batch_frames": pre}):
        dec = hv.Decoder(W, H, chroma=True, **kw)
        outs = [hv.alloc_out(W, H) for _ in range(n)]
        hv.decode_batch([dec] * n, fr, outs)
        dec.sync()
        got.append([[to_np(o).copy() for o in out] for out in outs] + [_planes(dec)])
        dec.close()
    for a, b in zip(got[0], got[1]):
        for p in range(3):
            assert np.array_equal(a[p], b[p])


def test_fullhd_gop_head(hv):
    """Paper-scale frames (FullHD 4:2:0): the intra frame and two inter
    frames, every pixel against the oracle."""
    gop = make_gop(0, 1920, 1080, n_frames=3)
    dec = hv.Decoder(1920, 1080, chroma=True)
    out = hv.alloc_out(1920, 1080)
    od = oracle.OracleDecoder(1920, 1080, True)
    for t in range(3):
        if t == 0:
            dec.decode_iframe(hv.device_iframe(gop.iframe), out)
            rec, _ = od.decode_iframe(gop.iframe)
        else:
            dec.decode_pframe(hv.device_pframe(gop.pframes[t - 1]), out)
            rec, _ = od.decode_pframe(gop.pframes[t - 1])
        dec.sync()
        for p, g in enumerate(_planes(dec)):
            assert np.abs(g - rec[p]).max() <= TOL_RECON, (t, p)
            assert abs(psnr(g, gop.sources[t][p]) - psnr(rec[p], gop.sources[t][p])) <= TOL_PSNR_DB


# ---------------------------------------------------------------------------
# error paths: host checks return at once, device data checks surface at sync
# ---------------------------------------------------------------------------
def test_pframe_before_iframe(hv):
    dec = hv.Decoder(32, 32, chroma=False)
    out = hv.alloc_out(32, 32, chroma=False)
    pfr = PFrame(np.zeros((32, 32, 2), np.float32), [empty_residual(32, 32, 16)])
    with pytest.raises(hv.HivcError) as e:
        dec.decode_pframe(hv.device_pframe(pfr), out)
    assert e.value.status == hv.HIVC_E_NO_REFERENCE


def test_unsorted_mask_is_reported_at_sync(hv):
    W, H = 40, 30
    idx = np.array([5, 100, 99, 700], np.uint32)
    ifr = IFrame(W, H, False, idx, np.array([10, 20, 30, 40], np.uint8))
    dec = hv.Decoder(W, H, chroma=False)
    out = hv.alloc_out(W, H, chroma=False)
    dec.decode_iframe(hv.device_iframe(ifr), out, allow_not_converged=True)
    dec.sync(raise_on_error=False)
    assert dec.last_status == hv.HIVC_E_INVALID


def test_bad_block_data_is_reported_at_sync(hv):
    src, ifr, pfr = make_config1(0, 64, 48)
    bp = pfr.res[0].block_ptr.copy()
    bp[3] = bp[4] + 5  # decreasing block_ptr
    pfr.res[0].block_ptr = bp
    dec = hv.Decoder(64, 48, chroma=False)
    out = hv.alloc_out(64, 48, chroma=False)
    dec.decode_iframe(hv.device_iframe(ifr), out)
    dec.sync()
    dec.decode_pframe(hv.device_pframe(pfr), out)
    st = dec.sync(raise_on_error=False)
    assert dec.last_status == hv.HIVC_E_INVALID and st.device_flags != 0
    assert np.all(np.isfinite(_planes(dec)[0]))


def test_not_converged_with_cycle_cap(hv):
    srcs, ifr = make_iframe_only(2, 128, 96, 0.002)
    dec = hv.Decoder(128, 96, chroma=False, iframe_tol=1e-12, max_cycles=1)
    out = hv.alloc_out(128, 96, chroma=False)
    # the solve decides its cycles on the device: the call returns at once,
    # and the sync reports the cap
    assert dec.decode_iframe(hv.device_iframe(ifr), out) == hv.HIVC_OK
    stats = dec.sync(raise_on_error=False)
    assert dec.last_status == hv.HIVC_E_NOT_CONVERGED
    assert stats.cycles == 1 and stats.resid[0] > 1e-12
    # the next sync starts afresh
    dec.sync()


def test_invalid_arguments(hv):
    with pytest.raises(hv.HivcError):
        hv.Decoder(0, 10)
    with pytest.raises(hv.HivcError):
        hv.Decoder(64, 64, block=32)
    dec = hv.Decoder(32, 32, chroma=False)
    ifr = IFrame(32, 32, False, np.zeros(0, np.uint32), np.zeros(0, np.uint8))
    torch = torch_cuda()
    f = {"y_idx": torch.zeros(0, dtype=torch.int32, device="cuda"),
         "y_val": torch.zeros(0, dtype=torch.uint8, device="cuda")}
    with pytest.raises(hv.HivcError) as e:
        dec.decode_iframe(f, hv.alloc_out(32, 32, chroma=False))
    assert e.value.status == hv.HIVC_E_INVALID


def test_sor_tiling_choice_does_not_change_results(hv):
    """The first intra frame of a new plane geometry times both SOR region
    widths on real sweeps of its solve; later frames use the faster one.
    Both widths perform the same global red-black sweeps, so a frame decoded
    while tuning and one decoded after it are bit-identical."""
    W, H = 1000, 610  # a geometry no other test uses
    _, ifr = make_iframe_only(17, W, H, 0.02, chroma=True)
    got = []
    for _ in range(2):
        dec = hv.Decoder(W, H, chroma=True, iframe_tol=1e-9)
        out = hv.alloc_out(W, H)
        dec.decode_iframe(hv.device_iframe(ifr), out)
        st = dec.sync()
        got.append(([to_np(dec.reference(p)) for p in range(3)], st.sweeps))
    assert got[0][1] == got[1][1]
    for a, b in zip(got[0][0], got[1][0]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("batched", [False, True])
def test_inter_frames_in_a_cuda_graph(hv, batched):
    """An inter frame's launches (coefficients, residual planes, pixels; or the
    batch path's block launches and pixel kernels) can be captured in a CUDA
    graph on the decoder's stream: replaying the graph decodes the frame
    exactly as a direct call, and decoding goes on from its result."""
    torch = torch_cuda()
    W, H = 160, 96
    gop = make_gop(23, W, H, n_frames=4)
    frames = [hv.device_pframe(p) for p in gop.pframes]
    ref_dec = hv.Decoder(W, H, chroma=True)
    o = hv.alloc_out(W, H)
    ref_dec.decode_iframe(hv.device_iframe(gop.iframe), o)
    want = []
    for f in frames:
        ref_dec.decode_pframe(f, o)
        ref_dec.sync()
        want.append([to_np(p).copy() for p in o])
    s = torch.cuda.Stream()
    dec = hv.Decoder(W, H, chroma=True, stream=s)
    out = hv.alloc_out(W, H)
    dec.decode_iframe(hv.device_iframe(gop.iframe), out)
    run = (lambda f: hv.decode_batch([dec], [("p", f)], [out])) if batched else (lambda f: dec.decode_pframe(f, out))
    run(frames[0])  # first call: lazy per-device setup and the batch pool happen outside the capture
    dec.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        run(frames[1])
    g.replay()
    dec.sync()
    for p in range(3):
        assert np.array_equal(to_np(out[p]), want[1][p]), p
    run(frames[2])
    dec.sync()
    for p in range(3):
        assert np.array_equal(to_np(out[p]), want[2][p]), p


@pytest.mark.parametrize("W,H", [(700, 333), (300, 140), (90, 50), (3, 40)])
def test_sor_variants_are_bit_identical(hv, W, H):
    """Each pinned sweep variant (pairs of 128 or 112 columns, quads of 128)
    decodes an intra frame to the same bits, on planes with interior and
    edge regions, planes of one region and planes a few pixels wide."""
    _, ifr = make_iframe_only(19, W, H, 0.02 if W * H > 5000 else 0.1, chroma=True)
    got = []
    try:
        for v in (0, 1, 2):
            hv.check(hv.lib().hivc_set_sor_variant(v))
            dec = hv.Decoder(W, H, chroma=True, iframe_tol=1e-9)
            out = hv.alloc_out(W, H)
            dec.decode_iframe(hv.device_iframe(ifr), out)
            st = dec.sync()
            got.append(([to_np(dec.reference(p)) for p in range(3)], st.sweeps))
    finally:
        hv.lib().hivc_set_sor_variant(-1)
    for planes, sweeps in got[1:]:
        assert sweeps == got[0][1]
        for a, b in zip(planes, got[0][0]):
            assert np.array_equal(a, b)
    assert hv.lib().hivc_set_sor_variant(3) == hv.HIVC_E_INVALID
