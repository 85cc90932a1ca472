"""Host staging helpers of the binding (CPU): FramePack lays the inputs of
several frames out in one buffer and gives frame dicts whose arrays are views
of it; alloc_out_block gives the output planes of several frames as views of
one buffer.  Only the layout is tested here (no decoding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2008_10273_gb300 import hivc  # noqa: E402
from workload import make_gop  # noqa: E402


def _leaves(obj, out):
    hivc._map_tensors(obj, lambda t: out.append(t) or t)
    return out


def test_framepack_views_equal_inputs_and_keep_sharing():
    g = make_gop(3, 70, 45, n_frames=4)
    frames = [("i", hivc.device_iframe(g.iframe, "cpu"))]
    frames += [("p", hivc.device_pframe(p, "cpu")) for p in g.pframes]
    # a chroma layout shared by Cb and Cr, as device_pframe makes it when the
    # layouts are equal
    f = frames[1][1]
    f["res"][2] = (f["res"][1][0], f["res"][1][1], f["res"][2][2])
    pack = hivc.FramePack(frames, device="cpu")
    pack.upload()
    got = pack.frames()
    assert [k for k, _ in got] == [k for k, _ in frames]
    a, b = _leaves([f for _, f in frames], []), _leaves([f for _, f in got], [])
    assert len(a) == len(b)
    base = pack.device.data_ptr()
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape and torch.equal(x, y)
        assert (y.data_ptr() - base) % 256 == 0 and y.data_ptr() - base + y.numel() * y.element_size() <= pack.nbytes
    r = got[1][1]["res"]
    assert r[1][0].data_ptr() == r[2][0].data_ptr() and r[1][1].data_ptr() == r[2][1].data_ptr()
    assert r[1][2].data_ptr() != r[2][2].data_ptr()
    # every array once: the buffer holds the sum of the distinct arrays, padded
    distinct = {id(t): t for t in a}.values()
    assert pack.nbytes == sum(-(-t.numel() * t.element_size() // 256) * 256 for t in distinct)


@pytest.mark.parametrize("W,H,chroma", [(1920, 1080, True), (131, 67, True), (64, 48, False), (33, 17, 2)])
def test_out_block_planes_are_disjoint_views(W, H, chroma):
    n = 3
    buf, outs = hivc.alloc_out_block(n, W, H, chroma=chroma, device="cpu")
    ref = hivc.alloc_out(W, H, chroma=chroma, device="cpu")
    assert len(outs) == n
    spans = []
    for o in outs:
        assert [tuple(p.shape) for p in o] == [tuple(p.shape) for p in ref]
        for p in o:
            assert p.is_contiguous() and p.dtype == torch.uint8
            s = p.data_ptr() - buf.data_ptr()
            assert s % 256 == 0
            spans.append((s, s + p.numel()))
    spans.sort()
    assert all(e0 <= s1 for (_, e0), (s1, _) in zip(spans, spans[1:]))
    assert spans[-1][1] <= buf.numel()
    # writing a plane shows in the buffer at its place only
    buf.zero_()
    outs[1][0].fill_(7)
    assert int(buf.sum()) == 7 * outs[1][0].numel()
