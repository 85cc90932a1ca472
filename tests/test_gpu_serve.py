"""Serving: streams of different sizes decoded with continuous batching as
their frames arrive.  Each stream's output must be the same decoded alone
and in the mix (batching reproduces per-frame decoding bit for bit), also
when the HBM budget admits one stream at a time."""
import numpy as np
import pytest

from gpu_util import hivc_module, to_np
from workload import make_gop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hv():
    return hivc_module()


def _streams(hv, serve, seed=0):
    rng = np.random.default_rng(seed)
    specs = [("a", 160, 90, True, 6), ("b", 96, 64, False, 5), ("c", 64, 48, True, 7), ("d", 131, 67, True, 4)]
    out = []
    for i, (name, W, H, ch, n) in enumerate(specs):
        g = make_gop(20 + i, W, H, n_frames=n, chroma=ch)
        frames = [("i", hv.device_iframe(g.iframe))] + [("p", hv.device_pframe(p)) for p in g.pframes]
        # 30 frames/s with exponential jitter (mean 3 ms), streams offset
        arr = 0.002 * i + np.arange(n) / 30.0 * 0.05 + rng.exponential(0.003, n)
        arr = np.maximum.accumulate(arr)
        out.append(serve.Stream(name, W, H, frames, list(arr), chroma=ch, keep_outputs=True))
    return out


def _alone(hv, s):
    dec = hv.Decoder(s.width, s.height, chroma=s.chroma)
    res = []
    for kind, f in s.frames:
        o = hv.alloc_out(s.width, s.height, chroma=s.chroma)
        if kind == "i":
            dec.decode_iframe(f, o)
        else:
            dec.decode_pframe(f, o)
        res.append(o)
    dec.sync()
    return [[to_np(p) for p in o] for o in res]


@pytest.mark.parametrize("budget_streams", [None, 1])
def test_mix_equals_alone(hv, budget_streams):
    from paper_2008_10273_gb300 import serve

    streams = _streams(hv, serve)
    need = max(serve.stream_budget_bytes(s, 8) for s in streams)
    budget = 1 << 40 if budget_streams is None else need + need // 2
    srv = serve.Server(budget)
    st = srv.run(streams)
    assert st["frames"] == sum(len(s.frames) for s in streams)
    if budget_streams == 1:
        # one stream at a time: each admission waits for the previous stream
        assert len(st["admitted"]) == len(streams)
        assert all(t2 >= t1 for (_, t1), (_, t2) in zip(st["admitted"], st["admitted"][1:]))
    for s in streams:
        ref = _alone(hv, s)
        got = [[to_np(p) for p in o] for o in s.outputs]
        for k, (a, b) in enumerate(zip(got, ref)):
            for p in range(len(a)):
                assert np.array_equal(a[p], b[p]), (s.name, k, p)
    assert st["p99_ms"] >= st["p50_ms"] >= 0


def test_plain_serving_matches(hv):
    from paper_2008_10273_gb300 import serve

    streams = _streams(hv, serve, seed=1)
    st = serve.Server(1 << 40).run(streams, batched=False)
    assert st["calls"] == sum(len(s.frames) for s in streams)
    for s in streams[:2]:
        ref = _alone(hv, s)
        for k, o in enumerate(s.outputs):
            for p, plane in enumerate(o):
                assert np.array_equal(to_np(plane), ref[k][p]), (s.name, k, p)


def test_stream_larger_than_budget_is_refused(hv):
    from paper_2008_10273_gb300 import serve

    streams = _streams(hv, serve)[:1]
    with pytest.raises(ValueError):
        serve.Server(1 << 20).run(streams)


def test_server_reuses_idle_decoders(hv):
    """A second run on the same server takes the idle decoders of the first
    (reset, no new allocation) and decodes the same frames identically."""
    from paper_2008_10273_gb300 import serve

    streams = _streams(hv, serve, seed=2)
    srv = serve.Server(1 << 40)
    st1 = srv.run(streams)
    first = [[[to_np(p).copy() for p in o] for o in s.outputs] for s in streams]
    st2 = srv.run(streams)
    assert st1["decoders_created"] == len(streams) and st2["decoders_created"] == 0
    for s, f in zip(streams, first):
        for k, o in enumerate(s.outputs):
            for p, plane in enumerate(o):
                assert np.array_equal(to_np(plane), f[k][p]), (s.name, k, p)
    srv.close()
    assert srv.used == 0
