"""Host logic of the serving loop on the CPU, with a fake device that
completes every decode at once: admission under the HBM budget (in order,
waiting for budget, refusing a stream larger than the whole budget),
continuous batching (at most per_stream consecutive arrived frames of each
admitted stream per call, frames of one stream in order), decoder pooling
(reuse per frame size, eviction for another size) and the result
bookkeeping."""
import pytest

from paper_2008_10273_gb300 import serve


class _Dec:
    def __init__(self, s, log):
        self.key = (s.width, s.height)
        self.resets = 0
        self.closed = False
        self.log = log

    def reset(self):
        self.resets += 1

    def sync(self):
        pass

    def close(self):
        self.closed = True
        self.log.append(("close", self.key))


class _Done:
    def query(self):
        return True


class FakeApi(serve.DeviceApi):
    def __init__(self):
        self.calls = []  # per call: [(decoder key, frame)]
        self.log = []

    def decoder(self, s):
        self.log.append(("create", (s.width, s.height)))
        return _Dec(s, self.log)

    def alloc_out(self, s):
        return object()

    def decode_batch(self, decs, frames, outs):
        self.calls.append([(d.key, f) for d, f in zip(decs, frames)])

    def decode_one(self, dec, frame, out):
        self.calls.append([(dec.key, frame)])

    def event_after(self, dec):
        return _Done()


def _stream(name, w, h, n, t0=0.0, dt=0.0):
    frames = [("i" if k % 30 == 0 else "p", (name, k)) for k in range(n)]
    return serve.Stream(name, w, h, frames, [t0 + k * dt for k in range(n)])


@pytest.fixture(autouse=True)
def _no_library_sizes(monkeypatch):
    # the decoder footprint is the library's host formula; keep this test
    # free of the native library
    monkeypatch.setattr(serve.hivc.Decoder, "bytes_for", staticmethod(lambda w, h, c, b: 4 * w * h))


def test_batches_keep_stream_order_and_limit():
    api = FakeApi()
    srv = serve.Server(1 << 40, per_stream=4, poll_s=1e-4, api=api)
    streams = [_stream("a", 64, 48, 10), _stream("b", 32, 16, 7)]
    st = srv.run(streams)
    assert st["frames"] == 17 and st["calls"] == len(api.calls)
    seen = {"a": -1, "b": -1}
    for call in api.calls:
        per = {}
        for key, (kind, (name, k)) in call:
            assert k == seen[name] + 1  # in order, no frame twice
            seen[name] = k
            per[name] = per.get(name, 0) + 1
        assert all(v <= 4 for v in per.values())
    assert seen == {"a": 9, "b": 6}
    assert st["decoders_created"] == 2 and st["max_active"] == 2


def test_admission_waits_for_budget_and_pools_decoders():
    api = FakeApi()
    need = serve.stream_budget_bytes(_stream("x", 64, 48, 1), 8)
    need_c = serve.stream_budget_bytes(_stream("y", 32, 16, 1), 8)
    srv = serve.Server(need + need_c - 1, per_stream=8, poll_s=1e-4, api=api)
    streams = [_stream("a", 64, 48, 5), _stream("b", 64, 48, 5), _stream("c", 32, 16, 5)]
    st = srv.run(streams)
    assert [n for n, _ in st["admitted"]] == ["a", "b", "c"]
    assert st["max_active"] == 1  # one stream fits at a time
    # b reuses a's decoder (same size, reset); c needs another size: a's pooled decoder is evicted
    assert [e for e in api.log if e[0] == "create"] == [("create", (64, 48)), ("create", (32, 16))]
    assert ("close", (64, 48)) in api.log
    assert srv.used <= srv.budget
    srv.close()
    assert srv.used == 0


def test_stream_larger_than_the_budget_is_refused():
    api = FakeApi()
    srv = serve.Server(1000, api=api)
    with pytest.raises(ValueError):
        srv.run([_stream("big", 64, 48, 3)])


def test_paced_arrivals_are_not_decoded_early():
    api = FakeApi()
    srv = serve.Server(1 << 40, per_stream=8, poll_s=1e-4, api=api)
    st = srv.run([_stream("a", 16, 16, 4, dt=0.01)])
    assert st["frames"] == 4 and st["calls"] >= 2  # the later frames had not arrived at the first call
    assert st["p50_ms"] >= 0.0 and st["p99_ms"] >= st["p50_ms"]
