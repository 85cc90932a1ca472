"""Serving loop: many concurrent video streams decoded as their frames arrive.

Each stream owns one decoder (its reference frames stay on the device) and
a queue of frames with arrival times.  The server admits streams, in order,
while their device bytes fit an HBM budget, and decodes with continuous
batching: every pass hands all frames that have arrived (up to
``per_stream`` consecutive frames of each admitted stream) to one
``hivc_decode_batch`` call.  Inter frames of a decoder share block launches,
and each decoder runs on its own stream, so the work of different streams
overlaps on the device.  A stream whose frames are all decoded leaves and
returns its decoder to an idle pool: a later stream of the same frame size
reuses it (reset, so its first frame must be an intra frame) without a new
allocation, and idle decoders are destroyed only when a stream of another
size needs their bytes.  The budget counts active and idle decoders.

A frame's latency is the time from its arrival to the moment the host sees
its decode complete (a CUDA event recorded after it on its decoder's
stream).  ``batched=False`` decodes the same arrivals with one call per
frame, earliest arrival first, for comparison (the plain path).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

from . import hivc


@dataclass
class Stream:
    """One video stream: frame size, frames (``('i' | 'p', device frame
    dict)``, decoded in order) and their arrival times in seconds from the
    start of the run."""

    name: str
    width: int
    height: int
    frames: Sequence
    arrivals: Sequence[float]
    chroma: bool = True
    block: int = 16
    iframe_tol: float = 1e-8
    keep_outputs: bool = False
    # state of a run
    decoder: Optional[hivc.Decoder] = None
    out: Optional[list] = None
    next_submit: int = 0
    done: int = 0
    budget_bytes: int = 0
    finish: List[float] = field(default_factory=list)
    outputs: Optional[List] = None
    pending: List = field(default_factory=list)  # (event, first frame, end frame)


def stream_budget_bytes(s: Stream, per_stream: int) -> int:
    """Device bytes a stream holds while admitted: its decoder plus the
    batch pool of ``per_stream`` inter frames (coefficients, block constants
    and residual planes of each; one launch's room for blocks with K > 32)."""
    w, h = s.width, s.height
    cw, ch = (w + 1) // 2, (h + 1) // 2
    pitch = lambda x: (x + 31) // 32 * 32
    planes = h * pitch(w) + (2 * ch * pitch(cw) if s.chroma else 0)
    nb = lambda a, b: -(-a // s.block) * -(-b // s.block)
    blocks = nb(w, h) + (2 * nb(cw, ch) if s.chroma else 0)
    per_frame = 4 * (planes + w * h + (cw * ch * 2 if s.chroma else 0) + 2 * blocks)
    scratch = -(-(16 * blocks) // 128) * 33408 * 4
    return hivc.Decoder.bytes_for(w, h, s.chroma, s.block) + per_stream * per_frame + scratch


class DeviceApi:
    """What the server needs of the device: decoders, output planes, decode
    calls and a completion event after a decoder's queued work (CUDA events
    recorded on the decoder's stream)."""

    def decoder(self, s: Stream):
        return hivc.Decoder(s.width, s.height, chroma=s.chroma, block=s.block, iframe_tol=s.iframe_tol)

    def alloc_out(self, s: Stream):
        return hivc.alloc_out(s.width, s.height, chroma=s.chroma)

    def decode_batch(self, decs, frames, outs):
        hivc.decode_batch(decs, frames, outs)

    def decode_one(self, dec, frame, out):
        kind, f = frame
        if kind == "i":
            dec.decode_iframe(f, out, allow_not_converged=True)
        else:
            dec.decode_pframe(f, out)

    def event_after(self, dec):
        import torch

        ev = torch.cuda.Event()
        ev.record(torch.cuda.ExternalStream(dec.stream_handle))
        return ev


class Server:
    """Continuous-batching decoder for many streams under an HBM budget.
    ``api`` supplies the device side (default :class:`DeviceApi`)."""

    def __init__(self, budget_bytes: int, per_stream: int = 8, max_frames_per_call: int = 256,
                 poll_s: float = 2e-4, api: Optional[DeviceApi] = None):
        self.api = api if api is not None else DeviceApi()
        self.budget = int(budget_bytes)
        self.per_stream = per_stream
        self.max_frames = max_frames_per_call
        self.poll = poll_s
        self.used = 0
        self.admit_log: List = []
        self.idle: dict = {}  # stream key -> [(decoder, budget bytes)]
        self.created = 0

    @staticmethod
    def _key(s: Stream):
        return (s.width, s.height, s.chroma, s.block, s.iframe_tol)

    def _evict_one(self) -> bool:
        for key, pool in self.idle.items():
            if pool:
                dec, nbytes = pool.pop()
                dec.close()
                self.used -= nbytes
                return True
        return False

    def _try_admit(self, s: Stream, now: float) -> bool:
        need = stream_budget_bytes(s, self.per_stream)
        pool = self.idle.get(self._key(s))
        if pool:
            s.decoder, need = pool.pop()
            s.decoder.reset()
        else:
            while self.used + need > self.budget and self._evict_one():
                pass
            if self.used + need > self.budget:
                return False
            s.decoder = self.api.decoder(s)
            self.created += 1
            self.used += need
        s.out = self.api.alloc_out(s)
        s.budget_bytes = need
        self.admit_log.append((s.name, round(now, 6)))
        return True

    def _release(self, s: Stream):
        s.decoder.sync()
        self.idle.setdefault(self._key(s), []).append((s.decoder, s.budget_bytes))
        s.decoder = None

    def close(self):
        """Destroy the idle decoders."""
        while self._evict_one():
            pass

    @staticmethod
    def _poll(s: Stream):
        while s.pending:
            ev, a, b = s.pending[0]
            if not ev.query():
                return
            t = time.perf_counter()
            for k in range(a, b):
                s.finish[k] = t
            s.done = b
            s.pending.pop(0)

    def _output(self, s: Stream):
        if not s.keep_outputs:
            return s.out
        o = self.api.alloc_out(s)
        s.outputs.append(o)
        return o

    def run(self, streams: Sequence[Stream], batched: bool = True) -> dict:
        """Decode every frame of every stream.  Returns throughput (FullHD
        frames/s over the wall time) and per-frame latency quantiles."""
        for s in streams:
            s.finish = [0.0] * len(s.frames)
            s.next_submit = s.done = 0
            s.pending = []
            s.outputs = [] if s.keep_outputs else None
        waiting = list(streams)
        active: List[Stream] = []
        self.admit_log = []
        created0 = self.created
        max_active = 0
        t0 = time.perf_counter()
        calls = 0
        while waiting or active:
            now = time.perf_counter() - t0
            while waiting and self._try_admit(waiting[0], now):
                active.append(waiting.pop(0))
            max_active = max(max_active, len(active))
            if waiting and not active:
                raise ValueError(f"stream {waiting[0].name} needs more than the whole budget "
                                 f"({stream_budget_bytes(waiting[0], self.per_stream)} > {self.budget} bytes)")
            decs, frames, outs, spans = [], [], [], []
            if batched:
                for s in active:
                    k = s.next_submit
                    while (k < len(s.frames) and s.arrivals[k] <= now and k - s.next_submit < self.per_stream
                           and len(frames) < self.max_frames):
                        decs.append(s.decoder)
                        frames.append(s.frames[k])
                        outs.append(self._output(s))
                        k += 1
                    if k > s.next_submit:
                        spans.append((s, s.next_submit, k))
                        s.next_submit = k
            else:
                ready = [s for s in active if s.next_submit < len(s.frames) and s.arrivals[s.next_submit] <= now]
                if ready:
                    s = min(ready, key=lambda x: x.arrivals[x.next_submit])
                    decs, frames, outs = [s.decoder], [s.frames[s.next_submit]], [self._output(s)]
                    spans.append((s, s.next_submit, s.next_submit + 1))
                    s.next_submit += 1
            if frames:
                if batched:
                    self.api.decode_batch(decs, frames, outs)
                else:
                    self.api.decode_one(decs[0], frames[0], outs[0])
                calls += 1
                for s, a, b in spans:
                    s.pending.append((self.api.event_after(s.decoder), a, b))
            for s in active:
                self._poll(s)
            for s in [x for x in active if x.done == len(x.frames)]:
                self._release(s)
                active.remove(s)
            if not frames:
                nxt = [s.arrivals[s.next_submit] for s in active if s.next_submit < len(s.frames)]
                wait = (min(nxt) - (time.perf_counter() - t0)) if nxt else self.poll
                if wait > 0:
                    time.sleep(min(wait, self.poll))
        wall = time.perf_counter() - t0
        lat, px = [], 0.0
        for s in streams:
            lat += [s.finish[k] - t0 - s.arrivals[k] for k in range(len(s.frames))]
            px += len(s.frames) * s.width * s.height
        lat.sort()
        q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
        return {"frames": len(lat), "wall_s": wall, "fullhd_fps": px / (1920 * 1080) / wall,
                "p50_ms": 1e3 * q(0.5), "p99_ms": 1e3 * q(0.99), "calls": calls,
                "admitted": list(self.admit_log), "decoders_created": self.created - created0,
                "max_active": max_active}
