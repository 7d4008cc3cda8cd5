"""The request loop's scheduling rules, on the CPU with a fake device whose
frames take a fixed time on a per-stream queue, and a simulated clock."""
import numpy as np
import pytest

from paper_1809_07986_gb300.serving import Backend, StreamSpec, poisson_arrivals, serve


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def idle(self, s):
        self.t += max(s, 1e-4)


class FakeDevice(Backend):
    """Each stream is a FIFO queue; a frame takes `service` seconds."""

    def __init__(self, clock, service):
        self.clock, self.service = clock, service
        self.busy, self.opened, self.closed = {}, [], []

    def footprint(self, spec):
        return spec.width * spec.height

    def open(self, spec):
        self.opened.append((self.clock.t, spec.sid))
        self.busy[spec.sid] = self.clock.t
        return spec.sid

    def submit(self, h, spec, k):
        end = max(self.clock.t, self.busy[h]) + self.service
        self.busy[h] = end
        return end

    def done(self, tok):
        return self.clock.t >= tok

    def close(self, h):
        self.closed.append((self.clock.t, h))


def specs(n, frames, rate, gap, w=100, h=100, seed=0):
    rng = np.random.default_rng(seed)
    return [StreamSpec(i, w, h, 64, i * gap, poisson_arrivals(rng, i * gap, rate, frames)) for i in range(n)]


def test_every_frame_completes_in_stream_order():
    c = Clock()
    dev = FakeDevice(c, 0.004)
    rep = serve(specs(5, 12, 25.0, 0.05), dev, budget_bytes=10 ** 9, clock=c, idle=c.idle)
    assert rep.frames == 60 and rep.order_ok
    assert min(rep.latencies_s) >= 0.004 - 1e-9
    assert len(dev.closed) == 5


def test_admission_respects_the_memory_budget():
    c = Clock()
    dev = FakeDevice(c, 0.004)
    ss = specs(6, 8, 20.0, 0.0)            # six streams appear at once, 10000 bytes each
    rep = serve(ss, dev, budget_bytes=25000, clock=c, idle=c.idle)
    assert rep.peak_bytes <= 25000 and rep.admitted_late >= 4
    assert rep.frames == 48 and rep.order_ok
    # a waiting stream is admitted only after an earlier one closed
    first_close = min(t for t, _ in dev.closed)
    late_opens = sorted(t for t, _ in dev.opened)[2:]
    assert all(t >= first_close for t in late_opens)


def test_a_stream_larger_than_the_budget_still_runs_alone():
    c = Clock()
    dev = FakeDevice(c, 0.002)
    big = StreamSpec(0, 1000, 1000, 64, 0.0, [0.0, 0.05, 0.1])
    rep = serve([big], dev, budget_bytes=10, clock=c, idle=c.idle)
    assert rep.frames == 3


def test_frames_of_different_streams_overlap():
    # two streams with identical arrivals: with continuous batching the total
    # time is that of one stream, not of the two in sequence
    c = Clock()
    dev = FakeDevice(c, 0.03)
    arr = [0.0, 0.01, 0.02, 0.03]
    two = [StreamSpec(0, 10, 10, 64, 0.0, arr), StreamSpec(1, 10, 10, 64, 0.0, arr)]
    rep = serve(two, dev, budget_bytes=10 ** 6, clock=c, idle=c.idle)
    assert rep.frames == 8
    assert rep.wall_s < 4 * 0.03 + 0.01      # one stream's worth of service time
