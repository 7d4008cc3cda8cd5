"""The request loop's scheduling rules, on the CPU with a fake device and a
simulated clock: a pool runs its launches one after another, each taking a
fixed time plus a time per frame it carries."""
import numpy as np

from paper_1809_07986_gb300.serving import Backend, PoolSpec, StreamSpec, plan_pools, poisson_arrivals, serve


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def idle(self, s):
        self.t += max(s, 1e-4)


class FakeDevice(Backend):
    """A pool is a FIFO of launches; a launch takes base + per_frame * frames.
    Device bytes of a pool: width * height per slot."""

    def __init__(self, clock, base, per_frame=0.0):
        self.clock, self.base, self.per_frame = clock, base, per_frame
        self.launches, self.released, self.pools = [], [], []

    def footprint(self, geometry, slots):
        return geometry[0] * geometry[1] * slots

    def open_pool(self, pool):
        h = dict(pool=pool, busy=self.clock.t, slots_in_use={})
        self.pools.append(h)
        return h

    def submit(self, h, work):
        slots = [slot for slot, _, _ in work]
        assert len(set(slots)) == len(slots) and all(0 <= s < h["pool"].slots for s in slots)
        for slot, spec, k in work:
            # a slot holds one stream at a time, and its frames go in order
            owner = h["slots_in_use"].setdefault(slot, spec.sid)
            assert owner == spec.sid
        end = max(self.clock.t, h["busy"]) + self.base + self.per_frame * len(work)
        h["busy"] = end
        self.launches.append((self.clock.t, h["pool"].geometry, [(spec.sid, k) for _, spec, k in work]))
        return end

    def done(self, tok):
        return self.clock.t >= tok

    def release(self, h, slot, spec):
        assert h["slots_in_use"].pop(slot) == spec.sid
        self.released.append((self.clock.t, spec.sid))

    def close_pool(self, h):
        pass


def specs(n, frames, rate, gap, w=100, h=100, seed=0):
    rng = np.random.default_rng(seed)
    return [StreamSpec(i, w, h, 64, i * gap, poisson_arrivals(rng, i * gap, rate, frames)) for i in range(n)]


def test_every_frame_completes_in_stream_order():
    c = Clock()
    dev = FakeDevice(c, 0.004)
    rep = serve(specs(5, 12, 25.0, 0.05), dev, budget_bytes=10 ** 9, clock=c, idle=c.idle)
    assert rep.frames == 60 and rep.order_ok
    assert min(rep.latencies_s) >= 0.004 - 1e-9
    assert len(dev.released) == 5
    # every stream's first frame runs before its later ones, one frame per launch
    for sid in range(5):
        ks = [k for _, _, work in dev.launches for s, k in work if s == sid]
        assert ks == list(range(12))


def test_frames_of_one_geometry_share_launches():
    # eight streams with identical arrivals: continuous batching puts their
    # frames into the same launches instead of one launch per frame
    c = Clock()
    dev = FakeDevice(c, 0.02, 0.001)
    arr = [0.0, 0.05, 0.1, 0.15]
    eight = [StreamSpec(i, 10, 10, 64, 0.0, arr) for i in range(8)]
    rep = serve(eight, dev, budget_bytes=10 ** 6, clock=c, idle=c.idle)
    assert rep.frames == 32 and rep.order_ok
    assert rep.launches == 4 and all(len(w) == 8 for _, _, w in dev.launches)
    assert rep.summary()["frames_per_launch"] == 8.0


def test_frames_arriving_during_a_launch_join_the_next_one():
    # stream 1 appears while stream 0's launch runs: it is admitted at once and
    # its first frame rides in the next launch, next to stream 0's later frames
    c = Clock()
    dev = FakeDevice(c, 0.03)
    s0 = StreamSpec(0, 10, 10, 64, 0.0, [0.0, 0.01, 0.02, 0.04])
    s1 = StreamSpec(1, 10, 10, 64, 0.015, [0.015, 0.03, 0.045])
    rep = serve([s0, s1], dev, budget_bytes=10 ** 6, clock=c, idle=c.idle)
    assert rep.frames == 7 and rep.order_ok
    mixed = [w for _, _, w in dev.launches if {s for s, _ in w} == {0, 1}]
    assert mixed and (1, 0) in mixed[0]


def test_pools_fit_the_budget_and_streams_wait_for_a_slot():
    c = Clock()
    dev = FakeDevice(c, 0.004)
    ss = specs(6, 8, 20.0, 0.0)            # six streams appear at once; 10000 bytes per slot
    rep = serve(ss, dev, budget_bytes=25000, clock=c, idle=c.idle)
    assert rep.pool_bytes <= 25000 and dev.pools[0]["pool"].slots == 2
    assert rep.frames == 48 and rep.order_ok and rep.admitted_late >= 4
    # a waiting stream's first frame runs only after an earlier stream finished
    first_release = min(t for t, _ in dev.released)
    starts = sorted(t for t, _, w in dev.launches for s, k in w if k == 0)
    assert all(t >= first_release for t in starts[2:])


def test_pool_planning_keeps_one_slot_per_geometry():
    class Sizes(Backend):
        def footprint(self, g, slots):
            return g[0] * g[1] * slots

    a = [StreamSpec(i, 100, 100, 64, 0.0, [0.0]) for i in range(6)]
    b = [StreamSpec(10 + i, 10, 10, 32, 0.0, [0.0]) for i in range(3)]
    pools = plan_pools(a + b, Sizes(), budget_bytes=10 ** 9)
    assert [(p.geometry[0], p.slots) for p in pools] == [(10, 3), (100, 6)]
    pools = plan_pools(a + b, Sizes(), budget_bytes=30000)
    assert sum(p.footprint for p in pools) <= 30000 and all(p.slots >= 1 for p in pools)
    pools = plan_pools(a + b, Sizes(), budget_bytes=1)     # below one slot each: one slot each
    assert all(p.slots == 1 for p in pools) and isinstance(pools[0], PoolSpec)


def test_different_geometries_overlap():
    # two pools run on their own queues: the total time is one stream's worth
    c = Clock()
    dev = FakeDevice(c, 0.03)
    arr = [0.0, 0.01, 0.02, 0.03]
    two = [StreamSpec(0, 10, 10, 64, 0.0, arr), StreamSpec(1, 20, 10, 64, 0.0, arr)]
    rep = serve(two, dev, budget_bytes=10 ** 6, clock=c, idle=c.idle)
    assert rep.frames == 8 and len(dev.pools) == 2
    assert rep.wall_s < 4 * 0.03 + 0.01
