"""Request loop over many camera streams with continuous batching.

Streams of one geometry (width, height, disparity range, window rule) share
a pool: one librsgm handle with a fixed number of slots, allocated once when
the loop starts, whose per-stream disparity and variance state stays
resident on the device by slot.  Frames arrive on their own schedule; the
loop
  * sizes the pools by device footprint (``rsgm_footprint``) so that all of
    them fit the memory budget, and admits a stream when a slot of its pool
    is free (a stream that finds none waits until a finished stream frees
    one),
  * at every tick gathers, per pool, the next arrived frame of each admitted
    stream into one launch (``rsgm_slot_frame``): a new stream's first frame
    runs at full range, later frames reduced, streams without an arrived
    frame sit the launch out; frames of one stream stay in order,
  * runs each pool on a CUDA stream of its own, so pools overlap on the GPU
    and a launch can be queued while the previous one runs,
  * records each frame's latency from arrival to the completion of its
    launch, and frees a stream's slot after its last frame.
The scheduling core talks to the device through `Backend`, so its admission,
batching and ordering rules are testable with a fake backend.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class StreamSpec:
    sid: int
    width: int
    height: int
    max_disp: int
    start_s: float              # when the stream appears
    arrivals_s: list            # arrival time of each frame (seconds from the loop's start)
    radius: int = 4

    @property
    def geometry(self):
        return (self.width, self.height, self.max_disp, self.radius)


def poisson_arrivals(rng: np.random.Generator, start_s: float, rate_hz: float, nframes: int) -> list:
    """Frame arrival times of a Poisson process of the given rate."""
    gaps = rng.exponential(1.0 / rate_hz, nframes)
    gaps[0] = 0.0
    return list(start_s + np.cumsum(gaps))


@dataclasses.dataclass
class PoolSpec:
    geometry: tuple             # (width, height, max_disp, radius)
    slots: int
    footprint: int              # device bytes of the pool's handle


class Backend:
    """What the loop needs from the device side."""

    def footprint(self, geometry: tuple, slots: int) -> int:
        """Device bytes of a pool of `slots` streams of this geometry."""
        raise NotImplementedError

    def open_pool(self, pool: PoolSpec):
        raise NotImplementedError

    def submit(self, pool_handle, work: list):
        """Enqueues one launch of the pool; work = [(slot, spec, k)], frame k
        of stream `spec` in `slot` (k = 0: full range).  Returns a token."""
        raise NotImplementedError

    def done(self, token) -> bool:
        raise NotImplementedError

    def release(self, pool_handle, slot: int, spec: StreamSpec) -> None:
        """The stream in `slot` has finished (its last launch completed)."""

    def close_pool(self, pool_handle) -> None:
        raise NotImplementedError


def plan_pools(specs: list, backend: Backend, budget_bytes: int, max_slots: int = 64) -> list:
    """One pool per geometry.  Slots start at the number of streams of the
    geometry (capped) and are taken away, one at a time from the pool whose
    streams have the most slots each, until the pools fit the budget; every
    pool keeps at least one slot."""
    count = {}
    for s in specs:
        count[s.geometry] = count.get(s.geometry, 0) + 1
    slots = {g: min(n, max_slots) for g, n in count.items()}
    fp = lambda g: backend.footprint(g, slots[g])
    while sum(fp(g) for g in slots) > budget_bytes:
        shrinkable = [g for g in slots if slots[g] > 1]
        if not shrinkable:
            break   # one slot per geometry is the minimum the loop can run with
        g = max(shrinkable, key=lambda g: (slots[g] / count[g], fp(g)))
        slots[g] -= 1
    return [PoolSpec(g, slots[g], fp(g)) for g in sorted(slots)]


@dataclasses.dataclass
class Report:
    latencies_s: list
    frames: int
    wall_s: float
    admitted_late: int          # streams that waited for a slot
    pool_bytes: int             # device bytes of all pools
    launches: int
    order_ok: bool

    def summary(self) -> dict:
        lat = sorted(self.latencies_s)
        q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))] if lat else float("nan")
        return {"frames": self.frames, "frames_per_s": self.frames / self.wall_s if self.wall_s else 0.0,
                "p50_ms": 1e3 * q(0.5), "p99_ms": 1e3 * q(0.99), "max_ms": 1e3 * q(1.0),
                "streams_waited_for_a_slot": self.admitted_late, "pool_device_bytes": self.pool_bytes,
                "launches": self.launches,
                "frames_per_launch": self.frames / self.launches if self.launches else 0.0}


def serve(specs: list, backend: Backend, budget_bytes: int, clock: Callable[[], float] = time.perf_counter,
          idle: Callable[[float], None] = lambda s: time.sleep(min(s, 2e-4)), max_queued: int = 2) -> Report:
    """Runs every stream of `specs` to its last frame; returns the latencies.
    max_queued: launches a pool may have in flight at once."""
    pools = plan_pools(specs, backend, budget_bytes)
    by_geom = {p.geometry: i for i, p in enumerate(pools)}
    handles = [backend.open_pool(p) for p in pools]
    free = [list(range(p.slots)) for p in pools]
    slot_of, next_k, done_k = {}, {}, {s.sid: -1 for s in specs}
    queued = [[] for _ in pools]       # per pool: in-flight launches [(token, [(sid, k, arrival)])]
    waiting = sorted(specs, key=lambda s: (s.start_s, s.sid))
    admitted = {}
    latencies, order_ok, late, launches = [], True, 0, 0
    remaining = sum(len(s.arrivals_s) for s in specs)
    t0 = clock()
    now = lambda: clock() - t0
    try:
        while remaining:
            t = now()
            # admission: a free slot of the stream's pool, in order of appearance
            still = []
            for spec in waiting:
                pi = by_geom[spec.geometry]
                if spec.start_s <= t and free[pi]:
                    slot_of[spec.sid] = (pi, free[pi].pop(0))
                    next_k[spec.sid] = 0
                    admitted[spec.sid] = spec
                    late += t - spec.start_s > 1e-3
                else:
                    still.append(spec)
            waiting = still
            # completions
            for pi, q in enumerate(queued):
                while q and backend.done(q[0][0]):
                    _, items = q.pop(0)
                    tc = now()
                    for sid, k, arr in items:
                        latencies.append(tc - arr)
                        order_ok &= done_k[sid] == k - 1
                        done_k[sid] = k
                        remaining -= 1
                        spec = admitted[sid]
                        if k == len(spec.arrivals_s) - 1:   # the stream is finished: free its slot
                            _, slot = slot_of.pop(sid)
                            backend.release(handles[pi], slot, spec)
                            free[pi].append(slot)
                            del admitted[sid]
            # one launch per pool with every admitted stream's next arrived frame
            for pi in range(len(pools)):
                if len(queued[pi]) >= max_queued:
                    continue
                work, items = [], []
                for sid, (qi, slot) in slot_of.items():
                    if qi != pi:
                        continue
                    spec, k = admitted[sid], next_k[sid]
                    if k < len(spec.arrivals_s) and spec.arrivals_s[k] <= t:
                        work.append((slot, spec, k))
                        items.append((sid, k, spec.arrivals_s[k]))
                        next_k[sid] = k + 1
                if work:
                    queued[pi].append((backend.submit(handles[pi], work), items))
                    launches += 1
            if remaining:
                pending = [s.start_s for s in waiting] + [
                    admitted[sid].arrivals_s[next_k[sid]] for sid in admitted
                    if next_k[sid] < len(admitted[sid].arrivals_s)]
                busy = any(queued)
                idle(max(0.0, min(pending) - now()) if pending and not busy else 0.0)
    finally:
        for h in handles:
            backend.close_pool(h)
    return Report(latencies, len(latencies), now(), late, sum(p.footprint for p in pools), launches, order_ok)


class GpuBackend(Backend):
    """One librsgm handle per pool, each on a CUDA stream of its own; the
    frames are device tensors.  With `network` (parameters of the learned
    window) the pools run the learned search window (RSGM_RADIUS_LEARNED),
    all sharing one read-only network."""

    def __init__(self, frames: dict, device="cuda", network=None):
        """frames[sid] = dict(left [F,H,W] u8 device, right, R [F,3,3], t [F,3], K [3,3], baseline)."""
        import torch
        import paper_1809_07986_gb300 as rs
        self.rs, self.torch, self.frames, self.device = rs, torch, frames, device
        self.finals = {}
        self.cnn = rs.rsgm_cnn_create(network, torch.cuda.current_stream()) if network is not None else None

    def params(self, geometry, slots):
        W, H, D, radius = geometry
        mode = self.rs.RSGM_RADIUS_LEARNED if self.cnn else self.rs.RSGM_RADIUS_FIXED
        return self.rs.rsgm_default_params(W, H, max_disp=D, radius=radius, batch=slots, radius_mode=mode)

    def footprint(self, geometry, slots):
        return self.rs.rsgm_footprint(self.params(geometry, slots))

    def open_pool(self, pool):
        W, H = pool.geometry[0], pool.geometry[1]
        cs = self.torch.cuda.Stream(self.device)
        st = self.rs.Stream(self.params(pool.geometry, pool.slots), cs)
        if self.cnn:
            self.rs.rsgm_attach_cnn(st.handle, self.cnn)
        L = self.torch.zeros(pool.slots, H, W, dtype=self.torch.uint8, device=self.device)
        return dict(stream=cs, st=st, L=L, R=self.torch.zeros_like(L), slots=pool.slots)

    def submit(self, h, work):
        B = h["slots"]
        roles = np.zeros(B, np.uint8)
        Rm = np.tile(np.eye(3, dtype=np.float32), (B, 1, 1))
        tv = np.zeros((B, 3), np.float32)
        K = base = None
        with self.torch.cuda.stream(h["stream"]):
            for slot, spec, k in work:
                f = self.frames[spec.sid]
                h["L"][slot].copy_(f["left"][k], non_blocking=True)
                h["R"][slot].copy_(f["right"][k], non_blocking=True)
                roles[slot] = self.rs.RSGM_SLOT_FULL if k == 0 else self.rs.RSGM_SLOT_REDUCED
                Rm[slot] = f["R"][k].cpu().numpy()
                tv[slot] = f["t"][k].cpu().numpy()
                K, base = f["K"], f["baseline"]
            self.rs.rsgm_slot_frame(h["st"].handle, roles, h["L"], h["R"], Rm, tv, K, base)
            ev = self.torch.cuda.Event()
            ev.record(h["stream"])
        return ev

    def done(self, token):
        return token.query()

    def release(self, h, slot, spec):
        # copied out on the pool's CUDA stream, behind the stream's last
        # launch and ahead of the slot's next occupant: the loop does not wait
        torch = self.torch
        B, H, W = h["st"].shape
        with torch.cuda.stream(h["stream"]):
            d = torch.empty(B, H, W, dtype=torch.float32, device=self.device)
            p = torch.empty_like(d)
            m = torch.empty(B, H, W, dtype=torch.uint8, device=self.device)
            di = torch.empty(B, H, W, dtype=torch.int16, device=self.device)
            self.rs.rsgm_state(h["st"].handle, d, p, m, di)
            # the slot's share only, cloned on the same stream; the pool-wide
            # copies return to the allocator, which reuses them in stream order
            self.finals[spec.sid] = tuple(x[slot].clone() for x in (d, p, m, di))

    def close_pool(self, h):
        h["st"].sync()  # the state copies are complete before the handle goes
        h["st"].close()

    def close(self):
        if self.cnn:
            self.rs.rsgm_cnn_destroy(self.cnn)
            self.cnn = None
