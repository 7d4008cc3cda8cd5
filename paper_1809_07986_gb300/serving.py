"""Request loop over many camera streams (continuous batching).

Each camera stream owns one librsgm handle (its disparity and variance state
stays resident on the device) on a CUDA stream of its own, so frames of
different streams overlap on the GPU.  Frames arrive on their own schedule;
the loop
  * admits a stream when its device footprint fits the memory budget (a
    stream that does not fit waits until finished streams free memory),
  * runs a stream's first frame at full range, later frames reduced,
  * dispatches every arrived frame of an admitted stream at once (frames of
    one stream stay in order on its CUDA stream),
  * records each frame's latency from arrival to completion and closes a
    stream after its last frame.
The scheduling core is independent of the GPU (see `Backend`), so its
admission and ordering rules are testable with a fake backend.
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


def poisson_arrivals(rng: np.random.Generator, start_s: float, rate_hz: float, nframes: int) -> list:
    """Frame arrival times of a Poisson process of the given rate."""
    gaps = rng.exponential(1.0 / rate_hz, nframes)
    gaps[0] = 0.0
    return list(start_s + np.cumsum(gaps))


class Backend:
    """What the loop needs from the device side."""

    def footprint(self, spec: StreamSpec) -> int:
        raise NotImplementedError

    def open(self, spec: StreamSpec):
        raise NotImplementedError

    def submit(self, handle, spec: StreamSpec, k: int):
        """Enqueues frame k (0: full range) and returns a completion token."""
        raise NotImplementedError

    def done(self, token) -> bool:
        raise NotImplementedError

    def close(self, handle) -> None:
        raise NotImplementedError


@dataclasses.dataclass
class Report:
    latencies_s: list
    frames: int
    wall_s: float
    admitted_late: int          # streams that waited for memory
    peak_bytes: int
    order_ok: bool

    def summary(self) -> dict:
        lat = sorted(self.latencies_s)
        q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))] if lat else float("nan")
        return {"frames": self.frames, "frames_per_s": self.frames / self.wall_s if self.wall_s else 0.0,
                "p50_ms": 1e3 * q(0.5), "p99_ms": 1e3 * q(0.99), "max_ms": 1e3 * q(1.0),
                "streams_waited_for_memory": self.admitted_late, "peak_device_bytes": self.peak_bytes}


def serve(specs: list, backend: Backend, budget_bytes: int, clock: Callable[[], float] = time.perf_counter,
          idle: Callable[[float], None] = lambda s: time.sleep(min(s, 2e-4))) -> Report:
    """Runs every stream of `specs` to its last frame; returns the latencies."""
    t0 = clock()
    now = lambda: clock() - t0
    waiting = sorted(specs, key=lambda s: (s.start_s, s.sid))   # not yet admitted
    active = {}           # sid -> [spec, handle, next frame to submit, footprint]
    inflight = []         # (sid, k, arrival, token)
    used = peak = 0
    admitted_late = 0
    latencies = []
    completed = {s.sid: -1 for s in specs}
    order_ok = True
    remaining = sum(len(s.arrivals_s) for s in specs)
    while remaining:
        t = now()
        # admission by device footprint, in order of appearance
        still = []
        for spec in waiting:
            if spec.start_s > t:
                still.append(spec)
                continue
            fp = backend.footprint(spec)
            if used + fp <= budget_bytes or (not active and not inflight):
                active[spec.sid] = [spec, backend.open(spec), 0, fp]
                used += fp
                peak = max(peak, used)
                if t - spec.start_s > 1e-3:
                    admitted_late += 1
            else:
                still.append(spec)
        waiting = still
        # dispatch every arrived frame of the admitted streams
        for sid, st in active.items():
            spec, handle, k, _ = st
            while k < len(spec.arrivals_s) and spec.arrivals_s[k] <= t:
                inflight.append((sid, k, spec.arrivals_s[k], backend.submit(handle, spec, k)))
                k += 1
            st[2] = k
        # completions
        keep = []
        for sid, k, arr, tok in inflight:
            if backend.done(tok):
                latencies.append(now() - arr)
                order_ok &= completed[sid] == k - 1
                completed[sid] = k
                remaining -= 1
            else:
                keep.append((sid, k, arr, tok))
        inflight = keep
        # streams whose last frame completed release their memory
        for sid in [s for s, st in active.items() if completed[s] == len(st[0].arrivals_s) - 1]:
            spec, handle, _, fp = active.pop(sid)
            backend.close(handle)
            used -= fp
        if remaining:
            nxt = [s.start_s for s in waiting] + [st[0].arrivals_s[st[2]] for st in active.values()
                                                  if st[2] < len(st[0].arrivals_s)]
            idle(max(0.0, min(nxt) - now()) if nxt and not inflight else 0.0)
    return Report(latencies, len(latencies), now(), admitted_late, peak, order_ok)


class GpuBackend(Backend):
    """librsgm handles, one per stream, each on its own CUDA stream."""

    def __init__(self, frames: dict, device="cuda"):
        """frames[sid] = dict(left [F,H,W] u8 device, right, R [F,3,3], t [F,3], K [3,3], baseline)."""
        import torch
        import paper_1809_07986_gb300 as rs
        self.rs, self.torch, self.frames, self.device = rs, torch, frames, device
        self.finals = {}

    def params(self, spec):
        return self.rs.rsgm_default_params(spec.width, spec.height, max_disp=spec.max_disp, radius=spec.radius)

    def footprint(self, spec):
        return self.rs.rsgm_footprint(self.params(spec))

    def open(self, spec):
        cs = self.torch.cuda.Stream(self.device)
        return (spec.sid, cs, self.rs.Stream(self.params(spec), cs))

    def submit(self, handle, spec, k):
        sid, cs, st = handle
        f = self.frames[sid]
        with self.torch.cuda.stream(cs):
            if k == 0:
                st.full_frame(f["left"][0], f["right"][0])
            else:
                st.reduced_frame(f["left"][k], f["right"][k], f["R"][k:k + 1], f["t"][k:k + 1], f["K"], f["baseline"])
            ev = self.torch.cuda.Event()
            ev.record(cs)
        return ev

    def done(self, token):
        return token.query()

    def close(self, handle):
        sid, cs, st = handle
        with self.torch.cuda.stream(cs):
            self.finals[sid] = tuple(x.clone() for x in st.state(device=self.device))
        st.close()
