#!/usr/bin/env python3
"""Throughput benchmark of the reduced-space SGM + per-pixel Kalman path.

Workload (per GPU): B seeded synthetic stereo streams shaped like the paper's
KITTI raw sequences -- 1242 x 375 uint8, f = 721 px, baseline 0.54 m, 128
disparities, ego-motion about 1 m/frame with at most 1 degree of yaw per frame,
ground plane + 20 boxes (3 moving).  Frame 0 of every stream is a full-range
frame (untimed); each step is one reduced frame (fixed +-r windows, 8 paths,
Kalman update and gate) of all B streams.  Inputs are resident in HBM before
the timed region; the per-step working set (ragged cost and aggregated volumes,
about 0.7 GB at B = 32) is larger than the 129 MB L2.

Prints one JSON line (rank 0).  ``--impl reference`` times the oracle (the
plain CPU restatement of the method) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H, D, F, BASE = 1242, 375, 128, 721.0, 0.54
N_PATHS = 8
METRIC = "frames/s and cost-cell updates/s at 1242x375 vs plain form; p99 latency"
# Algorithmic integer operations of one Eq. 1 update at one (pixel, disparity,
# direction): + C, two + P1, three min (d, d-1, d+1 against m + P2), - m, the
# running minimum for the next pixel, + into S.
OPS_PER_CELL_PATH = 9
# Whole-frame algorithmic work (the scope table's per-pixel and per-cell
# figures): 23 B per pixel (2 B images, 8 B state read, 8 B state write, 4 B
# disparity, 1 B mask) and 4 B per cell (S written once, read once by the
# winner-takes-all); 10 integer operations per cell and path (two neighbour
# loads, three minima, three additions/subtractions, the running minimum, the
# addition into S) plus 2 per cost (xor, popcount).
FRAME_BYTES_PER_PIXEL = 23
FRAME_BYTES_PER_CELL = 4
FRAME_OPS_PER_CELL = 10 * N_PATHS + 2
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per cell of the
# dominant kernel from one ncu capture; None while the kernel has changed
# since the last capture.  Captured: k_lines at register capacity 10 with 16
# rows per warp, one 32-stream launch of reduced frame 2 (188,694,827 cells):
# 3,544,918,784 B read + 2,052,158,464 B written.
NCU_DRAM_BYTES_PER_CELL = (3544918784 + 2052158464) / 188694827
# the configuration that figure was captured on: streams per launch, register
# capacity and rows per warp; other configurations report no traffic
NCU_DRAM_CONFIG = (32, 10, 16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=32, help="camera streams per GPU")
    ap.add_argument("--radius", type=int, default=4)
    ap.add_argument("--schedule", type=int, default=0,
                    help="path-sweep register capacity in cells for every handle (0: autotune each handle)")
    ap.add_argument("--rows", type=int, default=0, choices=[0, 8, 16, 32],
                    help="with --schedule: the rows' sweep (0: the row sweep beside the line sweep, "
                         "else rows per warp of the line sweep)")
    ap.add_argument("--priority", type=int, default=1, choices=[0, 1],
                    help="1 (default): each handle's CUDA stream gets a higher priority than the next one's; "
                         "0: equal priorities")
    ap.add_argument("--handles", type=int, default=2,
                    help="the GPU's streams are split over this many handles on as many CUDA streams")
    ap.add_argument("--learned", action="store_true",
                    help="train the learned search window on all 2000 frames of seeded 384x128 pairs (default: 512)")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the mixed-resolution group, learned-window and request-loop legs")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="host cores for the oracle legs (0: every core this process may run on)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-form, latency, e2e and CPU-baseline legs")
    return ap.parse_args()


def launches_per_frame(rows: int) -> int:
    """Kernels one reduced frame of an 8-path handle launches: splat, fill,
    window, row scan, census, cost, the aggregation (one sweep, or the row
    sweep beside the line sweep when rows = 0) and the update."""
    return 8 + (rows == 0)


def stream_seeds(rank: int, batch: int) -> list:
    """Seeds of the B streams a rank processes: disjoint across ranks, so the
    ranks shard independent streams (weak scaling, no data-path collective)."""
    return [1000 + 1000 * rank + b for b in range(batch)]


def reduce_over_ranks(x: float, op: str, world: int, device=None) -> float:
    """max or sum of a scalar over ranks (identity when world == 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ inputs

def make_inputs(seeds, nframes, device):
    import torch
    import synth
    Ls, Rs, Ms, Ts = [], [], [], []
    K = None
    for seed in seeds:
        s = synth.kitti_like_sequence(seed, n_frames=max(100, nframes), width=W, height=H, f=F,
                                      baseline=BASE, device=device, render_frames=nframes)
        Ls.append(s["left"])
        Rs.append(s["right"])
        Ms.append(s["R"])
        Ts.append(s["t"])
        K = s["K"]
    # [F, B, H, W] so that one frame of all streams is contiguous
    left = torch.stack(Ls, 1).contiguous()
    right = torch.stack(Rs, 1).contiguous()
    return left, right, torch.stack(Ms, 1).contiguous(), torch.stack(Ts, 1).contiguous(), K


# ------------------------------------------------------------------ reference arm: the oracle

def _reference_stream(job):
    """Reference-arm worker: renders its own seeded stream, runs frame 0 at
    full range and W warm-up frames untimed, then times K reduced frames."""
    seed, warmup, steps, radius = job
    import oracle
    import synth
    n = 1 + warmup + steps
    s = synth.kitti_like_sequence(seed, n_frames=max(100, n), width=W, height=H, f=F, baseline=BASE,
                                  render_frames=n)
    P = oracle.Params(W, H, max_disp=D, radius=radius)
    L, R = s["left"].numpy(), s["right"].numpy()
    o = oracle.frame(P, L[0], R[0])
    total, cells = 0.0, 0
    for k in range(1, n):
        t0 = time.perf_counter()
        o = oracle.frame(P, L[k], R[k], state=(o["d"], o["p"]),
                         motion=(s["R"][k].numpy(), s["t"][k].numpy(), s["K"].numpy(), BASE))
        dt = time.perf_counter() - t0
        if k > warmup:
            total += dt
            cells += o["ncells"]
    return steps, total, cells


def run_reference(args, rank, world):
    if rank != 0:
        return
    import multiprocessing as mp
    cores = args.cpu_cores or host_cores()
    jobs = [(1000 + b, args.warmup, args.steps, args.radius) for b in range(cores)]
    with mp.get_context("spawn").Pool(cores, initializer=_single_thread_worker) as pool:
        res = pool.map(_reference_stream, jobs)
    fps = sum(n / t for n, t, _ in res)
    cups = sum(c * N_PATHS / t for _, t, c in res)
    ms = 1e3 * max(t / n for n, t, _ in res)
    sample = ("%d single-threaded oracle processes, one per host core, each on its own seeded 1242x375 stream: "
              "reduced frames %d..%d (r=%d, 8 paths) timed; nproc=%d" % (
                  cores, args.warmup + 1, args.warmup + args.steps, args.radius, cores))
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic",
            "config": {"workload": "kitti-shaped stereo 1242x375, D=128, r=%d, 8 paths" % args.radius,
                       "streams": cores, "sample": sample},
            "cell_updates_per_s": cups,
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _single_thread_worker():
    """Pool initializer: one thread per oracle process (the renderer's torch
    and numpy would otherwise start a thread per core in every process)."""
    for k in ("OMP_NUM_THREADS", "MKL_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ[k] = "1"
    import torch
    torch.set_num_threads(1)


def _oracle_stream(job):
    """One oracle worker: frame 0 at full range (untimed), then reduced frames
    until the budget is spent; returns (frames, seconds, cells)."""
    L, R, Rm, tv, K, radius, budget_s = job
    import oracle
    P = oracle.Params(W, H, max_disp=D, radius=radius)
    o = oracle.frame(P, L[0], R[0])
    n, total, cells = 0, 0.0, 0
    for k in range(1, L.shape[0]):
        t0 = time.perf_counter()
        o = oracle.frame(P, L[k], R[k], state=(o["d"], o["p"]), motion=(Rm[k], tv[k], K, BASE))
        total += time.perf_counter() - t0
        n += 1
        cells += o["ncells"]
        if total >= budget_s and n >= 3:
            break
    return n, total, cells


def cpu_baseline(args, left, right, Rm, tv, K, budget_s=8.0, max_frames=16):
    """The oracle as it stands, on this host's cores: single-threaded on
    stream 0, then one single-threaded oracle process per core, each on a
    stream of its own (the oracle itself stays plain and serial)."""
    import multiprocessing as mp
    import numpy as np
    nf = min(max_frames, left.shape[0])
    Kn = K.numpy()

    def job(b):
        return (np.ascontiguousarray(left[:nf, b].cpu().numpy()), np.ascontiguousarray(right[:nf, b].cpu().numpy()),
                Rm[:nf, b].numpy(), tv[:nf, b].numpy(), Kn, args.radius, budget_s)

    n1, t1, _ = _oracle_stream(job(0))
    single = n1 / t1
    cores = args.cpu_cores or host_cores()
    jobs = [job(b % left.shape[1]) for b in range(cores)]
    # spawn, not fork: the parent holds a CUDA context
    with mp.get_context("spawn").Pool(cores, initializer=_single_thread_worker) as pool:
        res = pool.map(_oracle_stream, jobs)
    allcore = sum(n / t for n, t, _ in res)
    return {"value": allcore, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": "one single-threaded oracle process per host core (%d), each on its own stream of the "
                      "workload: frame 0 full range untimed, then up to %d reduced frames (r=%d, 8 paths) or "
                      "%.0f s; nproc=%d" % (cores, nf - 1, args.radius, budget_s, cores),
            "single_thread": {"value": single, "unit": "frames/s", "frames": n1,
                              "sample": "stream 0, reduced frames 1..%d, one thread" % n1}}


# ------------------------------------------------------------------ mixed-resolution group

MIXED = [(6, 640, 480, 64, 400.0), (6, 1242, 375, 128, 721.0), (4, 1920, 1080, 256, 1000.0)]


def mixed_group(args, dev, stream):
    """16 streams of three resolutions advanced by one CUDA graph launch per
    tick, each member with its autotuned aggregation schedule."""
    import torch
    import synth
    import paper_1809_07986_gb300 as rs
    nframes = 1 + args.warmup + args.steps
    members, data = [], []
    for gi, (B, Wm, Hm, Dm, f) in enumerate(MIXED):
        seqs = [synth.kitti_like_sequence(5000 + 100 * gi + b, n_frames=max(100, nframes), width=Wm, height=Hm,
                                          f=f, baseline=BASE, device=dev, render_frames=nframes)
                for b in range(B)]
        data.append(dict(L=torch.stack([q["left"] for q in seqs], 1).contiguous(),
                         R=torch.stack([q["right"] for q in seqs], 1).contiguous(),
                         Rm=torch.stack([q["R"] for q in seqs], 1).contiguous(),
                         t=torch.stack([q["t"] for q in seqs], 1).contiguous(), K=seqs[0]["K"]))
        members.append(rs.Stream(rs.rsgm_default_params(Wm, Hm, max_disp=Dm, radius=args.radius, batch=B), stream))
    group = rs.rsgm_group_create([m.handle for m in members])
    tuned = []

    def tick(k):
        rs.rsgm_group_reduced_frame(group, [x["L"][k] for x in data], [x["R"][k] for x in data],
                                    [x["Rm"][k] for x in data], [x["t"][k] for x in data],
                                    [x["K"] for x in data], [BASE] * len(data))

    with torch.cuda.stream(stream):
        for m, x in zip(members, data):
            m.full_frame(x["L"][0], x["R"][0])
        tick(1)
        for m in members:
            rs.rsgm_autotune(m.handle)
            tuned.append(rs.rsgm_get_schedule(m.handle))
        for k in range(2, 1 + args.warmup):
            tick(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(1 + args.warmup, nframes):
            tick(k)
        e1.record(stream)
        torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    rs.rsgm_group_destroy(group)
    for m in members:
        m.close()
    nstreams = sum(g[0] for g in MIXED)
    return {"frames_per_s": nstreams * args.steps / el, "ms_per_tick": 1e3 * el / args.steps,
            "streams": "6x640x480/D64 + 6x1242x375/D128 + 4x1920x1080/D256",
            "graph_launches_per_tick": 1,
            "schedule_tuned": [{"cells": c, "rows": "row sweep" if r == 0 else "%d per warp" % r} for c, r in tuned]}


# ------------------------------------------------------------------ request loop

def serving_loop(dev, nstreams=32, frames=20, budget_gb=48.0, seed=9, network=None):
    """32 streams appear over one second, each a Poisson process at 10-30 Hz
    of a resolution drawn from {640x480/D64, 1242x375/D128, 1920x1080/D256};
    pools sized by device footprint under a budget; a new stream's first frame
    runs at full range; with `network`, the learned search window."""
    import numpy as np
    import synth
    from paper_1809_07986_gb300.serving import GpuBackend, StreamSpec, poisson_arrivals, serve
    rng = np.random.default_rng(seed)
    kinds = [(640, 480, 64, 400.0), (1242, 375, 128, 721.0), (1920, 1080, 256, 1000.0)]
    specs, data = [], {}
    for i in range(nstreams):
        W_, H_, D_, f_ = kinds[int(rng.integers(0, 3))]
        s = synth.kitti_like_sequence(9000 + i, n_frames=100, width=W_, height=H_, f=f_, baseline=BASE, device=dev,
                                      render_frames=frames)
        data[i] = dict(left=s["left"], right=s["right"], R=s["R"], t=s["t"], K=s["K"], baseline=BASE)
        start = float(rng.uniform(0.0, 1.0))
        specs.append(StreamSpec(i, W_, H_, D_, start, poisson_arrivals(rng, start, float(rng.uniform(10, 30)), frames)))
    backend = GpuBackend(data, device=dev, network=network)
    try:
        rep = serve(specs, backend, budget_bytes=int(budget_gb * 1e9))
    finally:
        backend.close()
    out = rep.summary()
    out.update(streams=nstreams, frames_per_stream=frames, budget_gb=budget_gb, order_ok=rep.order_ok,
               window="learned (trained network, fallback +-8)" if network is not None else "fixed +-4",
               arrival="Poisson 10-30 Hz per stream, streams appearing over 1 s",
               batching="one pool handle per resolution, each launch carrying every admitted stream's next "
                        "arrived frame (rsgm_slot_frame)")
    return out


def path_ablation(dev, nstreams=8, nframes=11, radius=4):
    """The paper's path ablation (Section 5, Table 2: 8 paths against 4
    non-diagonal and 4 diagonal ones) on seeded paper-shaped sequences: for
    each path set the reduced method and the full-range (plain) form run on
    the same frames; reported per set are frames/s of the reduced form and
    bad-pixel rates over frames 1..nframes-1, against the renderer's ground
    truth (> 3 px and > 5 %, the KITTI outlier rule) and against the
    full-range result of the same path set (> 3 px)."""
    import numpy as np
    import torch
    import synth
    import paper_1809_07986_gb300 as rs
    seqs = [synth.kitti_like_sequence(7000 + b, n_frames=100, width=W, height=H, f=F, baseline=BASE, device=dev,
                                      render_frames=nframes) for b in range(nstreams)]
    st = lambda k: torch.stack([q[k] for q in seqs], 1).contiguous()
    L, R, gt, Rm, tv, K = st("left"), st("right"), st("disp"), st("R"), st("t"), seqs[0]["K"]
    out = {}
    for name, mask in (("8 paths", 0xFF), ("4 non-diagonal", 0x0F), ("4 diagonal", 0xF0)):
        res = {}
        for mode in (rs.RSGM_RADIUS_FIXED, rs.RSGM_RADIUS_FULL):
            P = rs.rsgm_default_params(W, H, max_disp=D, radius=radius, batch=nstreams, path_mask=mask,
                                       radius_mode=mode)
            ds, ms = [], 0.0
            with rs.Stream(P) as h:
                h.full_frame(L[0], R[0])
                for k in range(1, nframes):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    h.reduced_frame(L[k], R[k], Rm[k], tv[k], K, BASE)
                    e1.record()
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                    ds.append(h.state()[0].cpu().numpy())
            res[mode] = (ds, nstreams * (nframes - 1) / (ms / 1e3))
        red, full = res[rs.RSGM_RADIUS_FIXED][0], res[rs.RSGM_RADIUS_FULL][0]
        g = gt[1:].cpu().numpy()

        def kitti(d):
            ok = g > 0
            err = np.abs(np.stack(d) - g)
            return float(((err > 3) & (err > 0.05 * g) & ok).sum() / ok.sum())

        out[name] = {"frames_per_s": res[rs.RSGM_RADIUS_FIXED][1],
                     "bad_vs_gt": kitti(red), "bad_vs_gt_full_range": kitti(full),
                     "bad_vs_full_range": float((np.abs(np.stack(red) - np.stack(full)) > 3).mean())}
    out["workload"] = "%d seeded 1242x375 streams, D=128, r=%d, reduced frames 1..%d" % (nstreams, radius, nframes - 1)
    return out


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_1809_07986_gb300 as rs
    from paper_1809_07986_gb300 import build as pkg_build

    pkg_build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    B = args.batch
    nframes = 1 + args.warmup + args.steps
    left, right, Rm, tv, K = make_inputs(stream_seeds(rank, B), nframes, dev)
    stream = torch.cuda.Stream(dev)
    P = rs.rsgm_default_params(W, H, max_disp=D, radius=args.radius, batch=B)
    gs = rs.Stream(P, stream)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_over_ranks(x, "max", world, dev)

    def sum_over_ranks(x):
        return reduce_over_ranks(x, "sum", world, dev)

    def run(h, frames, host=None, out=None):
        for k in frames:
            if host is None:
                rs.rsgm_reduced_frame(h, left[k], right[k], Rm[k], tv[k], K, BASE)
            else:
                rs.rsgm_reduced_frame(h, host[0][k], host[1][k], Rm[k], tv[k], K, BASE)
                rs.rsgm_state(h, out[0], None, out[1], None)

    # The streams are split over `handles` handles, each on a CUDA stream of
    # its own: their kernels overlap, filling the tails of each other's launches.
    nh = max(1, min(args.handles, B))
    cut = [B * i // nh for i in range(nh + 1)]
    parts = []
    for i in range(nh):
        a, z = cut[i], cut[i + 1]
        Ph = rs.rsgm_default_params(W, H, max_disp=D, radius=args.radius, batch=z - a)
        # Each handle's CUDA stream outranks the next one's (--priority 1):
        # the first handle's kernels take the SMs first and the others fill
        # what is left, in order, so
        # the handles never fall into step (both sweeping, then both
        # updating), which with equal priorities happened in some runs.
        cs = torch.cuda.Stream(dev, priority=-(nh - 1 - i) if args.priority else 0)
        parts.append((rs.Stream(Ph, cs), cs, a, z))

    def tune(h):
        """Sets the handle's aggregation schedule; returns (cells, rows)."""
        if args.schedule > 0:
            rs.rsgm_set_schedule(h, args.schedule)
            rs.rsgm_set_rows_per_warp(h, args.rows)
        else:
            rs.rsgm_autotune(h)
        return rs.rsgm_get_schedule(h)

    def run_parts(frames, host=None, out=None):
        for k in frames:
            for ph, cs, a, z in parts:
                with torch.cuda.stream(cs):
                    if host is None:
                        rs.rsgm_reduced_frame(ph.handle, left[k][a:z], right[k][a:z], Rm[k][a:z], tv[k][a:z], K, BASE)
                    else:
                        rs.rsgm_reduced_frame(ph.handle, host[0][k][a:z], host[1][k][a:z], Rm[k][a:z], tv[k][a:z],
                                              K, BASE)
                        rs.rsgm_state(ph.handle, out[0][a:z], None, out[1][a:z], None)

    def start_parts(host=None):
        src = host if host is not None else (left, right)
        for ph, cs, a, z in parts:
            with torch.cuda.stream(cs):
                ph.full_frame(src[0][0][a:z], src[1][0][a:z])

    def timed_parts(frames, host=None, out=None):
        main = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for _, cs, _, _ in parts:
            cs.wait_event(e0)
        run_parts(frames, host, out)
        for _, cs, _, _ in parts:
            ev = torch.cuda.Event()
            ev.record(cs)
            main.wait_event(ev)
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    with ClockSampler(local_rank) as clk:
        # the sampler runs from the warm-up on, so that it sees the GPU under load
        start_parts()
        run_parts(range(1, 2))
        tuned = [tune(ph.handle) for ph, _, _, _ in parts]   # aggregation schedule per handle
        run_parts(range(2, 1 + args.warmup))
        torch.cuda.synchronize()
        c0 = sum(ph.counters()[1] for ph, _, _, _ in parts)
        barrier()
        torch.cuda.synchronize()
        elapsed = max_over_ranks(timed_parts(range(1 + args.warmup, nframes)))
        barrier()
        c1 = sum(ph.counters()[1] for ph, _, _, _ in parts)
    steps = args.steps
    frames_all = B * steps * world
    cells_local = c1 - c0
    cells_all = sum_over_ranks(cells_local)
    value = frames_all / elapsed
    result = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": steps,
              "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
              "config": {"workload": "kitti-shaped stereo 1242x375, D=128, r=%d, 8 paths, %d seeded streams "
                                     "per GPU, frames 1..%d of 100-frame sequences" % (args.radius, B, nframes - 1),
                         "streams_per_gpu": B, "width": W, "height": H, "max_disp": D, "radius": args.radius,
                         "paths": N_PATHS, "parallelism": "stream sharding, no collective" if world > 1 else "1 GPU",
                         "l2": "per-step working set (ragged volumes) larger than L2"},
              "cell_updates_per_s": cells_all * N_PATHS / elapsed,
              "cells_per_frame": cells_local / (B * steps),
              "schedule_tuned": [{"cells": c, "rows": "row sweep" if r == 0 else "%d per warp" % r}
                                 for c, r in tuned],
              "handles": "%d handles of %s streams on %d CUDA streams%s" % (
                  nh, "/".join(str(cut[i + 1] - cut[i]) for i in range(nh)), nh,
                  ", each at a higher stream priority than the next" if args.priority and nh > 1 else ""),
              "gpu_launches": steps * sum(launches_per_frame(r) for _, r in tuned),
              "clocks": clk.summary()}

    # ---- dominant kernel: stage times with CUDA events on the launching stream
    with torch.cuda.stream(stream):
        gs.full_frame(left[0], right[0])
        run(gs.handle, range(1, 2))
        gs_cells, gs_rows = tune(gs.handle)
        rs.rsgm_enable_stage_timing(gs.handle, True)
        rs.rsgm_stage_times(gs.handle)
        c_before = gs.counters()[1]
        run(gs.handle, range(2, nframes))
        st_ms, st_frames = rs.rsgm_stage_times(gs.handle)
        c_after = gs.counters()[1]
        rs.rsgm_enable_stage_timing(gs.handle, False)
    cells_per_frame = (c_after - c_before) / max(st_frames, 1)
    agg_ms = st_ms["aggregate"] / max(st_frames, 1)
    total_ms = sum(st_ms.values()) / max(st_frames, 1)
    # measured integer peaks of this device (the ALU roofline's denominator)
    with torch.cuda.stream(stream):
        int_peaks = {name: rs.rsgm_measure_int_peak(kind, stream) / 1e12
                     for kind, name in enumerate(rs.PEAK_NAMES)}
    int32_peak = min(int_peaks["i32_add"], int_peaks["i32_min"])
    achieved_tops = OPS_PER_CELL_PATH * cells_per_frame * N_PATHS / (agg_ms / 1e3) / 1e12
    result["stage_ms_per_step"] = {k: v / max(st_frames, 1) for k, v in st_ms.items()}
    result["int_peaks_tops"] = dict(int_peaks, note="measured by rsgm_measure_int_peak on this GPU (scalar operations "
                                                    "per second; a packed 16-bit-pair instruction counts two)")
    agg_kernel = ("k_lines (all 8 directions, one launch)" if gs_rows else
                  "k_lines (6 vertical and diagonal directions) beside k_rows (2 horizontal directions) "
                  "on a forked stream: the aggregation stage")
    result["roofline"] = {"kernel": agg_kernel, "bound": "alu", "achieved": achieved_tops,
                          "peak": int32_peak, "unit": "Tops/s", "frac": achieved_tops / int32_peak,
                          "frac_of_packed16_peak": achieved_tops / int_peaks["u16x2_mix"],
                          "traffic": (NCU_DRAM_BYTES_PER_CELL * cells_per_frame
                                      if NCU_DRAM_BYTES_PER_CELL and (B, gs_cells, gs_rows) == NCU_DRAM_CONFIG
                                      else None),
                          "traffic_unit": "bytes per launch (ncu per-cell figure of a 32-stream launch x this launch's cells)",
                          "peak_source": "measured: int32 add/min throughput (the slower of the two), "
                                         "rsgm_measure_int_peak",
                          "ops_per_cell_path": OPS_PER_CELL_PATH,
                          "share_of_step": agg_ms / total_ms if total_ms else None}
    # whole frame: max(algorithmic bytes / HBM peak, integer ops / integer peak) / measured time
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6783.5))
    px_step = B * W * H
    cells_step = result["cells_per_frame"] * B
    bytes_step = FRAME_BYTES_PER_PIXEL * px_step + FRAME_BYTES_PER_CELL * cells_step
    ops_step = FRAME_OPS_PER_CELL * cells_step
    t_bytes = bytes_step / (hbm * 1e9) * 1e3
    t_ops = ops_step / (int32_peak * 1e12) * 1e3
    result["frame_roofline"] = {"bytes_per_step": bytes_step, "int_ops_per_step": ops_step,
                                "t_bytes_ms": t_bytes, "t_int_ms": t_ops, "roofline_ms": max(t_bytes, t_ops),
                                "measured_ms": result["ms_per_step"],
                                "frac": max(t_bytes, t_ops) / result["ms_per_step"],
                                "frac_packed16": max(t_bytes, ops_step / (int_peaks["u16x2_mix"] * 1e12) * 1e3)
                                / result["ms_per_step"],
                                "hbm_peak_gbs": hbm, "int_peak_tops": int32_peak,
                                "counts": "23 B/pixel + 4 B/cell; 82 integer ops/cell (10 per path x 8 + 2 per cost)"}

    if not args.no_extras:
        # ---- e2e through the C ABI with host buffers (pinned), copies in the
        # timed region, on the same handles: one handle's copies overlap the
        # other handles' kernels.
        hl = left.cpu().pin_memory()
        hr = right.cpu().pin_memory()
        outd = torch.empty(B, H, W, dtype=torch.float32).pin_memory()
        outm = torch.empty(B, H, W, dtype=torch.uint8).pin_memory()
        start_parts(host=(hl, hr))
        run_parts(range(1, 1 + args.warmup), host=(hl, hr), out=(outd, outm))
        torch.cuda.synchronize()
        barrier()
        e2e_el = max_over_ranks(timed_parts(range(1 + args.warmup, nframes), host=(hl, hr), out=(outd, outm)))
        result["e2e"] = {"value": frames_all / e2e_el, "unit": "frames/s",
                         "h2d_bytes_per_step": 2 * B * H * W, "d2h_bytes_per_step": B * H * W * 5}

        # ---- plain form: full-range SGM + Kalman on every frame
        Pp = rs.rsgm_default_params(W, H, max_disp=D, radius=args.radius, batch=B,
                                    radius_mode=rs.RSGM_RADIUS_FULL)
        gp = rs.Stream(Pp, stream)
        nplain = min(5, steps)
        with torch.cuda.stream(stream):
            gp.full_frame(left[0], right[0])
            run(gp.handle, range(1, 3))
            gp.sync()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            run(gp.handle, range(3, 3 + nplain))
            p1.record(stream)
            torch.cuda.synchronize()
        gp.close()
        plain_el = max_over_ranks(p0.elapsed_time(p1) / 1e3)
        plain_fps = B * nplain * world / plain_el
        result["plain_form"] = {"value": plain_fps, "unit": "frames/s",
                                "cell_updates_per_s": B * nplain * world * W * H * D * N_PATHS / plain_el,
                                "speedup_of_reduced": value / plain_fps}

        # ---- single-stream per-frame latency
        P1s = rs.rsgm_default_params(W, H, max_disp=D, radius=args.radius, batch=1)
        g1 = rs.Stream(P1s, stream)
        lat = []
        with torch.cuda.stream(stream):
            g1.full_frame(left[0, 0], right[0, 0])
            rs.rsgm_reduced_frame(g1.handle, left[1, 0], right[1, 0], Rm[1, :1], tv[1, :1], K, BASE)
            rs.rsgm_autotune(g1.handle)
            sched1 = rs.rsgm_get_schedule(g1.handle)
            g1.full_frame(left[0, 0], right[0, 0])
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(nframes - 1)]
            for k in range(1, nframes):
                evs[k - 1][0].record(stream)
                rs.rsgm_reduced_frame(g1.handle, left[k, 0], right[k, 0], Rm[k, :1], tv[k, :1], K, BASE)
                evs[k - 1][1].record(stream)
            torch.cuda.synchronize()
        lat = sorted(a.elapsed_time(b) for a, b in evs[args.warmup:] or evs)
        # where a single stream's frame spends its time
        with torch.cuda.stream(stream):
            rs.rsgm_enable_stage_timing(g1.handle, True)
            for k in range(1, nframes):
                rs.rsgm_reduced_frame(g1.handle, left[k, 0], right[k, 0], Rm[k, :1], tv[k, :1], K, BASE)
            st1, n1 = rs.rsgm_stage_times(g1.handle)
        g1.close()
        q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
        result["latency_ms"] = {"p50": q(0.5), "p99": q(0.99), "frames": len(lat), "streams": 1,
                                "stage_ms": {k: v / max(n1, 1) for k, v in st1.items()},
                                "schedule_tuned": {"cells": sched1[0], "rows": "row sweep" if sched1[1] == 0
                                                   else "%d per warp" % sched1[1]}}

        # ---- after the path: 3x3 median output and moving-object boxes
        dp = rs.rsgm_default_detect_params()
        med = torch.empty(B, H, W, device=dev)
        with torch.cuda.stream(stream):
            rs.rsgm_median(gs.handle, med)
            rs.rsgm_detect(gs.handle, dp, B)
            gs.sync()
            t0 = time.perf_counter()
            for _ in range(5):
                rs.rsgm_median(gs.handle, med)
                boxes, counts = rs.rsgm_detect(gs.handle, dp, B)
            t_post = (time.perf_counter() - t0) / 5
        result["post_path"] = {"median_and_boxes_ms_per_step": 1e3 * t_post,
                               "boxes_per_stream": float(np.mean(counts)),
                               "note": "3x3 median + integral image + windows on the GPU, grouping on the host"}

        if rank == 0 and not args.no_next:
            # the configurations past the paper's path: the mixed-resolution
            # batch, the learned search window, the request loop
            result["mixed_group"] = mixed_group(args, dev, stream)
            from paper_1809_07986_gb300 import learned
            with torch.cuda.device(dev):
                nt = 2000 if args.learned else 512
                ev, theta = learned.run(train_frames=nt, eval_pairs=64, return_params=True)
                ev["note"] = ("trained on %d frames (config: 2000; bench.py --learned trains on all 2000); "
                              "held-out pairs, frame 1" % ev["train_frames"])
                result["learned_window"] = ev
                result["serving"] = serving_loop(dev, network=theta)
            result["path_ablation"] = path_ablation(dev)

        if rank == 0:
            result["cpu_baseline"] = cpu_baseline(args, left, right, Rm, tv, K)
    gs.close()
    for ph, _, _, _ in parts:
        ph.close()
    if rank == 0:
        print(json.dumps(result), flush=True)


def launch_ranks(n: int) -> int:
    """Runs this script as n ranks (one per GPU) under torch.distributed.run
    when it was started without a launcher; returns the launcher's status."""
    port = str(29500 + os.getpid() % 1000)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(n),
           "--master-addr", "127.0.0.1", "--master-port", port, os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    launched = "WORLD_SIZE" in os.environ
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if not launched and args.gpus > 1:
        sys.exit(launch_ranks(args.gpus))
    if world != args.gpus:
        raise SystemExit("bench.py: --gpus %d but the launcher started %d ranks" % (args.gpus, world))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
