"""Training and evaluation of the learned search window.

Two modes of the same seeded sequences are run side by side:
- a full-range handle (``RSGM_RADIUS_FULL``): full-range SGM plus the Kalman
  correction on every frame, whose state is the training target;
- a learned handle (``RSGM_RADIUS_LEARNED``) with the network attached,
  trained against that target after each of its reduced frames.

Every step runs in librsgm's kernels (the network's forward and backward
passes included); this module only orders the calls.  Sequences are the
seeded 384 x 128 pairs of ``synth.tiny_pair``: D = 64, frame 1 after a 0.5 m
forward motion with one box moving on its own.  Each pair gives one training
frame per stream.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B

W, H, D = 384, 128, 64


def init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters in the order of the C ABI (He-normal weights,
    zero biases), from the shared seeded generators."""
    import synth
    theta = synth.network_params(seed)
    assert theta.size == B.RSGM_CNN_PARAMS
    return theta


def pairs(seeds, device):
    """Stacked tiny pairs: left, right [2, B, H, W] u8, gt [2, B, H, W], R [B,3,3], t [B,3], K, baseline."""
    import torch
    import synth
    ss = [synth.tiny_pair(int(s), device=device) for s in seeds]
    st = lambda k: torch.stack([x[k] for x in ss], 1).contiguous()
    return (st("left"), st("right"), st("disp"), torch.stack([x["R"][1] for x in ss]).contiguous(),
            torch.stack([x["t"][1] for x in ss]).contiguous(), ss[0]["K"], ss[0]["baseline"])


def _run_pair(stream, left, right, R, t, K, b):
    stream.full_frame(left[0], right[0])
    stream.reduced_frame(left[1], right[1], R, t, K, b)


def train(seeds, batch: int = 32, lr: float = 3e-3, epochs: int = 1, params=None, seed: int = 0, device="cuda"):
    """Trains a network on the pairs of `seeds` (batch streams per step).
    Returns (cnn handle, parameters, per-step losses).  The caller destroys
    the network."""
    import torch
    from . import Stream
    cs = torch.cuda.current_stream()
    theta = init_params(seed) if params is None else np.asarray(params, np.float32)
    cnn = B.rsgm_cnn_create(theta, cs)
    full = Stream(B.rsgm_default_params(W, H, max_disp=D, batch=batch, radius_mode=B.RSGM_RADIUS_FULL), cs)
    lrn = Stream(B.rsgm_default_params(W, H, max_disp=D, batch=batch, radius_mode=B.RSGM_RADIUS_LEARNED), cs)
    B.rsgm_attach_cnn(lrn.handle, cnn)
    losses = []
    target = torch.empty(batch, H, W, dtype=torch.float32, device=device)
    try:
        for _ in range(epochs):
            for i in range(0, len(seeds) - batch + 1, batch):
                L, R, _, Rm, tv, K, b = pairs(seeds[i:i + batch], device)
                _run_pair(full, L, R, Rm, tv, K, b)
                B.rsgm_state(full.handle, target)
                _run_pair(lrn, L, R, Rm, tv, K, b)
                losses.append(B.rsgm_cnn_train_step(cnn, lrn.handle, target, lr))
        theta = B.rsgm_cnn_params(cnn)
    finally:
        full.close()
        lrn.close()
    return cnn, theta, losses


def bad_pixel_rate(d, gt) -> float:
    """Share of pixels with ground truth whose error exceeds 3 px and 5 % of the
    true disparity (the KITTI outlier rule)."""
    d = np.asarray(d, np.float64)
    gt = np.asarray(gt, np.float64)
    ok = gt > 0
    err = np.abs(d - gt)
    return float(((err > 3.0) & (err > 0.05 * gt) & ok).sum() / max(ok.sum(), 1))


def evaluate(cnn, seeds, batch: int = 32, fixed_radius: int = 8, reps: int = 5, device="cuda"):
    """Reduced frame 1 of the held-out pairs, learned window against the fixed
    half-width: frames/s of the reduced frame (CUDA events, the full frame
    excluded) and bad-pixel rates against the renderer's ground truth."""
    import torch
    from . import Stream
    cs = torch.cuda.current_stream()
    seeds = list(seeds)[: (len(seeds) // batch) * batch]
    out = {}
    for name in ("learned", "fixed"):
        mode = B.RSGM_RADIUS_LEARNED if name == "learned" else B.RSGM_RADIUS_FIXED
        st = Stream(B.rsgm_default_params(W, H, max_disp=D, batch=batch, radius_mode=mode, radius=fixed_radius), cs)
        if name == "learned":
            B.rsgm_attach_cnn(st.handle, cnn)
        bad, ms, cells = [], 0.0, 0
        try:
            for i in range(0, len(seeds), batch):
                L, R, gt, Rm, tv, K, b = pairs(seeds[i:i + batch], device)
                for _ in range(reps):
                    st.full_frame(L[0], R[0])
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    c0 = st.counters()[1]
                    e0.record(cs)
                    st.reduced_frame(L[1], R[1], Rm, tv, K, b)
                    e1.record(cs)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                    cells += st.counters()[1] - c0
                d = st.state()[0].cpu().numpy()
                bad.append(bad_pixel_rate(d, gt[1].cpu().numpy()))
        finally:
            st.close()
        n = len(seeds) * reps
        out[name] = {"frames_per_s": n / (ms / 1e3), "cells_per_frame": cells / n,
                     "bad_pixel_rate": float(np.mean(bad))}
    out["speedup"] = out["learned"]["frames_per_s"] / out["fixed"]["frames_per_s"]
    out["bad_pixel_delta_pp"] = 100.0 * (out["learned"]["bad_pixel_rate"] - out["fixed"]["bad_pixel_rate"])
    out["fixed_radius"] = fixed_radius
    return out


def run(train_frames: int = 2000, eval_pairs: int = 64, batch: int = 32, lr: float = 3e-3, epochs: int = 1):
    """Trains on train_frames / 2 pairs (two frames each) and evaluates on held-out pairs."""
    t0 = time.perf_counter()
    seeds = list(range(10_000, 10_000 + train_frames // 2))
    cnn, theta, losses = train(seeds, batch=batch, lr=lr, epochs=epochs)
    t1 = time.perf_counter()
    try:
        ev = evaluate(cnn, range(90_000, 90_000 + eval_pairs), batch=batch)
    finally:
        B.rsgm_cnn_destroy(cnn)
    ev.update(train_frames=2 * len(seeds) * epochs, train_s=t1 - t0, loss_first=losses[0] if losses else None,
              loss_last=losses[-1] if losses else None, steps=len(losses))
    return ev
