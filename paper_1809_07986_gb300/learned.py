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


def bad_vs_full(d, d_full) -> float:
    """Share of pixels whose disparity differs from the full-range result (the
    plain method on the same frames) by more than 3 px."""
    return float((np.abs(np.asarray(d, np.float64) - np.asarray(d_full, np.float64)) > 3.0).mean())


def evaluate(cnn, seeds, batch: int = 32, fixed_radius: int = 4, reps: int = 5, device="cuda", untrained=None):
    """Reduced frame 1 of the held-out pairs: the learned window against the
    fixed half-width (config 1's +-4 by default) and, if `untrained` holds a
    network, against that network.  Reports frames/s of the reduced frame
    (CUDA events, the full frame excluded), cells searched, and bad-pixel
    rates against the full-range result on the same frames (> 3 px) and
    against the renderer's ground truth (> 3 px and > 5 %)."""
    import torch
    from . import Stream
    cs = torch.cuda.current_stream()
    seeds = list(seeds)[: (len(seeds) // batch) * batch]
    arms = [("full", B.RSGM_RADIUS_FULL, None), ("fixed", B.RSGM_RADIUS_FIXED, None),
            ("learned", B.RSGM_RADIUS_LEARNED, cnn)]
    if untrained is not None:
        arms.append(("untrained", B.RSGM_RADIUS_LEARNED, untrained))
    out, full_d = {}, {}
    for name, mode, net in arms:
        st = Stream(B.rsgm_default_params(W, H, max_disp=D, batch=batch, radius_mode=mode, radius=fixed_radius), cs)
        if net is not None:
            B.rsgm_attach_cnn(st.handle, net)
        bad, badf, ms, cells = [], [], 0.0, 0
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
                if name == "full":
                    full_d[i] = d
                bad.append(bad_pixel_rate(d, gt[1].cpu().numpy()))
                badf.append(bad_vs_full(d, full_d[i]))
        finally:
            st.close()
        n = len(seeds) * reps
        out[name] = {"frames_per_s": n / (ms / 1e3), "cells_per_frame": cells / n,
                     "bad_vs_full": float(np.mean(badf)), "bad_pixel_rate_gt": float(np.mean(bad))}
    out["speedup"] = out["learned"]["frames_per_s"] / out["fixed"]["frames_per_s"]
    out["bad_vs_full_delta_pp"] = 100.0 * (out["learned"]["bad_vs_full"] - out["fixed"]["bad_vs_full"])
    out["bad_gt_delta_pp"] = 100.0 * (out["learned"]["bad_pixel_rate_gt"] - out["fixed"]["bad_pixel_rate_gt"])
    out["fixed_radius"] = fixed_radius
    return out


def run(train_frames: int = 2000, eval_pairs: int = 64, batch: int = 32, lr: float = 3e-3, epochs: int = 1,
        fixed_radius: int = 4, return_params: bool = False):
    """Trains on train_frames / 2 pairs (two frames each) and evaluates on
    held-out pairs against the fixed half-width and the untrained network.
    Returns the report, and with return_params also the trained parameters."""
    t0 = time.perf_counter()
    seeds = list(range(10_000, 10_000 + train_frames // 2))
    cnn, theta, losses = train(seeds, batch=batch, lr=lr, epochs=epochs)
    t1 = time.perf_counter()
    import torch
    untrained = B.rsgm_cnn_create(init_params(0), torch.cuda.current_stream())
    try:
        ev = evaluate(cnn, range(90_000, 90_000 + eval_pairs), batch=batch, fixed_radius=fixed_radius,
                      untrained=untrained)
    finally:
        B.rsgm_cnn_destroy(cnn)
        B.rsgm_cnn_destroy(untrained)
    ev.update(train_frames=2 * len(seeds) * epochs, train_s=t1 - t0, loss_first=losses[0] if losses else None,
              loss_last=losses[-1] if losses else None, steps=len(losses))
    return (ev, theta) if return_params else ev
