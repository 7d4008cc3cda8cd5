"""GB300-native reduced-space SGM with per-pixel Kalman fusion.

The compute path is librsgm (hand-written CUDA for sm_103a behind the C ABI in
include/rsgm.h); this package is its thin Python binding plus the in-tree
build.  ``Stream`` is a small convenience wrapper around one handle.
"""
from __future__ import annotations

from .binding import *  # noqa: F401,F403
from .binding import (RsgmError, lib, rsgm_counters, rsgm_default_params, rsgm_destroy_stream,
                      rsgm_full_frame, rsgm_init_stream, rsgm_read_buffer, rsgm_reduced_frame,
                      rsgm_set_state, rsgm_state, rsgm_sync)


class Stream:
    """One librsgm handle: B camera streams of one geometry on one CUDA stream."""

    def __init__(self, params, cuda_stream=None):
        self.params = params
        self.handle = rsgm_init_stream(params, cuda_stream)

    @property
    def shape(self):
        p = self.params
        return (p.batch, p.height, p.width)

    def full_frame(self, left, right):
        rsgm_full_frame(self.handle, left, right)

    def reduced_frame(self, left, right, R, t, K, baseline):
        if R.numel() != 9 * self.params.batch or t.numel() != 3 * self.params.batch:
            raise ValueError("R and t must hold one motion per stream (batch %d)" % self.params.batch)
        rsgm_reduced_frame(self.handle, left, right, R, t, K, baseline)

    def state(self, device="cuda"):
        """Returns (d, p, mask, d_int) as new tensors on `device`."""
        import torch
        shp = self.shape
        d = torch.empty(shp, dtype=torch.float32, device=device)
        p = torch.empty(shp, dtype=torch.float32, device=device)
        m = torch.empty(shp, dtype=torch.uint8, device=device)
        di = torch.empty(shp, dtype=torch.int16, device=device)
        rsgm_state(self.handle, d, p, m, di)
        rsgm_sync(self.handle)
        return d, p, m, di

    def set_state(self, d, p):
        rsgm_set_state(self.handle, d, p)

    def read(self, which, dtype):
        """Copies an intermediate buffer into a new CPU tensor of `dtype`."""
        import torch
        n = rsgm_read_buffer(self.handle, which)
        esz = torch.empty(0, dtype=dtype).element_size()
        out = torch.empty(n // esz, dtype=dtype)
        rsgm_read_buffer(self.handle, which, out)
        return out

    def counters(self):
        return rsgm_counters(self.handle)

    def sync(self):
        rsgm_sync(self.handle)

    def close(self):
        if self.handle:
            rsgm_destroy_stream(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
