"""Oracle for the reduced-space SGM + per-pixel Kalman path (test infrastructure).

This package is TEST INFRASTRUCTURE.  It wraps ``rsgm_oracle.c`` -- a plain,
slow, single-threaded CPU restatement of the paper's definitions -- with ctypes
and chains its stages into one frame of the method.  Only ``tests/``, the
package smoke check (``__graft_entry__.smoke``) and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path and imports
nothing from it.

Stage-to-paper map (the paper is "Computationally efficient dense moving object
detection based on reduced space disparity estimation"):

* census, cost          -- Section 2.1 (census window and Hamming cost; 5x5, Table 1)
* aggregate             -- Section 2.2, Eq. 1 (P1 = 6, P2 = 65, Table 1)
* wta                   -- Section 2.3 (winner-takes-all)
* warp                  -- Section 2.4, Eqs. 2-4 (prediction through ego-motion)
* resolve               -- Section 2.4 (zoom-hole filling, discontinuity reset, search limits)
* kalman32 / kalman64   -- Section 2.4, Eqs. 5-6 (correction) + the innovation gate

Parity status: every stage above is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``.  The scene-level accuracy of the paper's Table 2
(KITTI) is not reproducible here and is unpinned.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsgm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, strict IEEE single precision, no FMA contraction."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u32, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint, ctypes.c_float
            L.orc_census_bits.argtypes = [i32, i32]
            L.orc_census_bits.restype = i32
            L.orc_census.argtypes = [P, i32, i32, i32, i32, P]
            L.orc_cost.argtypes = [P, P, i32, i32, i32, P, P, P, P]
            L.orc_offsets.argtypes = [P, i64, P]
            L.orc_offsets.restype = ctypes.c_uint64
            L.orc_aggregate_dir.argtypes = [P, i32, i32, P, P, P, i32, i32, i32, i32, P]
            L.orc_aggregate.argtypes = [P, i32, i32, P, P, P, ctypes.c_uint64, u32, i32, i32, P, P]
            L.orc_direction.argtypes = [i32, P, P]
            L.orc_wta.argtypes = [P, i64, P, P, P, P, P]
            L.orc_predict_variance.argtypes = [f32, f32, f32]
            L.orc_predict_variance.restype = f32
            L.orc_warp.argtypes = [P, P, i32, i32, P, P, P, f32, f32, P, P, P, P, P]
            L.orc_resolve.argtypes = [P, P, P, i32, i32, i32, i32, i32, f32, f32, P, P, P, P, P]
            L.orc_resolve_map.argtypes = [P, P, P, i32, i32, i32, i32, i32, P, f32, f32, P, P, P, P, P]
            L.orc_kalman_update32.argtypes = [f32, f32, i32, f32, f32, f32, P, P, P, P]
            L.orc_kalman32.argtypes = [P, P, P, P, i64, f32, f32, P, P, P, P]
            L.orc_kalman64.argtypes = [P, P, P, P, i64, f32, f32, P, P]
            L.orc_kalman32_rmap.argtypes = [P, P, P, P, i64, P, f32, P, P, P, P]
            L.orc_kalman64_rmap.argtypes = [P, P, P, P, i64, P, f32, P, P]
            L.orc_median3.argtypes = [P, i32, i32, P]
            L.orc_abs_innovation_q.argtypes = [P, P, i64, P]
            L.orc_integral.argtypes = [P, i32, i32, P]
            L.orc_windows.argtypes = [P, i32, i32, P, i32, i32, i32, ctypes.c_uint32, P, i32]
            L.orc_windows.restype = i32
            L.orc_merge_boxes.argtypes = [P, i32, i64, i64, i64]
            L.orc_merge_boxes.restype = i32
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


# Direction r = (dx, dy) of each path_mask bit; the predecessor of p is p - r.
DIRECTIONS = [(+1, 0), (-1, 0), (0, +1), (0, -1), (+1, +1), (-1, -1), (-1, +1), (+1, -1)]


@dataclasses.dataclass
class Params:
    """Parameters of the method.  Paper-fixed values: census 5x5, P1 = 6,
    P2 = 65, 8 paths, 128 disparities (Table 1).  The rest are readings."""
    width: int
    height: int
    max_disp: int = 128
    census_w: int = 5
    census_h: int = 5
    path_mask: int = 0xFF
    radius_mode: int = 0          # 0 fixed +-radius, 1 +-ceil(p), 2 full range (plain form), 3 per-pixel map
    radius: int = 4
    P1: int = 6
    P2: int = 65
    q: float = 0.15               # process noise: >99% within +-1 px (Section 3.1)
    r_meas: float = 1.0           # measurement noise
    p_reset: float | None = None  # default D^2/12: variance of a uniform over [0, D)
    tau_disc: float = 2.0
    gate_gamma: float = 6.635     # chi-square, 1 dof, 99 %

    def reset_variance(self) -> float:
        return float(self.max_disp) ** 2 / 12.0 if self.p_reset is None else float(self.p_reset)


# ---------------------------------------------------------------- stages

def census_bits(cw: int, ch: int) -> int:
    return lib().orc_census_bits(cw, ch)


def census(img: np.ndarray, cw: int = 5, ch: int = 5) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.uint64)
    lib().orc_census(_p(img), W, H, cw, ch, _p(out))
    return out


def offsets(wd: np.ndarray) -> tuple[np.ndarray, int]:
    wd = np.ascontiguousarray(wd, dtype=np.uint16)
    off = np.zeros(wd.shape, np.uint32)
    total = lib().orc_offsets(_p(wd), wd.size, _p(off))
    return off, int(total)


def _u16(a):
    return np.ascontiguousarray(a, dtype=np.uint16)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def cost(cl, cr, lo, wd, off, ncells, nbits):
    cl = np.ascontiguousarray(cl, np.uint64)
    cr = np.ascontiguousarray(cr, np.uint64)
    lo, wd, off = _u16(lo), _u16(wd), _u32(off)
    H, W = cl.shape
    out = np.zeros(max(ncells, 1), np.uint8)
    lib().orc_cost(_p(cl), _p(cr), W, H, nbits, _p(lo), _p(wd), _p(off), _p(out))
    return out[:ncells]


def aggregate_dir(cost_v, lo, wd, off, ncells, direction, P1, P2):
    lo, wd, off = _u16(lo), _u16(wd), _u32(off)
    H, W = lo.shape
    dx, dy = DIRECTIONS[direction]
    Lr = np.zeros(max(ncells, 1), np.uint16)
    c = np.ascontiguousarray(np.concatenate([np.asarray(cost_v, np.uint8), np.zeros(1, np.uint8)]))
    lib().orc_aggregate_dir(_p(c), W, H, _p(lo), _p(wd), _p(off), dx, dy, P1, P2, _p(Lr))
    return Lr[:ncells]


def aggregate(cost_v, lo, wd, off, ncells, path_mask, P1, P2):
    lo, wd, off = _u16(lo), _u16(wd), _u32(off)
    H, W = lo.shape
    S = np.zeros(max(ncells, 1), np.uint16)
    scratch = np.zeros(max(ncells, 1), np.uint16)
    c = np.ascontiguousarray(np.concatenate([np.asarray(cost_v, np.uint8), np.zeros(1, np.uint8)]))
    lib().orc_aggregate(_p(c), W, H, _p(lo), _p(wd), _p(off), ncells, path_mask, P1, P2,
                        _p(S), _p(scratch))
    return S[:ncells]


def wta(S, lo, wd, off):
    lo, wd, off = _u16(lo), _u16(wd), _u32(off)
    n = lo.size
    d_int = np.zeros(lo.shape, np.int16)
    d_z = np.zeros(lo.shape, np.float32)
    s = np.ascontiguousarray(np.concatenate([np.asarray(S, np.uint16), np.zeros(1, np.uint16)]))
    lib().orc_wta(_p(s), n, _p(lo), _p(wd), _p(off), _p(d_int), _p(d_z))
    return d_int, d_z


def predict_variance(phi: float, p: float, q: float) -> float:
    return lib().orc_predict_variance(phi, p, q)


def warp(d, p, Rm, t, K, b, q, per_source=False):
    d = np.ascontiguousarray(d, np.float32)
    p = np.ascontiguousarray(p, np.float32)
    H, W = d.shape
    Rm = np.ascontiguousarray(np.asarray(Rm, np.float32).reshape(9))
    t = np.ascontiguousarray(np.asarray(t, np.float32).reshape(3))
    K = np.ascontiguousarray(np.asarray(K, np.float32).reshape(9))
    d0 = np.zeros((H, W), np.float32)
    p0 = np.zeros((H, W), np.float32)
    known0 = np.zeros((H, W), np.uint8)
    tgt = np.zeros((H, W), np.int32) if per_source else None
    dn = np.zeros((H, W), np.float32) if per_source else None
    lib().orc_warp(_p(d), _p(p), W, H, _p(Rm), _p(t), _p(K), float(b), float(q),
                   _p(d0), _p(p0), _p(known0), _p(tgt), _p(dn))
    if per_source:
        return d0, p0, known0, tgt, dn
    return d0, p0, known0


def resolve(d0, p0, known0, D, radius_mode, radius, p_reset, tau_disc, radius_map=None):
    """Hole fill, reset and windows; radius_mode 3 takes the half-width of
    each predicted pixel from radius_map (uint8 H x W)."""
    H, W = d0.shape
    d_pred = np.zeros((H, W), np.float32)
    p_pred = np.zeros((H, W), np.float32)
    cls = np.zeros((H, W), np.uint8)
    lo = np.zeros((H, W), np.uint16)
    wd = np.zeros((H, W), np.uint16)
    rmap = None if radius_map is None else np.ascontiguousarray(radius_map, np.uint8)
    if radius_mode == 3 and rmap is None:
        raise ValueError("radius_mode 3 needs a radius map")
    lib().orc_resolve_map(_p(np.ascontiguousarray(d0, np.float32)), _p(np.ascontiguousarray(p0, np.float32)),
                          _p(np.ascontiguousarray(known0, np.uint8)), W, H, D, radius_mode, radius, _p(rmap),
                          float(p_reset), float(tau_disc), _p(d_pred), _p(p_pred), _p(cls), _p(lo), _p(wd))
    return d_pred, p_pred, cls, lo, wd


def kalman_update32(dp, pv, cls, dz, r, gamma):
    d, p, nu = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    m = ctypes.c_uint8()
    lib().orc_kalman_update32(dp, pv, cls, dz, r, gamma, ctypes.byref(d), ctypes.byref(p),
                              ctypes.byref(m), ctypes.byref(nu))
    return d.value, p.value, m.value, nu.value


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def kalman32(d_pred, p_pred, cls, d_z, r, gamma):
    """r: a scalar, or a float32 map of per-pixel measurement variances."""
    d_pred, p_pred, d_z = _f32(d_pred), _f32(p_pred), _f32(d_z)
    cls = np.ascontiguousarray(cls, np.uint8)
    shape = d_pred.shape
    n = d_pred.size
    d = np.zeros(shape, np.float32)
    p = np.zeros(shape, np.float32)
    mask = np.zeros(shape, np.uint8)
    nu = np.zeros(shape, np.float32)
    if np.ndim(r) == 0:
        lib().orc_kalman32(_p(d_pred), _p(p_pred), _p(cls), _p(d_z), n, float(r), gamma,
                           _p(d), _p(p), _p(mask), _p(nu))
    else:
        lib().orc_kalman32_rmap(_p(d_pred), _p(p_pred), _p(cls), _p(d_z), n, _p(_f32(r)), gamma,
                                _p(d), _p(p), _p(mask), _p(nu))
    return d, p, mask, nu


def kalman64(d_pred, p_pred, cls, d_z, r, gamma):
    d_pred, p_pred, d_z = _f32(d_pred), _f32(p_pred), _f32(d_z)
    cls = np.ascontiguousarray(cls, np.uint8)
    shape = d_pred.shape
    d = np.zeros(shape, np.float64)
    p = np.zeros(shape, np.float64)
    if np.ndim(r) == 0:
        lib().orc_kalman64(_p(d_pred), _p(p_pred), _p(cls), _p(d_z), d_pred.size, float(r), gamma, _p(d), _p(p))
    else:
        lib().orc_kalman64_rmap(_p(d_pred), _p(p_pred), _p(cls), _p(d_z), d_pred.size, _p(_f32(r)), gamma,
                                _p(d), _p(p))
    return d, p


# ---------------------------------------------------------------- one frame

def frame(P: Params, left: np.ndarray, right: np.ndarray, state=None, motion=None, radius_map=None,
          r_map=None):
    """One frame of the method for one camera stream.

    ``state`` is ``(d, p)`` of the previous frame (float32 H x W) and
    ``motion`` is ``(R, t, K, b)`` (X_k = R X_{k-1} + t).  Without a state the
    frame is the paper's initial one: the whole disparity range is searched and
    every pixel takes the measurement (Section 2.4, last paragraph).  With
    ``radius_map`` (uint8 H x W, used when P.radius_mode == 3) and ``r_map``
    (float32 H x W) the window half-width and the measurement variance are
    per pixel, as the learned window chooses them.  Returns a dict of every
    intermediate and the new state.
    """
    H, W, D = P.height, P.width, P.max_disp
    nbits = census_bits(P.census_w, P.census_h)
    cl = census(left, P.census_w, P.census_h)
    cr = census(right, P.census_w, P.census_h)
    out = {"census_l": cl, "census_r": cr}
    if state is None:
        lo = np.zeros((H, W), np.uint16)
        wd = np.full((H, W), D, np.uint16)
        cls = np.full((H, W), 2, np.uint8)
        d_pred = np.zeros((H, W), np.float32)
        p_pred = np.zeros((H, W), np.float32)
    else:
        Rm, t, K, b = motion
        d0, p0, known0 = warp(state[0], state[1], Rm, t, K, b, P.q)
        d_pred, p_pred, cls, lo, wd = resolve(d0, p0, known0, D, P.radius_mode, P.radius,
                                              P.reset_variance(), P.tau_disc, radius_map)
        out.update(d0=d0, p0=p0, known0=known0)
    off, n = offsets(wd)
    cv = cost(cl, cr, lo, wd, off, n, nbits)
    S = aggregate(cv, lo, wd, off, n, P.path_mask, P.P1, P.P2)
    d_int, d_z = wta(S, lo, wd, off)
    r = P.r_meas if r_map is None else _f32(r_map)
    d, p, mask, nu = kalman32(d_pred, p_pred, cls, d_z, r, P.gate_gamma)
    d64, p64 = kalman64(d_pred, p_pred, cls, d_z, r, P.gate_gamma)
    out.update(lo=lo, wd=wd, off=off, ncells=n, cls=cls, d_pred=d_pred, p_pred=p_pred,
               cost=cv, S=S, d_int=d_int, d_z=d_z, d=d, p=p, mask=mask, nu=nu,
               d64=d64, p64=p64)
    return out


# ---------------------------------------------------------------- after the path (Sections 2.3, 4)

def median3(d):
    d = _f32(d)
    H, W = d.shape
    out = np.zeros((H, W), np.float32)
    lib().orc_median3(_p(d), W, H, _p(out))
    return out


def abs_innovation_q(nu, cls):
    nu = _f32(nu)
    cls = np.ascontiguousarray(cls, np.uint8)
    a = np.zeros(nu.shape, np.uint32)
    lib().orc_abs_innovation_q(_p(nu), _p(cls), nu.size, _p(a))
    return a


def integral(a):
    a = np.ascontiguousarray(a, np.uint32)
    H, W = a.shape
    sat = np.zeros((H + 1, W + 1), np.uint64)
    lib().orc_integral(_p(a), W, H, _p(sat))
    return sat


def windows(sat, sizes, stride, y_min, thresh_q, cap=1 << 16):
    sat = np.ascontiguousarray(sat, np.uint64)
    H, W = sat.shape[0] - 1, sat.shape[1] - 1
    sz = np.ascontiguousarray(np.asarray(sizes, np.int32).reshape(-1))
    boxes = np.zeros((cap, 4), np.int32)
    n = lib().orc_windows(_p(sat), W, H, _p(sz), len(sz) // 2, stride, y_min, int(thresh_q), _p(boxes), cap)
    return boxes[:n].copy()


def merge_boxes(boxes, iou_num, iou_den, min_area):
    b = np.ascontiguousarray(np.asarray(boxes, np.int32).reshape(-1, 4)).copy()
    n = lib().orc_merge_boxes(_p(b), len(b), iou_num, iou_den, min_area)
    return b[:n].copy()


@dataclasses.dataclass
class DetectParams:
    """Moving-object boxes (Section 4).  Window sizes span the paper's 20x20
    to 50x75; the rest are readings."""
    sizes: tuple = ((20, 20), (30, 30), (40, 40), (50, 50), (50, 75))
    stride: int = 10
    skip_top_fraction_num: int = 1        # upper third skipped: y_min = H * 1 / 3
    skip_top_fraction_den: int = 3
    thresh_px: float = 1.0                # mean |d_pred - d_meas| of a detection window, px
    iou_num: int = 0                      # merge while some IoU > iou_num / iou_den
    iou_den: int = 1
    min_area: int = 1500                  # smaller boxes are discarded

    def y_min(self, H):
        return H * self.skip_top_fraction_num // self.skip_top_fraction_den

    def thresh_q(self):
        return int(np.floor(np.float32(self.thresh_px) * np.float32(16.0) + np.float32(0.5)))


def detect(nu, cls, D: DetectParams):
    H, W = nu.shape
    sat = integral(abs_innovation_q(nu, cls))
    raw = windows(sat, D.sizes, D.stride, D.y_min(H), D.thresh_q())
    return merge_boxes(raw, D.iou_num, D.iou_den, D.min_area), raw, sat
