"""Thin ctypes binding of librsgm (the C ABI declared in include/rsgm.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Functions keep the C names.  Tensors are passed by data pointer
(device tensors, or host tensors for the host-buffer entry points); a
non-zero status raises RsgmError.  The library must have been built
(``paper_1809_07986_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RSGM_OK = 0
RSGM_ERR_INVALID_ARG = -1
RSGM_ERR_NO_STATE = -2
RSGM_ERR_OOM = -3
RSGM_ERR_CUDA = -4
RSGM_ERR_TIMEOUT = -5
RSGM_ERR_CHECK_FAILED = -6

RSGM_RADIUS_FIXED = 0
RSGM_RADIUS_VARIANCE = 1
RSGM_RADIUS_FULL = 2
RSGM_RADIUS_LEARNED = 3
RSGM_CNN_PARAMS = 21414
RSGM_MAX_BATCH = 256
RSGM_MAX_DISP = 256

RSGM_BUF_CENSUS_L = 0
RSGM_BUF_CENSUS_R = 1
RSGM_BUF_WINDOW = 2
RSGM_BUF_OFFSET = 3
RSGM_BUF_CLASS = 4
RSGM_BUF_D_PRED = 5
RSGM_BUF_P_PRED = 6
RSGM_BUF_COST = 7
RSGM_BUF_AGGREGATED = 8
RSGM_BUF_D_MEAS = 9
RSGM_BUF_INNOVATION = 10
RSGM_BUF_CNN_INPUT = 11
RSGM_BUF_CNN_OUTPUT = 12
RSGM_BUF_RADIUS = 13
RSGM_BUF_R_MEAS = 14

RSGM_PEAK_I32_ADD = 0
RSGM_PEAK_I32_MIN = 1
RSGM_PEAK_U16X2_MIN = 2
RSGM_PEAK_U16X2_MIX = 3
PEAK_NAMES = ("i32_add", "i32_min", "u16x2_min", "u16x2_mix")

RSGM_SLOT_IDLE = 0
RSGM_SLOT_REDUCED = 1
RSGM_SLOT_FULL = 2

RSGM_STAGE_PREDICT = 0
RSGM_STAGE_SCAN = 1
RSGM_STAGE_CENSUS = 2
RSGM_STAGE_COST = 3
RSGM_STAGE_AGGREGATE = 4
RSGM_STAGE_UPDATE = 5
RSGM_NUM_STAGES = 6
STAGE_NAMES = ("predict", "scan", "census", "cost", "aggregate", "update")


class rsgm_params(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("max_disp", ctypes.c_int32),
        ("batch", ctypes.c_int32), ("census_w", ctypes.c_int32), ("census_h", ctypes.c_int32),
        ("path_mask", ctypes.c_uint32), ("radius_mode", ctypes.c_int32), ("radius", ctypes.c_int32),
        ("P1", ctypes.c_int32), ("P2", ctypes.c_int32), ("q", ctypes.c_float), ("r_meas", ctypes.c_float),
        ("p_reset", ctypes.c_float), ("tau_disc", ctypes.c_float), ("gate_gamma", ctypes.c_float),
    ]


RSGM_MAX_WINDOW_SIZES = 8
RSGM_BOX_COORD_LIMIT = 1 << 20


class rsgm_box(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("x1", ctypes.c_int32), ("y1", ctypes.c_int32)]


class rsgm_detect_params(ctypes.Structure):
    _fields_ = [("nsizes", ctypes.c_int32), ("sizes", (ctypes.c_int32 * 2) * RSGM_MAX_WINDOW_SIZES),
                ("stride", ctypes.c_int32), ("skip_num", ctypes.c_int32), ("skip_den", ctypes.c_int32),
                ("thresh_px", ctypes.c_float), ("iou_num", ctypes.c_int32), ("iou_den", ctypes.c_int32),
                ("min_area", ctypes.c_int32)]


class RsgmError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__("%s failed: %s (%d): %s" % (where, status_string(code), code, detail))
        self.code = code


_lib = None

# name -> (restype, argtypes); matches include/rsgm.h
_P = ctypes.c_void_p
SIGNATURES = {
    "rsgm_default_params": (ctypes.c_int, [ctypes.POINTER(rsgm_params), ctypes.c_int32, ctypes.c_int32]),
    "rsgm_init_stream": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(rsgm_params), _P]),
    "rsgm_footprint": (ctypes.c_int, [ctypes.POINTER(rsgm_params), ctypes.POINTER(ctypes.c_uint64)]),
    "rsgm_full_frame": (ctypes.c_int, [_P, _P, _P]),
    "rsgm_reduced_frame": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_float]),
    "rsgm_slot_frame": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_float]),
    "rsgm_state": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "rsgm_set_state": (ctypes.c_int, [_P, _P, _P]),
    "rsgm_read_buffer": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "rsgm_counters": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "rsgm_median": (ctypes.c_int, [_P, _P]),
    "rsgm_default_detect_params": (ctypes.c_int, [ctypes.POINTER(rsgm_detect_params)]),
    "rsgm_detect": (ctypes.c_int, [_P, ctypes.POINTER(rsgm_detect_params), _P, ctypes.c_int32, _P]),
    "rsgm_group_boxes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "rsgm_enable_stage_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "rsgm_stage_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "rsgm_window_offsets_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "rsgm_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "rsgm_set_schedule": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rsgm_set_rows_per_warp": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rsgm_get_schedule": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "rsgm_autotune_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "rsgm_group_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int32]),
    "rsgm_group_reduced_frame": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                                ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    "rsgm_group_destroy": (ctypes.c_int, [_P]),
    "rsgm_cnn_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P]),
    "rsgm_cnn_params": (ctypes.c_int, [_P, _P]),
    "rsgm_cnn_grad": (ctypes.c_int, [_P, _P]),
    "rsgm_cnn_destroy": (ctypes.c_int, [_P]),
    "rsgm_attach_cnn": (ctypes.c_int, [_P, _P]),
    "rsgm_cnn_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "rsgm_measure_int_peak": (ctypes.c_int, [ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "rsgm_sync": (ctypes.c_int, [_P]),
    "rsgm_destroy_stream": (ctypes.c_int, [_P]),
    "rsgm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rsgm_last_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads librsgm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError("librsgm.so is not built (%s); run paper_1809_07986_gb300.build.build() "
                              "or __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().rsgm_status_string(code).decode()


def last_error() -> str:
    return lib().rsgm_last_error().decode()


def _check(rc: int, where: str):
    if rc != RSGM_OK:
        raise RsgmError(rc, where, last_error())


def _ptr(x):
    """Pointer of a tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to librsgm must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to librsgm must be C-contiguous")
        return x.ctypes.data
    raise TypeError("cannot pass %r to librsgm" % type(x))


def _host_f32(x, n=None):
    import numpy as np
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1))
    if n is not None and a.size != n:
        raise ValueError("expected %d floats, got %d" % (n, a.size))
    return a


# ------------------------------------------------------------------ the C entry points

def rsgm_default_params(width: int, height: int, **overrides) -> rsgm_params:
    p = rsgm_params()
    _check(lib().rsgm_default_params(ctypes.byref(p), width, height), "rsgm_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError("rsgm_params has no field %r" % k)
        setattr(p, k, v)
    return p


def rsgm_footprint(params: rsgm_params) -> int:
    n = ctypes.c_uint64()
    _check(lib().rsgm_footprint(ctypes.byref(params), ctypes.byref(n)), "rsgm_footprint")
    return n.value


def rsgm_init_stream(params: rsgm_params, cuda_stream=None) -> int:
    """Returns the handle (an int).  cuda_stream: a torch.cuda.Stream, a raw
    cudaStream_t int, or None for the legacy default stream."""
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    h = _P()
    _check(lib().rsgm_init_stream(ctypes.byref(h), ctypes.byref(params), cuda_stream), "rsgm_init_stream")
    return h.value


def rsgm_full_frame(h: int, left, right):
    _check(lib().rsgm_full_frame(h, _ptr(left), _ptr(right)), "rsgm_full_frame")


def rsgm_reduced_frame(h: int, left, right, R, t, K, baseline: float):
    """R: B x 3 x 3, t: B x 3, K: 3 x 3 (host arrays or CPU tensors, float32),
    B = the handle's batch."""
    Ra = _host_f32(R)
    if Ra.size == 0 or Ra.size % 9:
        raise ValueError("R must hold B 3x3 matrices")
    ta = _host_f32(t, Ra.size // 3)
    Ka = _host_f32(K, 9)
    _check(lib().rsgm_reduced_frame(h, _ptr(left), _ptr(right), _ptr(Ra), _ptr(ta), _ptr(Ka),
                                    float(baseline)), "rsgm_reduced_frame")


def rsgm_slot_frame(h: int, roles, left, right, R, t, K, baseline: float):
    """roles: B values of RSGM_SLOT_IDLE / _REDUCED / _FULL; R: B x 3 x 3,
    t: B x 3, K: 3 x 3 (host arrays or CPU tensors)."""
    import numpy as np
    ro = np.ascontiguousarray(np.asarray(roles, np.uint8).reshape(-1))
    Ra = _host_f32(R)
    if Ra.size != 9 * ro.size:
        raise ValueError("R must hold one 3x3 matrix per slot")
    ta = _host_f32(t, 3 * ro.size)
    Ka = _host_f32(K, 9)
    _check(lib().rsgm_slot_frame(h, _ptr(ro), _ptr(left), _ptr(right), _ptr(Ra), _ptr(ta), _ptr(Ka),
                                 float(baseline)), "rsgm_slot_frame")


def rsgm_state(h: int, disp=None, var=None, moving_mask=None, disp_int=None):
    _check(lib().rsgm_state(h, _ptr(disp), _ptr(var), _ptr(moving_mask), _ptr(disp_int)), "rsgm_state")


def rsgm_set_state(h: int, disp, var):
    _check(lib().rsgm_set_state(h, _ptr(disp), _ptr(var)), "rsgm_set_state")


def rsgm_read_buffer(h: int, which: int, dst=None, capacity: int | None = None) -> int:
    """Copies buffer `which` into dst (if given); returns its size in bytes."""
    n = ctypes.c_size_t()
    if capacity is None:
        capacity = 0
        if dst is not None:
            capacity = dst.numel() * dst.element_size() if hasattr(dst, "numel") else dst.nbytes
    _check(lib().rsgm_read_buffer(h, which, _ptr(dst), capacity, ctypes.byref(n)), "rsgm_read_buffer")
    return n.value


def rsgm_counters(h: int):
    f, c, l = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().rsgm_counters(h, ctypes.byref(f), ctypes.byref(c), ctypes.byref(l)), "rsgm_counters")
    return f.value, c.value, l.value


def rsgm_median(h: int, out):
    _check(lib().rsgm_median(h, _ptr(out)), "rsgm_median")


def rsgm_default_detect_params(**overrides) -> rsgm_detect_params:
    p = rsgm_detect_params()
    _check(lib().rsgm_default_detect_params(ctypes.byref(p)), "rsgm_default_detect_params")
    for k, v in overrides.items():
        if k == "sizes":
            p.nsizes = len(v)
            for i, (w, hh) in enumerate(v):
                p.sizes[i][0], p.sizes[i][1] = w, hh
        else:
            setattr(p, k, v)
    return p


def rsgm_detect(h: int, params: rsgm_detect_params, batch: int, capacity: int = 256):
    """Returns a list (one per stream) of numpy arrays of boxes (x0, y0, x1, y1)."""
    import numpy as np
    boxes = np.zeros((batch, max(capacity, 1), 4), np.int32)
    counts = np.zeros(batch, np.int32)
    _check(lib().rsgm_detect(h, ctypes.byref(params), _ptr(boxes), capacity, _ptr(counts)), "rsgm_detect")
    return [boxes[b, :min(int(counts[b]), capacity)].copy() for b in range(batch)], counts


def rsgm_group_boxes(boxes, iou_num: int = 0, iou_den: int = 1, min_area: int = 0):
    """Groups (x0, y0, x1, y1) boxes given in window order (on the CPU);
    returns the kept boxes as an (m, 4) int32 array."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(boxes, np.int32).reshape(-1, 4))
    out = np.zeros((max(len(a), 1), 4), np.int32)
    cnt = ctypes.c_int32()
    _check(lib().rsgm_group_boxes(_ptr(a) if len(a) else None, len(a), iou_num, iou_den, min_area, _ptr(out),
                                  len(a), ctypes.byref(cnt)), "rsgm_group_boxes")
    return out[:cnt.value].copy()


def rsgm_enable_stage_timing(h: int, enable: bool = True):
    _check(lib().rsgm_enable_stage_timing(h, 1 if enable else 0), "rsgm_enable_stage_timing")


def rsgm_stage_times(h: int):
    """Returns ({stage name: ms summed over timed frames}, frames)."""
    ms = (ctypes.c_double * RSGM_NUM_STAGES)()
    n = ctypes.c_int32()
    _check(lib().rsgm_stage_times(h, ms, ctypes.byref(n)), "rsgm_stage_times")
    return dict(zip(STAGE_NAMES, list(ms))), n.value


def rsgm_window_offsets_noalloc(windows, width: int, rows: int, offsets, total=None, cuda_stream=None):
    """Ragged offsets of `windows` into `offsets` (device tensors) without any
    device allocation; see include/rsgm.h."""
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    _check(lib().rsgm_window_offsets_noalloc(_ptr(windows), width, rows, _ptr(offsets), _ptr(total),
                                             cuda_stream), "rsgm_window_offsets_noalloc")


def rsgm_autotune(h: int) -> int:
    n = ctypes.c_int32()
    _check(lib().rsgm_autotune(h, ctypes.byref(n)), "rsgm_autotune")
    return n.value


def rsgm_set_schedule(h: int, cells: int):
    _check(lib().rsgm_set_schedule(h, cells), "rsgm_set_schedule")


def rsgm_set_rows_per_warp(h: int, rows: int):
    _check(lib().rsgm_set_rows_per_warp(h, rows), "rsgm_set_rows_per_warp")


def rsgm_autotune_times(h: int) -> list:
    """[(cells, rows, ms per launch)] of every candidate the latest rsgm_autotune timed."""
    n = ctypes.c_int32()
    _check(lib().rsgm_autotune_times(h, None, None, None, 0, ctypes.byref(n)), "rsgm_autotune_times")
    k = n.value
    c, r, m = (ctypes.c_int32 * max(k, 1))(), (ctypes.c_int32 * max(k, 1))(), (ctypes.c_float * max(k, 1))()
    _check(lib().rsgm_autotune_times(h, c, r, m, k, ctypes.byref(n)), "rsgm_autotune_times")
    return [(c[i], r[i], m[i]) for i in range(k)]


def rsgm_get_schedule(h: int) -> tuple:
    """(register capacity in cells, rows: 0 = row sweep, else rows per warp)."""
    c, r = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().rsgm_get_schedule(h, ctypes.byref(c), ctypes.byref(r)), "rsgm_get_schedule")
    return c.value, r.value


def rsgm_group_create(handles) -> int:
    arr = (_P * len(handles))(*handles)
    g = _P()
    _check(lib().rsgm_group_create(ctypes.byref(g), arr, len(handles)), "rsgm_group_create")
    return g.value


def rsgm_group_reduced_frame(g: int, lefts, rights, Rs, ts, Ks, baselines):
    """Per member k: device images lefts[k], rights[k]; host R (B x 3 x 3),
    t (B x 3), K (3 x 3); baseline.  Host arrays are kept alive for the call."""
    import numpy as np
    n = len(lefts)
    keep = [_host_f32(x) for x in Rs] + [_host_f32(x) for x in ts] + [_host_f32(x, 9) for x in Ks]
    P = lambda xs: (_P * n)(*[_ptr(x) for x in xs])
    bl = np.ascontiguousarray(np.asarray(baselines, np.float32))
    _check(lib().rsgm_group_reduced_frame(g, P(lefts), P(rights), P(keep[:n]), P(keep[n:2 * n]),
                                          P(keep[2 * n:]), _ptr(bl)), "rsgm_group_reduced_frame")


def rsgm_group_destroy(g: int):
    _check(lib().rsgm_group_destroy(g), "rsgm_group_destroy")


def rsgm_cnn_create(params, cuda_stream=None) -> int:
    """params: RSGM_CNN_PARAMS floats (host array or CPU tensor)."""
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    a = _host_f32(params, RSGM_CNN_PARAMS)
    c = _P()
    _check(lib().rsgm_cnn_create(ctypes.byref(c), _ptr(a), cuda_stream), "rsgm_cnn_create")
    return c.value


def _cnn_vector(fn, c: int, where: str):
    import numpy as np
    out = np.zeros(RSGM_CNN_PARAMS, np.float32)
    _check(fn(c, _ptr(out)), where)
    return out


def rsgm_cnn_params(c: int):
    return _cnn_vector(lib().rsgm_cnn_params, c, "rsgm_cnn_params")


def rsgm_cnn_grad(c: int):
    return _cnn_vector(lib().rsgm_cnn_grad, c, "rsgm_cnn_grad")


def rsgm_cnn_destroy(c: int):
    _check(lib().rsgm_cnn_destroy(c), "rsgm_cnn_destroy")


def rsgm_attach_cnn(h: int, c: int):
    _check(lib().rsgm_attach_cnn(h, c), "rsgm_attach_cnn")


def rsgm_cnn_train_step(c: int, h: int, d_target, lr: float, want_loss: bool = True):
    """One training step against d_target (device, B*H*W floats); returns the
    loss (synchronises) or None."""
    loss = ctypes.c_float()
    _check(lib().rsgm_cnn_train_step(c, h, _ptr(d_target), float(lr), ctypes.byref(loss) if want_loss else None),
           "rsgm_cnn_train_step")
    return loss.value if want_loss else None


def rsgm_measure_int_peak(kind: int, cuda_stream=None) -> float:
    """Measured integer operations per second of the current device (see
    include/rsgm.h); synchronises the stream."""
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    v = ctypes.c_double()
    _check(lib().rsgm_measure_int_peak(kind, cuda_stream, ctypes.byref(v)), "rsgm_measure_int_peak")
    return v.value


def rsgm_sync(h: int):
    _check(lib().rsgm_sync(h), "rsgm_sync")


def rsgm_destroy_stream(h: int):
    _check(lib().rsgm_destroy_stream(h), "rsgm_destroy_stream")


def rsgm_status_string(code: int) -> str:
    return status_string(code)


def rsgm_last_error() -> str:
    return last_error()
