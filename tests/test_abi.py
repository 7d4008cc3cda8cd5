"""C-ABI checks that need no GPU: the library loads, exports every function the
header declares, the binding covers them, and argument errors are reported
before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsgm.h")


@pytest.fixture(scope="module")
def rs():
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    rs.lib()
    return rs


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsgm_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function(rs):
    names = header_functions()
    assert len(names) >= 12
    L = ctypes.CDLL(rs.binding.library_path())
    for n in names:
        assert hasattr(L, n), n
    assert sorted(rs.binding.SIGNATURES) == names


def test_header_constants_match_the_binding(rs):
    text = open(HEADER).read()
    for name, val in re.findall(r"#define (RSGM_[A-Z_0-9]+) \(?(-?\d+)\)?", text):
        assert getattr(rs.binding, name) == int(val), name


def test_params_struct_layout(rs):
    text = open(HEADER).read()
    body = text[text.index("typedef struct {"): text.index("} rsgm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-zA-Z_0-9]+)\s*[,;]", body)
    assert [f for f, _ in rs.rsgm_params._fields_] == fields
    assert ctypes.sizeof(rs.rsgm_params) == 4 * len(fields)


def test_defaults_follow_table_1(rs):
    p = rs.rsgm_default_params(1242, 375)
    assert (p.census_w, p.census_h, p.P1, p.P2, p.max_disp, p.path_mask) == (5, 5, 6, 65, 128, 0xFF)
    assert p.batch == 1 and p.radius_mode == rs.RSGM_RADIUS_FIXED


@pytest.mark.parametrize("field,value", [
    ("width", 0), ("height", -3), ("max_disp", 0), ("max_disp", 257), ("batch", 0), ("batch", 257),
    ("census_w", 4), ("census_h", 17), ("path_mask", 0), ("path_mask", 0x100), ("radius_mode", 4),
    ("radius", -1), ("P1", -1), ("P2", 5000), ("r_meas", 0.0), ("q", -1.0), ("gate_gamma", 0.0),
])
def test_bad_parameters_are_rejected_before_device_work(rs, field, value):
    p = rs.rsgm_default_params(64, 32)
    setattr(p, field, value)
    h = ctypes.c_void_p(123)
    rc = rs.lib().rsgm_init_stream(ctypes.byref(h), ctypes.byref(p), None)
    assert rc == rs.RSGM_ERR_INVALID_ARG
    assert h.value is None
    assert rs.last_error()


def test_too_many_cells_is_rejected(rs):
    p = rs.rsgm_default_params(4096, 4096, max_disp=256)
    h = ctypes.c_void_p()
    assert rs.lib().rsgm_init_stream(ctypes.byref(h), ctypes.byref(p), None) == rs.RSGM_ERR_INVALID_ARG
    assert "2^32" in rs.last_error()


def test_null_arguments(rs):
    L = rs.lib()
    assert L.rsgm_init_stream(None, None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_full_frame(None, None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_reduced_frame(None, None, None, None, None, None, 0.5) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_state(None, None, None, None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_set_state(None, None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_read_buffer(None, 0, None, 0, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_counters(None, None, None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_sync(None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_destroy_stream(None) == rs.RSGM_OK
    assert L.rsgm_default_params(None, 1, 1) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_slot_frame(None, None, None, None, None, None, None, 0.5) == rs.RSGM_ERR_INVALID_ARG
    v = ctypes.c_double()
    assert L.rsgm_measure_int_peak(7, None, ctypes.byref(v)) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_measure_int_peak(rs.RSGM_PEAK_I32_ADD, None, None) == rs.RSGM_ERR_INVALID_ARG


def test_status_strings(rs):
    for code in range(-6, 1):
        assert rs.status_string(code) not in ("", "unknown status")
    assert rs.status_string(-99) == "unknown status"


def test_no_gpu_gives_a_cuda_status_not_a_crash(rs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = rs.rsgm_default_params(64, 32)
    with pytest.raises(rs.RsgmError) as e:
        rs.rsgm_init_stream(p)
    assert e.value.code == rs.RSGM_ERR_CUDA


def test_cnn_parameter_count_matches_the_oracle_layout(rs):
    from oracle import learned
    assert rs.RSGM_CNN_PARAMS == learned.n_params()


def test_cnn_entry_points_reject_null_before_device_work(rs):
    L = rs.lib()
    c = ctypes.c_void_p()
    assert L.rsgm_cnn_create(ctypes.byref(c), None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_cnn_create(None, None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_attach_cnn(None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_cnn_train_step(None, None, None, 0.0, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_cnn_params(None, None) == rs.RSGM_ERR_INVALID_ARG
    assert L.rsgm_cnn_destroy(None) == rs.RSGM_OK
