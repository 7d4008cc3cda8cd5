"""The integer-throughput microbenchmark (the denominator of the path sweep's
ALU roofline) returns rates that the device can physically reach: above a
tenth and below the ceiling of 128 scalar integer lanes per SM per clock
(twice that for packed 16-bit pairs)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


def test_integer_peaks_are_physical(rs):
    props = torch.cuda.get_device_properties(0)
    import subprocess
    try:
        mhz = float(subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                   capture_output=True, text=True, timeout=30).stdout.split()[0])
    except Exception:
        mhz = 2100.0
    lanes_per_s = props.multi_processor_count * 128 * mhz * 1e6
    rates = {name: rs.rsgm_measure_int_peak(kind) for kind, name in enumerate(rs.PEAK_NAMES)}
    print({k: "%.2f Tops/s" % (v / 1e12) for k, v in rates.items()})
    for name, v in rates.items():
        packed = name.startswith("u16x2")
        ceiling = lanes_per_s * (2.0 if packed else 1.0) * 1.05
        assert 0.1 * lanes_per_s < v <= ceiling, (name, v, ceiling)
