"""Host logic of the learned-window driver (CPU only): its parameter
initialisation follows the layout the oracle and the C ABI share, and the
bad-pixel rule is the KITTI outlier rule."""
import numpy as np

from oracle import learned as LO
from paper_1809_07986_gb300 import binding, learned


def test_initial_parameters_follow_the_shared_layout():
    theta = learned.init_params(11)
    assert theta.dtype == np.float32 and theta.size == binding.RSGM_CNN_PARAMS == LO.n_params()
    # the same seeded draws in the same (out, in, ky, kx) order as the oracle's layout
    assert np.array_equal(theta, LO.init_params(11))
    layers = LO.unpack(theta)
    for (ci, co), (W, b) in zip(LO.LAYERS, layers):
        assert W.shape == (co, ci, 3, 3) and not b.any()
        assert abs(W.std() - np.sqrt(2.0 / (ci * 9))) < 0.25 * np.sqrt(2.0 / (ci * 9))


def test_bad_pixel_rate_is_the_kitti_outlier_rule():
    gt = np.array([[10.0, 10.0, 100.0, 100.0, 0.0, 50.0]])
    d = np.array([[13.5, 12.9, 104.0, 106.0, 80.0, 50.0]])
    # 3.5 px on 10 -> outlier; 2.9 px -> not; 4 px on 100 (4 %) -> not; 6 px on 100 (6 %) -> outlier;
    # no ground truth -> ignored
    assert learned.bad_pixel_rate(d, gt) == 2 / 5
