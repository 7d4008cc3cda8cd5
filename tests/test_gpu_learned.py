"""The learned search window on the GPU against the oracle (the config-1
pair: 384x128, D = 64).

Bars:
- the network inputs are bit-exact (single-precision quotients of exact
  integer and float inputs, then round-to-nearest-even bfloat16);
- the network output stays within a bfloat16 tolerance.  The device
  accumulates in fp32, in its own order, and the oracle in float64.  A
  stored activation can then round to the neighbouring bfloat16 value (one
  part in 2^8), which the later layers carry.  The bound is max |diff| <= 2 %
  of the output's range, mean |diff| <= 0.1 %;
- the decisions are identical wherever the oracle's are not within rounding
  of a threshold;
- the rest of the frame, given the decided half-widths and variances, is
  bit-exact (the same bars as every other frame);
- the gradients are within 5 % of each layer's largest gradient, and the
  loss within 0.5 %.  The same rounding flips are amplified by the bfloat16
  gradients;
- Adam steps on one frame lower the loss.
"""
import numpy as np
import pytest
import torch

from oracle import learned as LO
from parity_util import compare_stream, oracle_params, read_all

pytestmark = pytest.mark.gpu

H, W, D, NBITS = 128, 384, 64, 24


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


def _bf16_words_to_f32(words):
    return (np.asarray(words, np.uint16).astype(np.uint32) << 16).view(np.float32)


class Learned:
    """One learned handle that has run the full frame and one reduced frame of
    a tiny pair, with the oracle's view of the same frame."""

    def __init__(self, rs, orc, seed=1, cnn_seed=0):
        import synth
        s = synth.tiny_pair(seed)
        self.rs, self.orc = rs, orc
        self.P = rs.rsgm_default_params(W, H, max_disp=D, radius=4, radius_mode=rs.RSGM_RADIUS_LEARNED)
        self.theta = LO.init_params(cnn_seed)
        st = torch.cuda.current_stream()
        self.gs = rs.Stream(self.P, st)
        self.cnn = rs.rsgm_cnn_create(self.theta, st)
        rs.rsgm_attach_cnn(self.gs.handle, self.cnn)
        L, R = s["left"], s["right"]
        self.gs.full_frame(L[0].cuda().contiguous(), R[0].cuda().contiguous())
        self.motion = (s["R"][1].numpy(), s["t"][1].numpy(), s["K"].numpy(), s["baseline"])
        self.gs.reduced_frame(L[1].cuda().contiguous(), R[1].cuda().contiguous(), s["R"][1:2].contiguous(),
                              s["t"][1:2].contiguous(), s["K"], s["baseline"])
        self.gs.sync()
        # the oracle: first frame, the hole-filled prediction before resets, the inputs
        self.Po = oracle_params(orc, self.P)
        self.left1, self.right1 = L[1].numpy(), R[1].numpy()
        self.f0 = orc.frame(self.Po, L[0].numpy(), R[0].numpy())
        Rm, t, K, b = self.motion
        d0, p0, known0 = orc.warp(self.f0["d"], self.f0["p"], Rm, t, K, b, self.Po.q)
        self.d_fill, self.p_fill, cls_f, _, _ = orc.resolve(d0, p0, known0, D, 0, 4, self.Po.reset_variance(),
                                                            float("inf"))
        self.known = cls_f != 2
        cl = orc.census(self.left1, 5, 5)
        cr = orc.census(self.right1, 5, 5)
        self.feats = LO.features(self.left1, cl, cr, self.d_fill, self.p_fill, self.known, D, NBITS)

    def read(self, which, dtype, view):
        return self.gs.read(which, dtype).numpy().view(view)

    def close(self):
        self.gs.close()
        self.rs.rsgm_cnn_destroy(self.cnn)


@pytest.fixture(scope="module")
def frame(rs, orc):
    f = Learned(rs, orc)
    yield f
    f.close()


def test_inputs_are_bit_exact(rs, frame):
    got = _bf16_words_to_f32(frame.read(rs.RSGM_BUF_CNN_INPUT, torch.int16, np.uint16)).reshape(H * W, 16)
    want = LO.bf16(frame.feats).reshape(4, H * W).T
    np.testing.assert_array_equal(got[:, :4], want)
    assert not got[:, 4:].any()


def test_output_within_bfloat16_tolerance(rs, frame):
    out = frame.read(rs.RSGM_BUF_CNN_OUTPUT, torch.float32, np.float32).reshape(H * W, 8)[:, :LO.N_OUT]
    _, want = LO.forward(frame.theta, frame.feats, quant=True)
    want = want.reshape(LO.N_OUT, H * W).T
    scale = max(1.0, float(np.abs(want).max()))
    diff = np.abs(out.astype(np.float64) - want)
    assert diff.max() <= 0.02 * scale, diff.max()
    assert diff.mean() <= 1e-3 * scale, diff.mean()


def test_decisions_match_away_from_thresholds(rs, frame):
    out = frame.read(rs.RSGM_BUF_CNN_OUTPUT, torch.float32, np.float32).reshape(H * W, 8)
    radius = frame.read(rs.RSGM_BUF_RADIUS, torch.uint8, np.uint8)
    r_map = frame.read(rs.RSGM_BUF_R_MEAS, torch.float32, np.float32)
    # the oracle's rule applied to the device output (decision rounding only)
    o = out[:, :LO.N_OUT].T.reshape(LO.N_OUT, H, W).astype(np.float64)
    want_r, want_rm, conf = LO.decide(o)
    z = np.sort(o[:LO.N_CLASSES], axis=0)
    stable = (np.abs(conf - LO.CONFIDENCE) > 1e-5) & (z[-1] - z[-2] > 1e-5)
    assert stable.mean() > 0.99
    np.testing.assert_array_equal(radius.reshape(H, W)[stable], want_r[stable])
    assert np.allclose(r_map.reshape(H, W), want_rm, rtol=1e-5)
    assert set(np.unique(radius)) <= set(LO.RADII)


def test_frame_given_the_decisions_is_bit_exact(rs, orc, frame):
    radius = frame.read(rs.RSGM_BUF_RADIUS, torch.uint8, np.uint8).reshape(H, W)
    r_map = frame.read(rs.RSGM_BUF_R_MEAS, torch.float32, np.float32).reshape(H, W)
    o = orc.frame(frame.Po, frame.left1, frame.right1, state=(frame.f0["d"], frame.f0["p"]), motion=frame.motion,
                  radius_map=radius, r_map=r_map)
    g = read_all(rs, frame.gs)
    compare_stream(g, 0, o, H, W)
    # the learned half-widths reach the windows of predicted pixels
    sel = o["cls"] == 0
    c = np.clip(np.floor(o["d_pred"] + np.float32(0.5)), 0, D - 1).astype(int)
    assert np.array_equal(o["lo"][sel], np.maximum(0, c - radius.astype(int))[sel])


def _target(frame, seed=7):
    rng = np.random.default_rng(seed)
    t = frame.d_fill + rng.choice([-20.0, -6.0, -2.5, -0.4, 0.0, 0.3, 1.6, 3.2, 9.0, 17.0], frame.d_fill.shape)
    return np.clip(t, 0.0, D - 1.0).astype(np.float32)


def test_gradients_match_the_oracle(rs, frame):
    target = _target(frame)
    loss = rs.rsgm_cnn_train_step(frame.cnn, frame.gs.handle, torch.from_numpy(target).cuda(), 0.0)
    grad = rs.rsgm_cnn_grad(frame.cnn)
    cls = frame.read(rs.RSGM_BUF_CLASS, torch.uint8, np.uint8).reshape(H, W)
    acts, out = LO.forward(frame.theta, frame.feats, quant=True)
    loss_o, g_out = LO.loss_and_grad(out, frame.d_fill, target, cls == 0, D)
    grad_o = LO.backward(frame.theta, acts, g_out, quant=True)
    assert abs(loss - loss_o) <= 5e-3 * abs(loss_o), (loss, loss_o)
    k = 0
    for ci, co in LO.LAYERS:
        for n in (co * ci * 9, co):
            g, o = grad[k:k + n].astype(np.float64), grad_o[k:k + n]
            assert np.abs(g - o).max() <= 0.05 * np.abs(o).max() + 1e-12, (k, np.abs(g - o).max(), np.abs(o).max())
            k += n
    assert k == LO.n_params()
    # lr = 0 leaves the parameters as they were
    assert np.array_equal(rs.rsgm_cnn_params(frame.cnn), frame.theta)


def test_adam_steps_lower_the_loss(rs, orc):
    f = Learned(rs, orc, seed=2, cnn_seed=3)
    try:
        target = torch.from_numpy(_target(f, seed=3)).cuda()
        losses = [rs.rsgm_cnn_train_step(f.cnn, f.gs.handle, target, 3e-3) for _ in range(25)]
        assert losses[-1] < 0.8 * losses[0], losses
        assert not np.array_equal(rs.rsgm_cnn_params(f.cnn), f.theta)
    finally:
        f.close()


def test_learned_mode_needs_a_network_and_a_learned_frame(rs):
    P = rs.rsgm_default_params(64, 32, max_disp=16, radius_mode=rs.RSGM_RADIUS_LEARNED)
    z = torch.zeros(32, 64, dtype=torch.uint8, device="cuda")
    K = torch.tensor([[30.0, 0, 31.5], [0, 30.0, 15.5], [0, 0, 1]])
    st = torch.cuda.current_stream()
    with rs.Stream(P, st) as s:
        s.full_frame(z, z)
        with pytest.raises(rs.RsgmError) as e:
            s.reduced_frame(z, z, torch.eye(3)[None], torch.zeros(1, 3), K, 0.5)
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG
        c = rs.rsgm_cnn_create(LO.init_params(0), st)
        try:
            rs.rsgm_attach_cnn(s.handle, c)
            with pytest.raises(rs.RsgmError) as e:
                rs.rsgm_cnn_train_step(c, s.handle, torch.zeros(32 * 64, device="cuda"), 0.0)
            assert e.value.code == rs.RSGM_ERR_NO_STATE
            s.reduced_frame(z, z, torch.eye(3)[None], torch.zeros(1, 3), K, 0.5)
            s.sync()
            with pytest.raises(rs.RsgmError) as e:
                rs.rsgm_group_create([s.handle])
            assert e.value.code == rs.RSGM_ERR_INVALID_ARG
        finally:
            s.close()
            rs.rsgm_cnn_destroy(c)


def test_training_driver_runs_end_to_end(rs):
    # the module that orders training and evaluation calls (2 steps, 1 batch)
    from paper_1809_07986_gb300 import learned
    cnn, theta, losses = learned.train(list(range(500, 508)), batch=4, lr=3e-3)
    try:
        assert len(losses) == 2 and all(np.isfinite(losses))
        assert theta.shape == (rs.RSGM_CNN_PARAMS,)
        ev = learned.evaluate(cnn, range(600, 604), batch=4, reps=1)
    finally:
        rs.rsgm_cnn_destroy(cnn)
    for k in ("learned", "fixed", "full"):
        assert ev[k]["frames_per_s"] > 0 and 0.0 <= ev[k]["bad_pixel_rate_gt"] <= 1.0
        assert 0.0 <= ev[k]["bad_vs_full"] <= 1.0 and ev[k]["cells_per_frame"] > 0
    assert ev["full"]["bad_vs_full"] == 0.0 and ev["fixed_radius"] == 4


def test_trained_network_gains_over_the_untrained_network_and_the_fixed_window(rs):
    # 512 training frames (16 steps of 32 pairs' frames), then held-out pairs:
    # the trained network searches fewer cells than the untrained one (which
    # falls back to +-8 almost everywhere) and than the fixed +-4 window of the
    # tiny configuration, with at most 0.5 percentage points more pixels that
    # differ from the full-range result by more than 3 px.
    from paper_1809_07986_gb300 import learned
    cnn, theta, losses = learned.train(list(range(10_000, 10_256)), batch=32)
    untrained = rs.rsgm_cnn_create(learned.init_params(0), torch.cuda.current_stream())
    try:
        ev = learned.evaluate(cnn, range(90_000, 90_064), batch=32, reps=1, fixed_radius=4, untrained=untrained)
    finally:
        rs.rsgm_cnn_destroy(cnn)
        rs.rsgm_cnn_destroy(untrained)
    print({k: (round(v["cells_per_frame"]), round(100 * v["bad_vs_full"], 3)) for k, v in ev.items()
           if isinstance(v, dict)})
    assert losses[-1] < 0.5 * losses[0]
    assert ev["learned"]["cells_per_frame"] < 0.6 * ev["untrained"]["cells_per_frame"]
    assert ev["learned"]["cells_per_frame"] < 0.8 * ev["fixed"]["cells_per_frame"]
    assert ev["learned"]["bad_vs_full"] <= ev["fixed"]["bad_vs_full"] + 0.005
