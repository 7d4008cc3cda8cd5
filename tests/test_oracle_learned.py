"""Pins for the learned-window oracle (CPU only): bfloat16 rounding against
torch's conversion, the 3x3 correlation and the Sobel magnitude against
scipy, the gradients against central finite differences, Adam's first step
in closed form, the labels and the decision rule on constructed cases, and
the per-pixel radius / variance maps of the C oracle against its scalar
forms."""
import numpy as np
import pytest
import torch

from oracle import learned as L


def test_bf16_matches_torch_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 3, 5000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8)]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(L.bf16(x), want)
    # the tie 1 + 2^-8 rounds to even (1.0); 1 + 3 * 2^-8 rounds up to 1 + 2^-6
    assert L.bf16(np.float32(1.0 + 2 ** -8)) == 1.0
    assert L.bf16(np.float32(1.0 + 3 * 2 ** -8)) == np.float32(1.0 + 2 ** -6)


def test_conv3x3_matches_scipy_correlate():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 7, 9))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = L.conv3x3(x, W, b)
    for o in range(4):
        want = b[o] + sum(scipy_signal.correlate2d(x[i], W[o, i], mode="same", boundary="fill") for i in range(3))
        assert np.allclose(y[o], want, atol=1e-12)


def test_sobel_matches_scipy_with_nearest_border():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, (11, 13)).astype(np.uint8)
    gx = ndimage.sobel(img.astype(np.int32), axis=1, mode="nearest")
    gy = ndimage.sobel(img.astype(np.int32), axis=0, mode="nearest")
    assert np.array_equal(L.sobel_magnitude(img), np.abs(gx) + np.abs(gy))


def test_features_closed_forms():
    rng = np.random.default_rng(3)
    H, W, D, nbits = 5, 12, 16, 24
    left = rng.integers(0, 256, (H, W)).astype(np.uint8)
    cl = rng.integers(0, 1 << 24, (H, W)).astype(np.uint64)
    cr = rng.integers(0, 1 << 24, (H, W)).astype(np.uint64)
    d = rng.uniform(0, 10, (H, W)).astype(np.float32)
    p = rng.uniform(0.1, 50, (H, W)).astype(np.float32)
    known = rng.random((H, W)) > 0.2
    f = L.features(left, cl, cr, d, p, known, D, nbits)
    for y in range(H):
        for x in range(W):
            if not known[y, x]:
                assert (f[0, y, x], f[1, y, x], f[2, y, x]) == (0.0, 1.0, 1.0)
                continue
            assert f[0, y, x] == np.float32(d[y, x]) / np.float32(D)
            assert f[1, y, x] == np.sqrt(np.float32(p[y, x])) / np.float32(D)
            c = int(min(max(np.floor(d[y, x] + np.float32(0.5)), 0), D - 1))
            if x - c < 0:
                assert f[2, y, x] == 1.0
            else:
                ham = bin(int(cl[y, x]) ^ int(cr[y, x - c])).count("1")
                assert f[2, y, x] == np.float32(ham) / np.float32(nbits)
    assert f[3].min() >= 0 and f[3].max() <= 1


def _tiny_problem(seed, H=5, W=6, D=12):
    rng = np.random.default_rng(seed)
    theta = L.init_params(seed).astype(np.float64)
    theta[np.arange(theta.size) % 7 == 3] += 0.05          # non-zero biases too
    feats = rng.uniform(0, 1, (4, H, W))
    d_fill = rng.uniform(0, D - 1, (H, W))
    d_target = d_fill + rng.normal(0, 4, (H, W))
    valid = rng.random((H, W)) > 0.25
    return theta, feats, d_fill, d_target, valid, D


def _loss(theta, feats, d_fill, d_target, valid, D):
    _, out = L.forward(theta, feats, quant=False)
    return L.loss_and_grad(out, d_fill, d_target, valid, D)[0]


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    theta, feats, d_fill, d_target, valid, D = _tiny_problem(seed)
    acts, out = L.forward(theta, feats, quant=False)
    loss, g_out = L.loss_and_grad(out, d_fill, d_target, valid, D)
    grad = L.backward(theta, acts, g_out, quant=False)
    rng = np.random.default_rng(10 + seed)
    # every bias and a sample of weights of every layer
    idx = np.unique(np.concatenate([rng.choice(theta.size, 120, replace=False),
                                    np.cumsum([co * ci * 9 + co for ci, co in L.LAYERS]) - 1]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (_loss(theta + e, feats, d_fill, d_target, valid, D) -
              _loss(theta - e, feats, d_fill, d_target, valid, D)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_output_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    H, W, D = 3, 4, 12
    out = rng.normal(0, 2, (L.N_OUT, H, W))
    d_fill = rng.uniform(0, D - 1, (H, W))
    d_target = d_fill + rng.normal(0, 3, (H, W))
    valid = rng.random((H, W)) > 0.3
    _, g = L.loss_and_grad(out, d_fill, d_target, valid, D)
    h = 1e-6
    for c in range(L.N_OUT):
        for y in range(H):
            for x in range(W):
                e = np.zeros_like(out)
                e[c, y, x] = h
                fd = (L.loss_and_grad(out + e, d_fill, d_target, valid, D)[0] -
                      L.loss_and_grad(out - e, d_fill, d_target, valid, D)[0]) / (2 * h)
                assert abs(fd - g[c, y, x]) < 1e-8


def test_quantised_forward_rounds_only_at_the_stored_points():
    theta, feats, *_ = _tiny_problem(2)
    acts, out = L.forward(theta, feats, quant=True)
    for a in acts:   # every stored activation is a bfloat16 value
        assert np.array_equal(L.bf16(a.astype(np.float32)), a.astype(np.float32))
    acts64, out64 = L.forward(theta, feats, quant=False)
    # bfloat16 keeps 8 significant bits: the two forms stay close
    assert np.max(np.abs(out - out64)) < 0.05 * (1 + np.max(np.abs(out64)))


def test_adam_first_step_and_convergence():
    theta = np.array([1.0, -2.0, 0.5])
    m = np.zeros(3)
    v = np.zeros(3)
    g = np.array([0.3, -4.0, 1e-3])
    t1, _, _ = L.adam(theta, m, v, g, 1, lr=0.01)
    # bias-corrected first step: lr * g / (|g| + eps) ~ lr * sign(g)
    assert np.allclose(t1 - theta, -0.01 * g / (np.abs(g) + 1e-8))
    # minimises a quadratic
    x, m, v = np.array([3.0]), np.zeros(1), np.zeros(1)
    for k in range(1, 3001):
        x, m, v = L.adam(x, m, v, 2 * (x - 1.5), k, lr=0.01)
    assert abs(x[0] - 1.5) < 1e-3


def test_labels_pick_the_smallest_covering_radius():
    d_fill = np.array([[10.2, 10.2, 10.2, 10.2, 10.2, 0.4, 60.0]], np.float32)
    d_target = np.array([[10.6, 12.4, 14.0, 18.4, 40.0, 0.0, 63.7]], np.float32)
    # rounded distances: 1, 2, 4, 8, 30, 0, 3 (target 63.7 rounds to 64 -> clamped to 63)
    assert L.labels(d_fill, d_target, 64).tolist() == [[0, 1, 2, 3, 4, 0, 2]]


def test_decide_confidence_fallback_and_variance_clamp():
    out = np.zeros((L.N_OUT, 1, 4))
    out[1, 0, 0] = 10.0                     # class 1 (radius 2), confident
    out[3, 0, 1] = 1.0                      # class 3 but softmax ~0.40: falls back to 8
    out[4, 0, 2] = 10.0
    out[L.N_CLASSES, 0, 2] = 10.0           # r = e^10 -> clamped to 64
    out[L.N_CLASSES, 0, 3] = -10.0          # r -> clamped to 1/16
    radius, r, conf = L.decide(out)
    assert radius.tolist() == [[2, 8, 16, 8]]
    assert r[0, 2] == L.R_MAX and r[0, 3] == L.R_MIN and r[0, 0] == 1.0
    assert conf[0, 0] > 0.99 and conf[0, 1] < 0.9


def test_per_pixel_maps_reduce_to_the_scalar_forms(orc):
    import synth
    s = synth.tiny_pair(3)
    P = orc.Params(384, 128, max_disp=64, radius=4)
    L0, R0 = s["left"][0].numpy(), s["right"][0].numpy()
    f0 = orc.frame(P, L0, R0)
    motion = (s["R"][1].numpy(), s["t"][1].numpy(), s["K"].numpy(), s["baseline"])
    L1, R1 = s["left"][1].numpy(), s["right"][1].numpy()
    ref = orc.frame(P, L1, R1, state=(f0["d"], f0["p"]), motion=motion)
    P3 = orc.Params(384, 128, max_disp=64, radius=4, radius_mode=3)
    got = orc.frame(P3, L1, R1, state=(f0["d"], f0["p"]), motion=motion,
                    radius_map=np.full((128, 384), 4, np.uint8), r_map=np.full((128, 384), P.r_meas, np.float32))
    for k in ("lo", "wd", "cls", "S", "d_int", "d", "p", "mask", "nu", "d64", "p64"):
        assert np.array_equal(ref[k], got[k]), k
    # a per-pixel map takes each pixel's own half-width and variance
    rng = np.random.default_rng(0)
    rmap = rng.choice(np.array(L.RADII, np.uint8), (128, 384))
    rr = rng.uniform(0.2, 4.0, (128, 384)).astype(np.float32)
    mix = orc.frame(P3, L1, R1, state=(f0["d"], f0["p"]), motion=motion, radius_map=rmap, r_map=rr)
    c = np.clip(np.floor(mix["d_pred"] + np.float32(0.5)), 0, 63).astype(int)
    sel = mix["cls"] == 0
    want_lo = np.maximum(0, c - rmap.astype(int))
    want_hi = np.minimum(63, c + rmap.astype(int))
    assert np.array_equal(mix["lo"][sel], want_lo[sel])
    assert np.array_equal(mix["wd"][sel], (want_hi - want_lo + 1)[sel])
    d, p, m, nu = orc.kalman32(mix["d_pred"], mix["p_pred"], mix["cls"], mix["d_z"], rr, P.gate_gamma)
    assert np.array_equal(d, mix["d"]) and np.array_equal(p, mix["p"])
    unknown = mix["cls"] == 2
    assert np.array_equal(mix["p"][unknown], rr[unknown])
