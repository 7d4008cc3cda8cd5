"""Oracle for the learned search window (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import
this module; the library never does.  Plain numpy, float64 arithmetic, with
values rounded to bfloat16 exactly where the device stores bfloat16.

The paper fixes the search range per pixel from the predicted variance
(Section 2.4: a window of d_pred +- p).  The learned variant replaces that
rule by a small per-pixel network that picks the half-width from {1, 2, 4, 8,
16} and a measurement variance r, from four inputs: the predicted disparity,
the predicted variance, the census residual at the predicted disparity and
the image gradient magnitude.  The readings (feature scaling, labels, loss,
confidence fallback) are this module's and are listed with the design notes.

Layout: activations are (channels, H, W) float arrays; layer l has weights
W[l] of shape (out, in, 3, 3) (cross-correlation, zero padding) and bias b[l].
"""
from __future__ import annotations

import numpy as np

RADII = (1, 2, 4, 8, 16)        # radius classes
N_CLASSES = len(RADII)
N_OUT = N_CLASSES + 1           # class logits, then the log measurement variance
LAYERS = ((4, 32), (32, 32), (32, 32), (32, N_OUT))   # (in, out) channels, 3x3 each
CONFIDENCE = 0.9                # below this softmax probability the window falls back
FALLBACK_RADIUS = 8
R_MIN, R_MAX = 1.0 / 16.0, 64.0  # clamp of the learned measurement variance
SOBEL_SCALE = 2040.0            # |gx| + |gy| <= 2 * 4 * 255
NLL_WEIGHT = 0.1                # weight of the variance term in the loss


# ---------------------------------------------------------------- parameters

def n_params() -> int:
    return sum(co * ci * 9 + co for ci, co in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W (out, in, 3, 3), b (out,)), ...] float64.
    Order: layer by layer, the weights in (out, in, ky, kx) order, then the bias."""
    theta = np.asarray(theta, np.float64)
    out, k = [], 0
    for ci, co in LAYERS:
        W = theta[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    assert k == theta.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in layers])


def init_params(seed: int) -> np.ndarray:
    """The seeded initial parameters (from the shared input generators)."""
    import synth
    return synth.network_params(seed, LAYERS)


# ---------------------------------------------------------------- bfloat16

def bf16(x) -> np.ndarray:
    """Rounds float32 values to bfloat16 (nearest, ties to even); returns float32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


# ---------------------------------------------------------------- inputs

def sobel_magnitude(img) -> np.ndarray:
    """|gx| + |gy| of the 3x3 Sobel operator, coordinates clamped at the border (int32)."""
    I = np.pad(np.asarray(img, np.int32), 1, mode="edge")
    H, W = img.shape
    s = lambda dy, dx: I[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    gx = (s(-1, 1) + 2 * s(0, 1) + s(1, 1)) - (s(-1, -1) + 2 * s(0, -1) + s(1, -1))
    gy = (s(1, -1) + 2 * s(1, 0) + s(1, 1)) - (s(-1, -1) + 2 * s(-1, 0) + s(-1, 1))
    return np.abs(gx) + np.abs(gy)


def popcount64(a) -> np.ndarray:
    a = np.asarray(a, np.uint64)
    return np.unpackbits(a.view(np.uint8).reshape(a.shape + (8,)), axis=-1).sum(-1).astype(np.int64)


def features(left, cen_l, cen_r, d_fill, p_fill, known, D: int, nbits: int) -> np.ndarray:
    """The four inputs per pixel (float32, shape (4, H, W)), from the hole-filled
    prediction before the discontinuity reset:
      0  d / D                 (0 without a prediction)
      1  sqrt(p) / D           (1 without a prediction)
      2  census Hamming distance at the rounded predicted disparity / nbits
         (1 without a prediction or when the match falls left of the image)
      3  (|gx| + |gy|) / 2040  (Sobel on the left image)
    Every quotient is one float32 division, as on the device."""
    d = np.asarray(d_fill, np.float32)
    p = np.asarray(p_fill, np.float32)
    known = np.asarray(known, bool)
    H, W = d.shape
    fD = np.float32(D)
    f0 = np.where(known, d / fD, np.float32(0))
    f1 = np.where(known, np.sqrt(np.where(known, p, np.float32(0))) / fD, np.float32(1))
    cf = np.floor(d + np.float32(0.5))
    c = np.clip(cf, 0, D - 1).astype(np.int64)
    xs = np.arange(W)[None, :] - c
    ok = known & (xs >= 0)
    rows = np.arange(H)[:, None].repeat(W, 1)
    ham = popcount64(np.asarray(cen_l, np.uint64) ^ np.asarray(cen_r, np.uint64)[rows, np.clip(xs, 0, W - 1)])
    f2 = np.where(ok, ham.astype(np.float32) / np.float32(nbits), np.float32(1))
    f3 = sobel_magnitude(left).astype(np.float32) / np.float32(SOBEL_SCALE)
    return np.stack([f0, f1, f2, f3]).astype(np.float32)


# ---------------------------------------------------------------- the network

def conv3x3(x, W, b=None) -> np.ndarray:
    """y[o] = b[o] + sum_{i, ky, kx} W[o, i, ky, kx] x[i, y + ky - 1, x + kx - 1], zero padded."""
    x = np.asarray(x, np.float64)
    C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    y = np.zeros((W.shape[0], H, Wd))
    for ky in range(3):
        for kx in range(3):
            y += np.tensordot(W[:, :, ky, kx], xp[:, ky:ky + H, kx:kx + Wd], axes=(1, 0))
    if b is not None:
        y += np.asarray(b, np.float64)[:, None, None]
    return y


def flip_transpose(W) -> np.ndarray:
    """Weights of the input-gradient correlation: F[i, o, ky, kx] = W[o, i, 2 - ky, 2 - kx]."""
    return np.ascontiguousarray(np.transpose(W, (1, 0, 2, 3))[:, :, ::-1, ::-1])


def forward(theta, feats, quant: bool = True):
    """Returns (acts, out): acts[l] is the input of layer l (acts[0] = the
    features), out the last layer's output (N_OUT, H, W) float64.  With quant,
    the weights and every stored activation are bfloat16 values and the
    hidden layers apply ReLU before rounding (the device's epilogue)."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    layers = unpack(theta)
    h = q(feats).astype(np.float64)
    acts = [h]
    for l, (W, b) in enumerate(layers):
        z = conv3x3(h, q(W).astype(np.float64), np.asarray(b, np.float32).astype(np.float64) if quant else b)
        if l == len(layers) - 1:
            return acts, z
        h = q(np.maximum(z, 0.0)).astype(np.float64)
        acts.append(h)


def labels(d_fill, d_target, D: int) -> np.ndarray:
    """Radius class that the target needs: the smallest k with
    |round(d_target) - round(d_fill)| <= RADII[k] (rounded centres clamped to
    [0, D - 1], as the window rule rounds), else the widest class."""
    c = np.clip(np.floor(np.asarray(d_fill, np.float32) + np.float32(0.5)), 0, D - 1)
    t = np.clip(np.floor(np.asarray(d_target, np.float32) + np.float32(0.5)), 0, D - 1)
    dist = np.abs(t - c)
    lab = np.full(dist.shape, N_CLASSES - 1, np.int64)
    for k in reversed(range(N_CLASSES)):
        lab = np.where(dist <= RADII[k], k, lab)
    return lab


def loss_and_grad(out, d_fill, d_target, valid, D: int, npix: int | None = None):
    """Mean over all pixels (valid ones contribute) of cross-entropy of the
    radius class plus NLL_WEIGHT * 0.5 (e^2 exp(-s) + s), e = d_target - d_fill,
    s = the log-variance output.  Returns (loss, d loss / d out)."""
    out = np.asarray(out, np.float64)
    valid = np.asarray(valid, bool)
    npix = valid.size if npix is None else npix
    z = out[:N_CLASSES]
    s = out[N_CLASSES]
    lab = labels(d_fill, d_target, D)
    zmax = z.max(0)
    ez = np.exp(z - zmax)
    sm = ez / ez.sum(0)
    lse = zmax + np.log(ez.sum(0))
    ce = lse - np.take_along_axis(z, lab[None], 0)[0]
    e = np.asarray(d_target, np.float64) - np.asarray(d_fill, np.float64)
    es = e * e * np.exp(-s)
    nll = 0.5 * (es + s)
    loss = float(np.sum(np.where(valid, ce + NLL_WEIGHT * nll, 0.0))) / npix
    g = np.zeros_like(out)
    onehot = (np.arange(N_CLASSES)[:, None, None] == lab[None]).astype(np.float64)
    g[:N_CLASSES] = np.where(valid[None], sm - onehot, 0.0) / npix
    g[N_CLASSES] = np.where(valid, NLL_WEIGHT * 0.5 * (1.0 - es), 0.0) / npix
    return loss, g


def backward(theta, acts, g_out, quant: bool = True):
    """Gradients of the loss for every parameter, given the forward's stored
    activations and d loss / d out.  With quant the output gradient and each
    layer's input gradient are rounded to bfloat16 where the device stores
    them, and the input gradient uses the bfloat16 weights.  Returns a flat
    vector in the order of `pack`."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    layers = unpack(theta)
    g = q(g_out).astype(np.float64)
    grads = [None] * len(layers)
    for l in reversed(range(len(layers))):
        W, _ = layers[l]
        x = acts[l]
        C, H, Wd = x.shape
        xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
        dW = np.zeros(W.shape)
        for ky in range(3):
            for kx in range(3):
                dW[:, :, ky, kx] = np.tensordot(g, xp[:, ky:ky + H, kx:kx + Wd], axes=([1, 2], [1, 2]))
        grads[l] = (dW, g.sum((1, 2)))
        if l > 0:
            dx = conv3x3(g, flip_transpose(q(W).astype(np.float64)))
            g = q(dx * (x > 0)).astype(np.float64)
    return pack(grads)


def adam(theta, m, v, grad, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected, step counted from 1); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def decide(out):
    """Per-pixel half-width and measurement variance from the network output:
    the most probable class's radius when its softmax probability is at least
    CONFIDENCE, else FALLBACK_RADIUS; r = exp(s) clamped to [R_MIN, R_MAX].
    Also returns the winning probability."""
    out = np.asarray(out, np.float64)
    z = out[:N_CLASSES]
    ez = np.exp(z - z.max(0))
    sm = ez / ez.sum(0)
    k = sm.argmax(0)
    conf = sm.max(0)
    radius = np.where(conf >= CONFIDENCE, np.asarray(RADII)[k], FALLBACK_RADIUS).astype(np.uint8)
    r = np.clip(np.exp(out[N_CLASSES]), R_MIN, R_MAX)
    return radius, r, conf
