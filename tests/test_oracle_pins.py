"""Pins for the oracle (CPU only): each stage is tied to something other than itself.

* census: closed-form codes of intensity ramps and constant images (bit order,
  bit sense, border clamping), Section 2.1;
* cost: exact shifts give zero cost, out-of-image matches cost every bit;
* aggregation: Eq. 1 equals exhaustive minimisation over all disparity
  sequences on tiny scanlines and tiny images (all 8 directions, random
  ragged windows, full windows = plain SGM), Section 2.2;
* winner-takes-all: exact parabola vertices, first-minimum ties, Section 2.3;
* fronto-parallel textured planes at integer disparity come back exactly;
* warp: identity motion, closed-form forward and lateral translation, the
  z-buffer rule, Eqs. 2-4;
* resolve: hand-derived fixtures in tests/golden/resolve_cases.json, Section 2.4;
* Kalman: closed-form steady state of the scalar Riccati recursion, the K = 1/2
  case, the gate threshold, Eqs. 5-6.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ census

def test_census_increasing_ramp_sets_the_first_half(orc):
    # I strictly increasing in row-major order: every window pixel before the
    # centre is darker -> bits 0..11 set (centre skipped, LSB first).
    img = np.arange(9 * 11).reshape(9, 11).astype(np.uint8)
    c = orc.census(img)
    assert int(c[4, 5]) == 0x000FFF
    rev = (255 - img).astype(np.uint8)
    assert int(orc.census(rev)[4, 5]) == 0xFFF000


def test_census_column_and_row_ramps(orc):
    y_ramp = np.repeat(np.arange(8)[:, None] * 10, 8, axis=1).astype(np.uint8)
    # rows above the centre are darker: 2 rows x 5 = bits 0..9
    assert int(orc.census(y_ramp)[4, 4]) == 0x3FF
    x_ramp = np.repeat(np.arange(8)[None, :] * 10, 8, axis=0).astype(np.uint8)
    # columns dx = -2, -1 are darker in each row; bit positions in the
    # centre-skipped row-major order:
    expect = sum(1 << b for b in (0, 1, 5, 6, 10, 11, 14, 15, 19, 20))
    assert int(orc.census(x_ramp)[4, 4]) == expect


def test_census_constant_image_and_border_clamp(orc):
    assert not orc.census(np.full((6, 7), 77, np.uint8)).any()
    x_ramp = np.repeat(np.arange(8)[None, :] * 10, 8, axis=0).astype(np.uint8)
    # at x = 0 the left neighbours clamp onto the centre column: equal, no bit
    assert int(orc.census(x_ramp)[4, 0]) == 0
    # at x = 1, only dx = -1 is darker; dx = -2 clamps to x = 0 (also darker)
    assert int(orc.census(x_ramp)[4, 1]) == sum(1 << b for b in (0, 1, 5, 6, 10, 11, 14, 15, 19, 20))


def test_census_window_sizes(orc):
    assert orc.census_bits(5, 5) == 24
    assert orc.census_bits(9, 7) == 62
    # strictly increasing image, 7x7 window: the 24 pixels before the centre are darker
    img = np.arange(15 * 15).reshape(15, 15).astype(np.uint8)
    assert int(orc.census(img, 7, 7)[7, 7]) == (1 << 24) - 1
    # 9x7 window (62 bits): 31 pixels precede the centre
    img = np.arange(15 * 17).reshape(15, 17).astype(np.uint8)
    assert int(orc.census(img, 9, 7)[7, 8]) == (1 << 31) - 1


# ------------------------------------------------------------------ cost

def test_cost_exact_shift_is_zero_and_left_overhang_costs_every_bit(orc):
    rng = np.random.default_rng(5)
    H, W, D, dtrue = 6, 40, 12, 5
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = np.empty_like(left)
    right[:, : W - dtrue] = left[:, dtrue:]
    right[:, W - dtrue:] = rng.integers(0, 256, (H, dtrue), dtype=np.uint8)
    cl, cr = orc.census(left), orc.census(right)
    lo = np.zeros((H, W), np.uint16)
    wd = np.full((H, W), D, np.uint16)
    off, n = orc.offsets(wd)
    c = orc.cost(cl, cr, lo, wd, off, n, 24).reshape(H, W, D)
    for x in range(dtrue + 2, W - 2):
        assert (c[:, x, dtrue] == 0).all()
    for x in range(W):
        for d in range(D):
            if x - d < 0:
                assert (c[:, x, d] == 24).all()
    # complementary codes differ in every bit
    inc = np.arange(9 * 11).reshape(9, 11).astype(np.uint8)
    a, b = orc.census(inc), orc.census((255 - inc).astype(np.uint8))
    one = np.ones((9, 11), np.uint16)
    off1, n1 = orc.offsets(one)
    cc = orc.cost(a, b, np.zeros((9, 11), np.uint16), one, off1, n1, 24).reshape(9, 11)
    assert cc[4, 5] == 24


def test_offsets_are_an_exclusive_prefix_sum(orc):
    rng = np.random.default_rng(0)
    wd = rng.integers(1, 200, size=(13, 17)).astype(np.uint16)
    off, n = orc.offsets(wd)
    flat = wd.ravel().astype(np.int64)
    assert n == flat.sum()
    assert off.ravel()[0] == 0
    assert (np.diff(off.ravel().astype(np.int64)) == flat[:-1]).all()


# ------------------------------------------------------------------ aggregation (Eq. 1)

def _pen(k, d, P1, P2):
    if k == d:
        return 0
    if abs(k - d) == 1:
        return min(P1, P2)
    return P2


def _line_losses_by_enumeration(costs, windows, P1, P2):
    """A_i(d) = min over every disparity sequence ending in d at position i of
    (sum of costs + sum of transition penalties); returns the normalised
    L(i, d) = A_i(d) - min_k A_{i-1}(k) that Eq. 1 with min-subtraction gives."""
    n = len(costs)
    A = []
    for i in range(n):
        Ai = {}
        for seq in itertools.product(*[range(lo, lo + w) for lo, w in windows[: i + 1]]):
            tot = sum(costs[j][seq[j] - windows[j][0]] for j in range(i + 1))
            tot += sum(_pen(seq[j - 1], seq[j], P1, P2) for j in range(1, i + 1))
            Ai[seq[-1]] = min(Ai.get(seq[-1], 1 << 30), tot)
        A.append(Ai)
    L = []
    for i in range(n):
        base = 0 if i == 0 else min(A[i - 1].values())
        L.append([A[i][d] - base for d in range(windows[i][0], windows[i][0] + windows[i][1])])
    return L


@pytest.mark.parametrize("seed", range(12))
def test_path_aggregation_equals_exhaustive_enumeration_on_scanlines(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 7))
    D = int(rng.integers(2, 7))
    P1, P2 = int(rng.integers(1, 10)), int(rng.integers(10, 40))
    if seed % 4 == 3:
        P1, P2 = 30, 12            # P1 > P2 is still well defined
    windows = []
    for _ in range(n):
        if seed % 3 == 0:
            windows.append((0, D))            # full range = plain SGM
        else:
            lo = int(rng.integers(0, D))
            windows.append((lo, int(rng.integers(1, D - lo + 1))))
    lo = np.array([[w[0] for w in windows]], np.uint16)
    wd = np.array([[w[1] for w in windows]], np.uint16)
    off, ncells = orc.offsets(wd)
    cost = rng.integers(0, 25, size=ncells).astype(np.uint8)
    costs = [cost[off[0, i]: off[0, i] + wd[0, i]].tolist() for i in range(n)]
    expect = _line_losses_by_enumeration(costs, windows, P1, P2)
    got = orc.aggregate_dir(cost, lo, wd, off, ncells, 0, P1, P2)   # direction (+1, 0)
    for i in range(n):
        assert got[off[0, i]: off[0, i] + wd[0, i]].tolist() == expect[i], (i, windows)
    # the reverse direction equals enumeration over the reversed line
    rexp = _line_losses_by_enumeration(costs[::-1], windows[::-1], P1, P2)[::-1]
    got = orc.aggregate_dir(cost, lo, wd, off, ncells, 1, P1, P2)
    for i in range(n):
        assert got[off[0, i]: off[0, i] + wd[0, i]].tolist() == rexp[i]


def _lines(W, H, dx, dy):
    """Every path of direction (dx, dy): start where the predecessor is outside."""
    out = []
    for y in range(H):
        for x in range(W):
            if 0 <= x - dx < W and 0 <= y - dy < H:
                continue
            line, cx, cy = [], x, y
            while 0 <= cx < W and 0 <= cy < H:
                line.append((cx, cy))
                cx, cy = cx + dx, cy + dy
            out.append(line)
    return out


@pytest.mark.parametrize("seed", range(4))
def test_eight_path_sum_equals_enumeration_on_tiny_images(orc, seed):
    rng = np.random.default_rng(100 + seed)
    W, H, D = 4, 3, 4
    P1, P2 = 3, 11
    lo = rng.integers(0, D, size=(H, W)).astype(np.uint16)
    wd = np.array([[rng.integers(1, D - lo[y, x] + 1) for x in range(W)] for y in range(H)], np.uint16)
    if seed == 0:
        lo[:] = 0
        wd[:] = D
    off, ncells = orc.offsets(wd)
    cost = rng.integers(0, 25, size=ncells).astype(np.uint8)
    S = np.zeros(ncells, np.int64)
    for k, (dx, dy) in enumerate(orc.DIRECTIONS):
        Lk = np.zeros(ncells, np.int64)
        for line in _lines(W, H, dx, dy):
            wins = [(int(lo[y, x]), int(wd[y, x])) for x, y in line]
            costs = [cost[off[y, x]: off[y, x] + wd[y, x]].tolist() for x, y in line]
            L = _line_losses_by_enumeration(costs, wins, P1, P2)
            for (x, y), l in zip(line, L):
                Lk[off[y, x]: off[y, x] + wd[y, x]] = l
        got = orc.aggregate_dir(cost, lo, wd, off, ncells, k, P1, P2)
        assert (got.astype(np.int64) == Lk).all(), k
        S += Lk
    assert (orc.aggregate(cost, lo, wd, off, ncells, 0xFF, P1, P2).astype(np.int64) == S).all()
    # a subset of paths sums only those
    sub = np.zeros(ncells, np.int64)
    for k in (0, 1, 2, 3):
        sub += orc.aggregate_dir(cost, lo, wd, off, ncells, k, P1, P2).astype(np.int64)
    assert (orc.aggregate(cost, lo, wd, off, ncells, 0x0F, P1, P2).astype(np.int64) == sub).all()


def test_disjoint_windows_cost_exactly_P2(orc):
    lo = np.array([[0, 10]], np.uint16)
    wd = np.array([[3, 3]], np.uint16)
    off, n = orc.offsets(wd)
    cost = np.array([5, 1, 7, 2, 9, 4], np.uint8)
    L = orc.aggregate_dir(cost, lo, wd, off, n, 0, 6, 65)
    assert L[3:].tolist() == [2 + 65, 9 + 65, 4 + 65]


# ------------------------------------------------------------------ WTA

def test_wta_parabola_vertex_and_ties(orc):
    # S(d) = 4 (d - 5.25)^2 sampled at integers, shifted to integers: the
    # parabola through the 3 samples around the minimum has its vertex at 5.25.
    d = np.arange(12)
    S = (4 * (d - 5.25) ** 2 * 4).round().astype(np.uint16)   # 16 (d-5.25)^2 is integral
    assert np.allclose(S, 16 * (d - 5.25) ** 2)
    lo = np.zeros((1, 1), np.uint16)
    wd = np.full((1, 1), 12, np.uint16)
    off = np.zeros((1, 1), np.uint32)
    di, dz = orc.wta(S, lo, wd, off)
    assert di[0, 0] == 5 and dz[0, 0] == np.float32(5.25)
    # ties: the smallest d wins, and a winner at the window edge stays integral
    S2 = np.array([3, 1, 4, 1, 5], np.uint16)
    di, dz = orc.wta(S2, np.full((1, 1), 7, np.uint16), np.full((1, 1), 5, np.uint16), off)
    assert di[0, 0] == 8 and dz[0, 0] == np.float32(8 + (3 - 4) / (2 * (3 - 2 + 4)))
    S3 = np.array([0, 1, 4], np.uint16)
    di, dz = orc.wta(S3, np.full((1, 1), 2, np.uint16), np.full((1, 1), 3, np.uint16), off)
    assert di[0, 0] == 2 and dz[0, 0] == 2.0


def test_fronto_parallel_plane_returns_exact_disparity(orc):
    rng = np.random.default_rng(11)
    H, W, D = 24, 96, 32
    for dtrue in (0, 3, 17):
        left = rng.integers(0, 256, (H, W), dtype=np.uint8)
        right = rng.integers(0, 256, (H, W), dtype=np.uint8)
        right[:, : W - dtrue] = left[:, dtrue:]
        P = orc.Params(W, H, max_disp=D)
        out = orc.frame(P, left, right)
        core = out["d_int"][:, dtrue + 2: W - 2]
        assert (core == dtrue).all(), dtrue


# ------------------------------------------------------------------ warp (Eqs. 2-4)

K = np.array([400.0, 0.0, 191.5, 0.0, 400.0, 63.5, 0.0, 0.0, 1.0], np.float32)


def test_identity_motion_keeps_disparity_and_adds_q(orc):
    rng = np.random.default_rng(2)
    d = rng.uniform(1.0, 60.0, (16, 24)).astype(np.float32)
    p = rng.uniform(0.1, 3.0, (16, 24)).astype(np.float32)
    d0, p0, known0 = orc.warp(d, p, np.eye(3), np.zeros(3), K, 0.5, 0.15)
    assert known0.all()
    assert np.allclose(d0, d, rtol=2e-7, atol=0)
    assert np.allclose(p0, p + np.float32(0.15), rtol=1e-6)


def test_forward_translation_matches_closed_form(orc):
    # camera moves t_f forward: X_k = X_{k-1} - (0, 0, t_f);
    # d' = f b d / (f b - d t_f), x' - cx = (x - cx) Z / (Z - t_f)
    H, W, tf, b = 20, 30, 0.5, 0.5
    fb = 400.0 * b
    d = np.full((H, W), 10.0, np.float32)
    p = np.ones((H, W), np.float32)
    d0, p0, known0, tgt, dn = orc.warp(d, p, np.eye(3), [0, 0, -tf], K, b, 0.0, per_source=True)
    dexp = fb * 10.0 / (fb - 10.0 * tf)
    assert np.allclose(dn[tgt >= 0], dexp, rtol=1e-6)
    Z = fb / 10.0
    for y in (0, 7, 19):
        for x in (0, 13, 29):
            xe = 191.5 + (x - 191.5) * Z / (Z - tf)
            ye = 63.5 + (y - 63.5) * Z / (Z - tf)
            xi, yi = math.floor(xe + 0.5), math.floor(ye + 0.5)
            inside = 0 <= xi < W and 0 <= yi < H
            assert (tgt[y, x] >= 0) == inside
            if inside:
                assert tgt[y, x] == yi * W + xi
    # the plane stays fronto-parallel; Phi = d'/d enters Eq. 4
    phi = dexp / 10.0
    assert np.allclose(p0[known0 == 1], phi * phi * 1.0, rtol=1e-5)


def test_lateral_translation_shifts_by_disparity_times_t_over_b(orc):
    H, W, b = 4, 64, 0.5
    d = np.zeros((H, W), np.float32)
    d[:, :] = 8.0
    d[1, :] = 16.0
    p = np.ones((H, W), np.float32)
    # camera moves +0.25 m to the right: X_k = X_{k-1} - 0.25 -> x' = x - d * 0.25 / b
    _, _, _, tgt, dn = orc.warp(d, p, np.eye(3), [-0.25, 0, 0], K, b, 0.0, per_source=True)
    for y, dv in ((0, 8.0), (1, 16.0)):
        for x in range(20, 40):
            xe = x - dv * 0.25 / b
            assert tgt[y, x] == y * W + int(math.floor(xe + 0.5))
            assert dn[y, x] == np.float32(dv)


def test_zbuffer_nearest_wins_and_ties_go_to_the_smaller_index(orc):
    rng = np.random.default_rng(3)
    H, W = 12, 40
    d = rng.uniform(4.0, 20.0, (H, W)).astype(np.float32)
    d[5, :] = 9.0   # one row of equal disparity moved backwards collides with itself
    p = rng.uniform(0.5, 2.0, (H, W)).astype(np.float32)
    Rm = np.eye(3)
    t = [0.0, 0.0, 1.5]                      # camera moves back: the image shrinks
    d0, p0, known0, tgt, dn = orc.warp(d, p, Rm, t, K, 0.5, 0.15, per_source=True)
    n_ties = 0
    for q in np.unique(tgt[tgt >= 0]):
        srcs = np.flatnonzero(tgt.ravel() == q)
        vals = dn.ravel()[srcs]
        best = vals.max()
        winner = srcs[vals == best].min()
        n_ties += int((vals == best).sum() > 1)
        y, x = divmod(int(q), W)
        assert known0[y, x] == 1 and d0[y, x] == best
        ds, ps = d.ravel()[winner], p.ravel()[winner]
        assert p0[y, x] == orc.predict_variance(np.float32(best / ds), ps, 0.15)
    assert n_ties > 0
    assert (known0.sum() == len(np.unique(tgt[tgt >= 0])))


def test_points_behind_the_camera_or_invalid_are_dropped(orc):
    d = np.array([[0.4, 10.0, 10.0]], np.float32)    # d <= 0.5 is not moved
    p = np.ones_like(d)
    _, _, known0, tgt, _ = orc.warp(d, p, np.eye(3), [0, 0, -100.0], K, 0.5, 0.1, per_source=True)
    assert (tgt == -1).all() and not known0.any()     # Z' = 20 - 100 < 0


# ------------------------------------------------------------------ resolve (Section 2.4)

def test_resolve_golden_cases(orc):
    doc = json.load(open(os.path.join(GOLDEN, "resolve_cases.json")))
    for case in doc["cases"]:
        d0 = np.array(case["d0"], np.float32)
        p0 = np.array(case["p0"], np.float32)
        k0 = np.array(case["known0"], np.uint8)
        dp, pp, cls, lo, wd = orc.resolve(d0, p0, k0, case["D"], case["radius_mode"], case["radius"],
                                          case["p_reset"], case["tau_disc"])
        for e in case["expect"]:
            y, x = e["y"], e["x"]
            assert cls[y, x] == e["cls"], case["name"]
            assert lo[y, x] == e["lo"] and wd[y, x] == e["wd"], case["name"]
            if "d" in e:
                assert dp[y, x] == np.float32(e["d"]) and pp[y, x] == np.float32(e["p"]), case["name"]


# ------------------------------------------------------------------ Kalman (Eqs. 5-6)

def test_kalman_steady_state_matches_the_riccati_closed_form(orc):
    q, r = 0.15, 1.0
    p = 5.0
    for _ in range(200):
        pv = orc.predict_variance(1.0, p, q)       # Eq. 4 with Phi = 1
        d, p, m, nu = orc.kalman_update32(10.0, pv, 0, 10.0, r, 6.635)
    p_inf = (-q + math.sqrt(q * q + 4 * q * r)) / 2
    assert abs(p - p_inf) < 2e-6
    K_inf = (p_inf + q) / (p_inf + q + r)
    assert abs(K_inf - p_inf / r) < 1e-12
    assert abs(p_inf - 0.31949) < 1e-5


def test_kalman_equal_variances_average_and_gate(orc):
    d, p, m, nu = orc.kalman_update32(10.0, 1.0, 0, 12.0, 1.0, 6.635)
    assert (d, p, m, nu) == (11.0, 0.5, 0, 2.0)          # K = 1/2
    # gate: nu^2 > gamma (p + r) flags the pixel and resets to the measurement
    g = 6.635 * 2.0
    nu_in = math.sqrt(g) * 1.01
    d, p, m, _ = orc.kalman_update32(10.0, 1.0, 0, 10.0 + nu_in, 1.0, 6.635)
    assert m == 1 and d == np.float32(10.0 + nu_in) and p == 1.0
    nu_in = math.sqrt(g) * 0.99
    d, p, m, _ = orc.kalman_update32(10.0, 1.0, 0, 10.0 + nu_in, 1.0, 6.635)
    assert m == 0 and p == 0.5
    # no prediction: take the measurement
    assert orc.kalman_update32(0.0, 0.0, 2, 7.5, 1.0, 6.635) == (7.5, 1.0, 0, 0.0)


def test_kalman64_agrees_with_kalman32_within_single_precision(orc):
    rng = np.random.default_rng(9)
    n = 5000
    dp = rng.uniform(1, 100, n).astype(np.float32)
    pv = rng.uniform(0.05, 1500, n).astype(np.float32)
    dz = (dp + rng.normal(0, 1.0, n)).astype(np.float32)
    cls = rng.integers(0, 3, n).astype(np.uint8)
    d32, p32, m, _ = orc.kalman32(dp, pv, cls, dz, 1.0, 6.635)
    d64, p64 = orc.kalman64(dp, pv, cls, dz, 1.0, 6.635)
    assert np.max(np.abs(d32 - d64) / np.abs(d64)) < 1e-6
    assert np.max(np.abs(p32 - p64) / np.abs(p64)) < 1e-6


def test_full_window_reduced_frame_equals_the_initial_full_range_frame(orc):
    # Section 2.4: search limits covering the whole space turn the method into
    # conventional SGM; only the Kalman fusion differs.
    import synth
    s = synth.tiny_pair(4)
    P = orc.Params(384, 128, max_disp=64, radius_mode=2)
    L, R = s["left"].numpy(), s["right"].numpy()
    f0 = orc.frame(P, L[1], R[1])
    prev = orc.frame(P, L[0], R[0])
    f1 = orc.frame(P, L[1], R[1], state=(prev["d"], prev["p"]),
                   motion=(s["R"][1].numpy(), s["t"][1].numpy(), s["K"].numpy(), s["baseline"]))
    assert (f1["wd"] == 64).all()
    assert (f1["S"] == f0["S"]).all() and (f1["d_int"] == f0["d_int"]).all()
