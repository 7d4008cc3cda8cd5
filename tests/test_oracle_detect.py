"""Pins for the oracle's post-path steps (CPU only): the 3x3 median output
(Section 2.3) and the moving-object boxes of Section 4 (integral image,
sliding windows, greedy IoU grouping, small-box discard)."""
import numpy as np
import pytest


def test_median3_matches_numpy_median_with_clamped_border(orc):
    rng = np.random.default_rng(0)
    d = rng.uniform(0, 100, (13, 17)).astype(np.float32)
    got = orc.median3(d)
    pad = np.pad(d, 1, mode="edge")
    want = np.zeros_like(d)
    for y in range(13):
        for x in range(17):
            want[y, x] = np.median(pad[y:y + 3, x:x + 3])   # odd count: an element, exact
    assert np.array_equal(got, want)


def test_median3_removes_an_isolated_outlier_and_keeps_constants(orc):
    d = np.full((7, 7), 12.5, np.float32)
    assert np.array_equal(orc.median3(d), d)
    d[3, 3] = 99.0
    assert (orc.median3(d) == 12.5).all()


def test_quantised_innovation(orc):
    nu = np.array([[0.03125, -1.0, 0.02, 5000.0, 2.0]], np.float32)
    cls = np.array([[0, 0, 1, 0, 2]], np.uint8)
    assert orc.abs_innovation_q(nu, cls).tolist() == [[1, 16, 0, 65535, 0]]


def test_integral_image_is_the_2d_cumulative_sum(orc):
    rng = np.random.default_rng(1)
    a = rng.integers(0, 65536, (11, 9)).astype(np.uint32)
    sat = orc.integral(a)
    assert (sat[0] == 0).all() and (sat[:, 0] == 0).all()
    assert np.array_equal(sat[1:, 1:], a.astype(np.uint64).cumsum(0).cumsum(1))


def test_windows_match_brute_force_sums(orc):
    rng = np.random.default_rng(2)
    H, W = 60, 90
    a = np.zeros((H, W), np.uint32)
    a[30:55, 40:75] = rng.integers(10, 40, (25, 35))     # a "moving" patch, mean ~25 (1.5 px)
    a += rng.integers(0, 4, (H, W)).astype(np.uint32)    # noise
    sizes, stride, y_min, tq = [(20, 20), (30, 30), (25, 40)], 5, H // 3, 16
    got = orc.windows(orc.integral(a), sizes, stride, y_min, tq)
    want = []
    for ww, wh in sizes:
        for y0 in range(y_min, H - wh + 1, stride):
            for x0 in range(0, W - ww + 1, stride):
                if int(a[y0:y0 + wh, x0:x0 + ww].sum(dtype=np.uint64)) > tq * ww * wh:
                    want.append((x0, y0, x0 + ww, y0 + wh))
    assert [tuple(b) for b in got] == want and len(want) > 0
    assert all(b[1] >= y_min for b in got)


def test_greedy_merge_cases(orc):
    # two overlapping boxes become their union; a disjoint one stays
    b = [(0, 0, 10, 10), (5, 0, 15, 10), (40, 40, 50, 50)]
    assert orc.merge_boxes(b, 0, 1, 0).tolist() == [[0, 0, 15, 10], [40, 40, 50, 50]]
    # the best pair goes first: (A, C) have IoU 0.9 > (A, B) at 1/3; the union
    # of A and C then also absorbs B
    A, B, C = (0, 0, 100, 10), (50, 0, 150, 10), (0, 0, 90, 10)
    assert orc.merge_boxes([A, B, C], 0, 1, 0).tolist() == [[0, 0, 150, 10]]
    # with a threshold IoU > 1/2 only the (A, C) pair merges
    assert orc.merge_boxes([A, B, C], 1, 2, 0).tolist() == [[0, 0, 100, 10], [50, 0, 150, 10]]
    # touching boxes do not overlap; small boxes are discarded afterwards
    t = [(0, 0, 10, 10), (10, 0, 20, 10), (30, 30, 33, 33)]
    assert orc.merge_boxes(t, 0, 1, 50).tolist() == [[0, 0, 10, 10], [10, 0, 20, 10]]
    # a chain of overlaps collapses to one box
    chain = [(i * 8, 0, i * 8 + 10, 10) for i in range(6)]
    assert orc.merge_boxes(chain, 0, 1, 0).tolist() == [[0, 0, 50, 10]]


def test_detection_finds_the_independently_moving_box(orc):
    # Section 4: the box moving on its own differs from the ego-motion
    # prediction; the merged detections cover it.
    import synth
    s = synth.tiny_pair(1)
    P = orc.Params(384, 128, max_disp=64, radius=4)
    L, R = s["left"].numpy(), s["right"].numpy()
    f0 = orc.frame(P, L[0], R[0])
    f1 = orc.frame(P, L[1], R[1], state=(f0["d"], f0["p"]),
                   motion=(s["R"][1].numpy(), s["t"][1].numpy(), s["K"].numpy(), s["baseline"]))
    Dp = orc.DetectParams(min_area=400)
    boxes, raw, _ = orc.detect(f1["nu"], f1["cls"], Dp)
    assert len(raw) > 0 and len(boxes) >= 1


def _fixpoint(boxes):
    """Merge overlapping boxes until none overlap, each group at the position
    of its first box (rounds of all-pairs union-find)."""
    v = [list(b) for b in boxes]
    while True:
        n = len(v)
        parent = list(range(n))

        def find(a):
            while parent[a] != a:
                a = parent[a]
            return a
        merged = False
        for i in range(n):
            for j in range(i + 1, n):
                a, b = v[i], v[j]
                if a[0] < b[2] and b[0] < a[2] and a[1] < b[3] and b[1] < a[3]:
                    ri, rj = find(i), find(j)
                    if ri != rj:
                        parent[max(ri, rj)] = min(ri, rj)
                        merged = True
        if not merged:
            return v
        out, slot = [], {}
        for i in range(n):
            r = find(i)
            if r not in slot:
                slot[r] = len(out)
                out.append(list(v[i]))
            else:
                g = out[slot[r]]
                g[:] = [min(g[0], v[i][0]), min(g[1], v[i][1]), max(g[2], v[i][2]), max(g[3], v[i][3])]
        v = out


@pytest.mark.parametrize("seed", range(6))
def test_greedy_merge_at_iou_zero_is_order_independent(orc, seed):
    # The greedy of Section 4 with "any overlap" merges ends in the same boxes,
    # in the same order, as the order-free fixpoint; the library relies on it.
    rng = np.random.default_rng(seed)
    n = 120
    x0 = rng.integers(0, 400, n)
    y0 = rng.integers(0, 200, n)
    w = rng.integers(5, 40, n)
    h = rng.integers(5, 40, n)
    boxes = np.stack([x0, y0, x0 + w, y0 + h], 1).astype(np.int32)
    got = orc.merge_boxes(boxes, 0, 1, 0).tolist()
    assert got == _fixpoint(boxes.tolist())
