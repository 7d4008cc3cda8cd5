"""The box grouping of Section 4 as the library runs it (rsgm_group_boxes,
host code, no GPU) against the oracle's literal greedy merge: random boxes
and the sliding-window detections of a synthetic frame, for "any overlap"
and for IoU thresholds."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def rs():
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


def _random_boxes(rng, n, extent=400, size=(5, 60)):
    x0 = rng.integers(0, extent, n)
    y0 = rng.integers(0, extent // 2, n)
    w = rng.integers(size[0], size[1], n)
    h = rng.integers(size[0], size[1], n)
    return np.stack([x0, y0, x0 + w, y0 + h], 1).astype(np.int32)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("iou", [(0, 1), (1, 3), (1, 2), (3, 4)])
def test_random_boxes_match_the_oracle(rs, orc, seed, iou):
    rng = np.random.default_rng(seed)
    boxes = _random_boxes(rng, int(rng.integers(0, 160)))
    min_area = int(rng.choice([0, 400, 1500]))
    got = rs.rsgm_group_boxes(boxes, iou[0], iou[1], min_area)
    want = orc.merge_boxes(boxes, iou[0], iou[1], min_area)
    assert np.array_equal(got, want)


def test_lattice_windows_of_a_frame_match_the_oracle(rs, orc):
    # the detections of a synthetic frame: windows on a regular lattice, heavily overlapping
    import synth
    s = synth.tiny_pair(1)
    P = orc.Params(384, 128, max_disp=64, radius=4)
    L, R = s["left"].numpy(), s["right"].numpy()
    f0 = orc.frame(P, L[0], R[0])
    f1 = orc.frame(P, L[1], R[1], state=(f0["d"], f0["p"]),
                   motion=(s["R"][1].numpy(), s["t"][1].numpy(), s["K"].numpy(), s["baseline"]))
    Dp = orc.DetectParams(min_area=400)
    _, raw, _ = orc.detect(f1["nu"], f1["cls"], Dp)
    assert len(raw) > 10
    for iou in [(0, 1), (1, 2)]:
        assert np.array_equal(rs.rsgm_group_boxes(raw, iou[0], iou[1], 400), orc.merge_boxes(raw, iou[0], iou[1], 400))


def test_arguments_are_checked(rs):
    with pytest.raises(rs.RsgmError):
        rs.rsgm_group_boxes(np.zeros((1, 4)), 0, 0, 0)      # iou_den < 1
    assert rs.rsgm_group_boxes(np.zeros((0, 4))).shape == (0, 4)


@pytest.mark.parametrize("seed", range(6))
def test_lattice_and_degenerate_boxes_match_the_oracle(rs, orc, seed):
    # windows on a stride-10 lattice of the default sizes (dense overlaps, many
    # merge rounds), plus boxes without area, which never merge (IoU 0)
    rng = np.random.default_rng(100 + seed)
    sizes = [(20, 20), (30, 30), (40, 40), (50, 50), (50, 75)]
    boxes = []
    for w, h in sizes:
        for iy in range(12):
            for ix in range(30):
                if rng.random() < 0.25:
                    x0, y0 = ix * 10, 125 + iy * 10
                    boxes.append((x0, y0, x0 + w, y0 + h))
    for _ in range(10):
        x0, y0 = int(rng.integers(0, 300)), int(rng.integers(100, 250))
        boxes.append((x0, y0, x0 + int(rng.integers(0, 2)) * 30, y0 + int(rng.integers(0, 2)) * 30))
    boxes = np.array(boxes, np.int32)
    boxes = boxes[rng.permutation(len(boxes))]
    for iou, min_area in [((0, 1), 0), ((0, 1), 1500), ((1, 2), 0)]:
        got = rs.rsgm_group_boxes(boxes, iou[0], iou[1], min_area)
        assert np.array_equal(got, orc.merge_boxes(boxes, iou[0], iou[1], min_area)), (iou, min_area)


def test_coordinates_beyond_the_limit_are_rejected(rs):
    lim = 1 << 20
    assert rs.rsgm_group_boxes(np.array([[-lim, -lim, lim, lim]], np.int32)).shape == (1, 4)
    for bad in ([-lim - 1, 0, 10, 10], [0, 0, lim + 1, 10], [0, -2 ** 31, 10, 2 ** 31 - 1]):
        with pytest.raises(rs.RsgmError) as e:
            rs.rsgm_group_boxes(np.array([bad], np.int32))
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG


def test_nested_boxes_and_extreme_areas_match_the_oracle(rs, orc):
    import time
    # 1000 nested boxes: a 2000 x 2000 grid whose painting would cost about
    # 1e9 cell writes, where checking the pairs costs 5e5
    n = 1000
    nested = np.array([[i, i, 4000 - i, 4000 - i] for i in range(n)], np.int32)[::-1].copy()
    t0 = time.perf_counter()
    got = rs.rsgm_group_boxes(nested)
    assert time.perf_counter() - t0 < 2.0
    assert np.array_equal(got, orc.merge_boxes(nested, 0, 1, 0))
    # areas near 2^42 with an IoU threshold: exact comparisons, no overflow
    lim = 1 << 20
    big = np.array([[-lim, -lim, lim, lim], [-lim + 1, -lim, lim, lim], [0, 0, lim, lim]], np.int32)
    for iou in [(1, 2), (999999, 1000000), (1, 4)]:
        assert np.array_equal(rs.rsgm_group_boxes(big, *iou), orc.merge_boxes(big, iou[0], iou[1], 0)), iou
