"""GPU parity of the post-path steps: the 3x3 median output (Section 2.3) and
the moving-object boxes (Section 4), bit-exact against the oracle on the same
frames (both sides compute from their own, bit-equal, path outputs)."""
import numpy as np
import pytest
import torch

from parity_util import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


def _run(rs, orc, P, L, R, Rm, tv, K, b, nframes, dparams):
    op = oracle_params(orc, P)
    B, H, W = P.batch, P.height, P.width
    ok_boxes = 0
    with rs.Stream(P) as gs:
        states = [None] * B
        for k in range(nframes):
            l, r = L[:, k].cuda().contiguous(), R[:, k].cuda().contiguous()
            if k == 0:
                gs.full_frame(l, r)
            else:
                gs.reduced_frame(l, r, Rm[:, k].contiguous(), tv[:, k].contiguous(), K, b)
            med = torch.empty(B, H, W, device="cuda")
            rs.rsgm_median(gs.handle, med)
            gboxes, counts = rs.rsgm_detect(gs.handle, dparams, B, capacity=512)
            med = med.cpu().numpy()
            for s in range(B):
                if k == 0:
                    o = orc.frame(op, L[s, k].numpy(), R[s, k].numpy())
                else:
                    o = orc.frame(op, L[s, k].numpy(), R[s, k].numpy(), state=states[s],
                                  motion=(Rm[s, k].numpy(), tv[s, k].numpy(), K.numpy(), b))
                states[s] = (o["d"], o["p"])
                np.testing.assert_array_equal(med[s], orc.median3(o["d"]), "median")
                D = orc.DetectParams(sizes=tuple(tuple(dparams.sizes[i]) for i in range(dparams.nsizes)),
                                     stride=dparams.stride, skip_top_fraction_num=dparams.skip_num,
                                     skip_top_fraction_den=dparams.skip_den, thresh_px=dparams.thresh_px,
                                     iou_num=dparams.iou_num, iou_den=dparams.iou_den, min_area=dparams.min_area)
                want, raw, _ = orc.detect(o["nu"], o["cls"], D)
                assert counts[s] == len(want), (k, s, counts[s], len(want))
                np.testing.assert_array_equal(gboxes[s], want.reshape(-1, 4), "boxes")
                ok_boxes += len(want)
    return ok_boxes


def test_tiny_pair_median_and_boxes(rs, orc):
    import synth
    seqs = [synth.tiny_pair(s) for s in (1, 2)]
    st = lambda key: torch.stack([q[key] for q in seqs])
    P = rs.rsgm_default_params(384, 128, max_disp=64, radius=4, batch=2)
    n = _run(rs, orc, P, st("left"), st("right"), st("R"), st("t"), seqs[0]["K"], seqs[0]["baseline"], 2,
             rs.rsgm_default_detect_params(min_area=400))
    assert n >= 1   # the independently moving box is found


@pytest.mark.parametrize("over", [dict(), dict(iou_num=1, iou_den=4, min_area=0),
                                  dict(sizes=[(16, 24), (64, 32)], stride=7, thresh_px=0.5, skip_num=0)])
def test_kitti_shaped_median_and_boxes(rs, orc, over):
    import synth
    seqs = [synth.kitti_like_sequence(s, n_frames=3, device="cpu") for s in (61, 62)]
    st = lambda key: torch.stack([q[key] for q in seqs])
    P = rs.rsgm_default_params(1242, 375, max_disp=128, radius=4, batch=2)
    _run(rs, orc, P, st("left"), st("right"), st("R"), st("t"), seqs[0]["K"], 0.54, 3,
         rs.rsgm_default_detect_params(**over))


def test_detect_rejects_bad_parameters(rs):
    P = rs.rsgm_default_params(64, 32, max_disp=16)
    with rs.Stream(P) as gs:
        p = rs.rsgm_default_detect_params()
        with pytest.raises(rs.RsgmError) as e:
            rs.rsgm_detect(gs.handle, p, 1)
        assert e.value.code == rs.RSGM_ERR_NO_STATE
        z = torch.zeros(32, 64, dtype=torch.uint8, device="cuda")
        gs.full_frame(z, z)
        p.stride = 0
        with pytest.raises(rs.RsgmError) as e:
            rs.rsgm_detect(gs.handle, p, 1)
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG
