"""GPU parity: the CUDA path (through the C ABI) against the oracle, stage by
stage, on seeded synthetic inputs.  Integer stages and single-precision
decision values must be bit-exact; the Kalman mean and variance within 1e-5
relative of the single-precision oracle, with the double-precision difference
bounded by single-precision rounding."""
import numpy as np
import pytest
import torch

from parity_util import compare_stream, oracle_params, read_all, run_sequence

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


def batch_sequences(seeds, nframes, width, height, f, baseline, device="cpu"):
    import synth
    seqs = [synth.kitti_like_sequence(s, n_frames=nframes, width=width, height=height, f=f,
                                      baseline=baseline, device=device) for s in seeds]
    st = lambda k: torch.stack([q[k] for q in seqs])
    return st("left").cpu(), st("right").cpu(), st("R"), st("t"), seqs[0]["K"], baseline


def tiny_batch(seeds):
    import synth
    seqs = [synth.tiny_pair(s) for s in seeds]
    st = lambda k: torch.stack([q[k] for q in seqs])
    return st("left"), st("right"), st("R"), st("t"), seqs[0]["K"], seqs[0]["baseline"]


# ------------------------------------------------------------------ the tiny workload

def test_tiny_pair_full_then_reduced(rs, orc):
    L, R, Rm, tv, K, b = tiny_batch([1])
    P = rs.rsgm_default_params(384, 128, max_disp=64, radius=4)
    stats = run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 2)
    assert stats[1]["ncells"] < stats[0]["ncells"] / 3


@pytest.mark.parametrize("overrides", [
    dict(path_mask=0x0F), dict(path_mask=0xF0), dict(path_mask=0x10), dict(path_mask=0x02),
    dict(census_w=7, census_h=7), dict(census_w=9, census_h=7), dict(census_w=3, census_h=3),
    dict(radius_mode=1), dict(radius_mode=2), dict(radius_mode=2, max_disp=128), dict(radius=0), dict(radius=16),
    dict(P1=30, P2=12), dict(P1=0, P2=0), dict(tau_disc=0.5, p_reset=40.0), dict(gate_gamma=0.5, q=0.0),
])
def test_tiny_pair_parameter_variants(rs, orc, overrides):
    L, R, Rm, tv, K, b = tiny_batch([2])
    P = rs.rsgm_default_params(384, 128, **{"max_disp": 64, "radius": 4, **overrides})
    run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 2)


def test_tiny_batch_of_three_streams(rs, orc):
    L, R, Rm, tv, K, b = tiny_batch([3, 4, 5])
    P = rs.rsgm_default_params(384, 128, max_disp=64, radius=4, batch=3)
    run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 2)


# ------------------------------------------------------------------ ragged sizes, several frames

def test_odd_sizes_several_frames_batch(rs, orc):
    L, R, Rm, tv, K, b = batch_sequences([21, 22], 4, 77, 45, 60.0, 0.54)
    P = rs.rsgm_default_params(77, 45, max_disp=37, radius=3, batch=2)
    run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 4)


def test_wide_disparity_range_256(rs, orc):
    L, R, Rm, tv, K, b = batch_sequences([31], 3, 300, 40, 720.0, 0.54)
    P = rs.rsgm_default_params(300, 40, max_disp=256, radius=8)
    run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 3)


# ------------------------------------------------------------------ the paper-shaped workload

@pytest.mark.parametrize("radius", [2, 4, 8])
def test_kitti_shaped_frames(rs, orc, radius):
    L, R, Rm, tv, K, b = batch_sequences([40 + radius], 3, 1242, 375, 721.0, 0.54)
    P = rs.rsgm_default_params(1242, 375, max_disp=128, radius=radius)
    stats = run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 3)
    assert all(s["bit_equal_f32"] for s in stats)
    print("f64 oracle: max rel err of d %.3g (operand-relative %.3g), of p %.3g" % (
        max(s["max_rel_d_vs_f64"] for s in stats), max(s["max_operand_rel_d_vs_f64"] for s in stats),
        max(s["max_rel_p_vs_f64"] for s in stats)))


def test_kitti_shaped_sixteen_consecutive_frames(rs, orc):
    # One paper-shaped stream over a full-range frame and 15 reduced frames:
    # the state carried from frame to frame (Section 2.4) stays identical to
    # the oracle's at every frame, not only after the first prediction.
    L, R, Rm, tv, K, b = batch_sequences([77], 16, 1242, 375, 721.0, 0.54, device="cuda")
    P = rs.rsgm_default_params(1242, 375, max_disp=128, radius=4)
    stats = run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 16)
    assert len(stats) == 16 and all(s["bit_equal_f32"] for s in stats)
    assert all(s["ncells"] < stats[0]["ncells"] / 3 for s in stats[1:])


def test_kitti_shaped_batch_in_the_benchmark_launch_configuration(rs, orc):
    # 32 streams as in the throughput benchmark; the oracle checks two of them.
    B = 32
    L, R, Rm, tv, K, b = batch_sequences(list(range(100, 100 + B)), 2, 1242, 375, 721.0, 0.54, device="cuda")
    P = rs.rsgm_default_params(1242, 375, max_disp=128, radius=4, batch=B)
    run_sequence(rs, orc, P, L, R, Rm, tv, K, b, 2, streams_to_check=[0, B - 1])


# ------------------------------------------------------------------ degenerate shapes and states

def random_pair(seed, H, W, shift):
    g = np.random.default_rng(seed)
    left = g.integers(0, 256, (H, W), dtype=np.uint8)
    right = g.integers(0, 256, (H, W), dtype=np.uint8)
    if shift < W:
        right[:, : W - shift] = left[:, shift:]
    return left, right


@pytest.mark.parametrize("H,W,D", [(1, 40, 8), (40, 1, 4), (1, 1, 1), (3, 3, 2), (17, 33, 1), (5, 300, 256)])
def test_degenerate_shapes(rs, orc, H, W, D):
    frames = [random_pair(7 + k, H, W, min(3, D - 1)) for k in range(2)]
    L = torch.from_numpy(np.stack([f[0] for f in frames]))[None]
    R = torch.from_numpy(np.stack([f[1] for f in frames]))[None]
    Rm = torch.eye(3).repeat(1, 2, 1, 1)
    tv = torch.tensor([[[0.0, 0.0, 0.0], [0.0, 0.0, -0.3]]])
    K = torch.tensor([[50.0, 0.0, (W - 1) / 2], [0.0, 50.0, (H - 1) / 2], [0.0, 0.0, 1.0]])
    P = rs.rsgm_default_params(W, H, max_disp=D, radius=1)
    run_sequence(rs, orc, P, L, R, Rm, tv, K, 0.5, 2)


def test_state_without_any_valid_disparity_searches_everything(rs, orc):
    left, right = random_pair(3, 30, 50, 4)
    P = rs.rsgm_default_params(50, 30, max_disp=16, radius=2)
    zero = np.zeros((30, 50), np.float32)
    K = torch.tensor([[50.0, 0.0, 24.5], [0.0, 50.0, 14.5], [0.0, 0.0, 1.0]])
    with rs.Stream(P) as gs:
        gs.set_state(torch.zeros(1, 30, 50, device="cuda"), torch.ones(1, 30, 50, device="cuda"))
        gs.reduced_frame(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                         torch.eye(3)[None], torch.zeros(1, 3), K, 0.5)
        g = read_all(rs, gs)
    o = orc.frame(oracle_params(orc, P), left, right, state=(zero, np.ones_like(zero)),
                  motion=(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), K.numpy(), 0.5))
    assert (o["cls"] == 2).all()
    compare_stream(g, 0, o, 30, 50)


# ------------------------------------------------------------------ host buffers, resume, errors

def test_host_buffers_match_device_buffers(rs):
    L, R, Rm, tv, K, b = tiny_batch([6, 7])
    P = rs.rsgm_default_params(384, 128, max_disp=64, radius=4, batch=2)
    outs = []
    for mode in ("device", "pinned", "pageable"):
        with rs.Stream(P, torch.cuda.current_stream()) as gs:
            for k in range(2):
                l, r = L[:, k].contiguous(), R[:, k].contiguous()
                if mode == "device":
                    l, r = l.cuda(), r.cuda()
                elif mode == "pinned":
                    l, r = l.pin_memory(), r.pin_memory()
                if k == 0:
                    gs.full_frame(l, r)
                else:
                    gs.reduced_frame(l, r, Rm[:, k].contiguous(), tv[:, k].contiguous(), K, b)
            d = torch.empty(2, 128, 384).pin_memory() if mode != "device" else torch.empty(2, 128, 384, device="cuda")
            m = torch.empty(2, 128, 384, dtype=torch.uint8)
            rs.rsgm_state(gs.handle, d, None, m if mode != "device" else None, None)
            gs.sync()
            outs.append(d.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_resume_from_exported_state_is_bit_identical(rs):
    L, R, Rm, tv, K, b = batch_sequences([55], 4, 160, 64, 120.0, 0.54)
    P = rs.rsgm_default_params(160, 64, max_disp=48, radius=3)

    def step(gs, k):
        l, r = L[:, k].cuda().contiguous(), R[:, k].cuda().contiguous()
        if k == 0:
            gs.full_frame(l, r)
        else:
            gs.reduced_frame(l, r, Rm[:, k].contiguous(), tv[:, k].contiguous(), K, b)

    with rs.Stream(P) as a:
        for k in range(4):
            step(a, k)
            if k == 1:
                d1, p1, _, _ = a.state()
        ref = a.state()
    with rs.Stream(P) as c:
        c.set_state(d1, p1)
        for k in (2, 3):
            step(c, k)
        got = c.state()
    for x, y in zip(ref, got):
        assert torch.equal(x, y)


def test_reduced_before_full_reports_no_state(rs):
    P = rs.rsgm_default_params(32, 16, max_disp=8)
    z = torch.zeros(16, 32, dtype=torch.uint8, device="cuda")
    with rs.Stream(P) as gs:
        with pytest.raises(rs.RsgmError) as e:
            gs.reduced_frame(z, z, torch.eye(3)[None], torch.zeros(1, 3),
                             torch.tensor([[20.0, 0, 15.5], [0, 20.0, 7.5], [0, 0, 1]]), 0.5)
        assert e.value.code == rs.RSGM_ERR_NO_STATE
        with pytest.raises(rs.RsgmError) as e:   # skewed K is rejected
            gs.full_frame(z, z)
            gs.reduced_frame(z, z, torch.eye(3)[None], torch.zeros(1, 3),
                             torch.tensor([[20.0, 1.0, 15.5], [0, 20.0, 7.5], [0, 0, 1]]), 0.5)
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG


def test_counters_count_frames_and_cells(rs):
    L, R, Rm, tv, K, b = tiny_batch([8])
    P = rs.rsgm_default_params(384, 128, max_disp=64, radius=4)
    with rs.Stream(P) as gs:
        gs.full_frame(L[:, 0].cuda().contiguous(), R[:, 0].cuda().contiguous())
        f, c, last = gs.counters()
        assert (f, c, last) == (1, 384 * 128 * 64, 384 * 128 * 64)
        gs.reduced_frame(L[:, 1].cuda().contiguous(), R[:, 1].cuda().contiguous(), Rm[:, 1], tv[:, 1], K, b)
        f2, c2, last2 = gs.counters()
        wd = (gs.read(rs.RSGM_BUF_WINDOW, torch.int32).numpy().view(np.uint32) >> 16).sum()
        assert f2 == 2 and last2 == wd and c2 == c + wd
