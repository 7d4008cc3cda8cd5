"""Mixed-resolution groups (several handles of different geometry, one CUDA
graph launch per tick) and the schedule autotuner: results are the same,
bit for bit, alone and in the mix, and the same whatever schedule the tuner
picks; one member is also checked against the oracle."""
import numpy as np
import pytest
import torch

from parity_util import compare_stream, oracle_params, read_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


GEOMS = [  # (B, W, H, D, f)
    (2, 160, 120, 32, 100.0),
    (2, 300, 90, 64, 200.0),
    (1, 200, 150, 96, 250.0),
]


def _inputs(nframes):
    import synth
    out = []
    for gi, (B, W, H, D, f) in enumerate(GEOMS):
        seqs = [synth.kitti_like_sequence(300 + 10 * gi + b, n_frames=nframes, width=W, height=H, f=f,
                                          baseline=0.54) for b in range(B)]
        st = lambda k: torch.stack([q[k] for q in seqs])
        out.append(dict(L=st("left"), R=st("right"), Rm=st("R"), t=st("t"), K=seqs[0]["K"]))
    return out


def _params(rs, B, W, H, D):
    return rs.rsgm_default_params(W, H, max_disp=D, radius=4, batch=B)


def test_group_matches_members_run_alone(rs, orc):
    nframes = 4
    data = _inputs(nframes)
    stream = torch.cuda.current_stream()
    alone, grouped = [], []
    for (B, W, H, D, f), x in zip(GEOMS, data):
        alone.append(rs.Stream(_params(rs, B, W, H, D), stream))
        grouped.append(rs.Stream(_params(rs, B, W, H, D), stream))
    group = rs.rsgm_group_create([s.handle for s in grouped])
    try:
        for k in range(nframes):
            L = [x["L"][:, k].cuda().contiguous() for x in data]
            R = [x["R"][:, k].cuda().contiguous() for x in data]
            if k == 0:
                for s, l, r in zip(alone + grouped, L + L, R + R):
                    s.full_frame(l, r)
                continue
            for s, x, l, r in zip(alone, data, L, R):
                s.reduced_frame(l, r, x["Rm"][:, k].contiguous(), x["t"][:, k].contiguous(), x["K"], 0.54)
            rs.rsgm_group_reduced_frame(group, L, R, [x["Rm"][:, k].contiguous() for x in data],
                                        [x["t"][:, k].contiguous() for x in data], [x["K"] for x in data],
                                        [0.54] * len(data))
            if k == 2:   # tune the members' schedules in the middle of the sequence
                for s in grouped:
                    rs.rsgm_autotune(s.handle)
            for a, b in zip(alone, grouped):
                for u, v in zip(a.state(), b.state()):
                    assert torch.equal(u, v), "frame %d" % k
        # one member against the oracle on the last frame
        g = read_all(rs, grouped[1])
        B, W, H, D, f = GEOMS[1]
        op = oracle_params(orc, _params(rs, B, W, H, D))
        x = data[1]
        for b in range(B):
            st = None
            for k in range(nframes):
                if k == 0:
                    o = orc.frame(op, x["L"][b, 0].numpy(), x["R"][b, 0].numpy())
                else:
                    o = orc.frame(op, x["L"][b, k].numpy(), x["R"][b, k].numpy(), state=st,
                                  motion=(x["Rm"][b, k].numpy(), x["t"][b, k].numpy(), x["K"].numpy(), 0.54))
                st = (o["d"], o["p"])
            compare_stream(g, b, o, H, W)
    finally:
        rs.rsgm_group_destroy(group)
        for s in alone + grouped:
            s.close()


def test_group_with_a_full_hd_d256_member_against_the_oracle(rs, orc):
    # The largest geometry of the mixed-resolution batch (1920x1080, 256
    # disparities) inside a group beside a small member; both are checked
    # against the oracle chained over the same frames.
    import synth
    geoms = [(1, 1920, 1080, 256, 1000.0), (2, 160, 120, 32, 100.0)]
    nframes = 3
    data = []
    for gi, (B, W, H, D, f) in enumerate(geoms):
        seqs = [synth.kitti_like_sequence(900 + 10 * gi + b, n_frames=nframes, width=W, height=H, f=f,
                                          baseline=0.54, device="cuda") for b in range(B)]
        st = lambda k: torch.stack([q[k] for q in seqs])
        data.append(dict(L=st("left"), R=st("right"), Rm=st("R").cpu(), t=st("t").cpu(), K=seqs[0]["K"].cpu()))
    stream = torch.cuda.current_stream()
    members = [rs.Stream(_params(rs, B, W, H, D), stream) for (B, W, H, D, f) in geoms]
    group = rs.rsgm_group_create([m.handle for m in members])
    try:
        for m, x in zip(members, data):
            m.full_frame(x["L"][:, 0].contiguous(), x["R"][:, 0].contiguous())
        for k in range(1, nframes):
            rs.rsgm_group_reduced_frame(group, [x["L"][:, k].contiguous() for x in data],
                                        [x["R"][:, k].contiguous() for x in data],
                                        [x["Rm"][:, k].contiguous() for x in data],
                                        [x["t"][:, k].contiguous() for x in data], [x["K"] for x in data],
                                        [0.54] * len(data))
        for m, (B, W, H, D, f), x in zip(members, geoms, data):
            g = read_all(rs, m)
            op = oracle_params(orc, _params(rs, B, W, H, D))
            for b in range(B):
                Lb, Rb = x["L"][b].cpu().numpy(), x["R"][b].cpu().numpy()
                o = orc.frame(op, Lb[0], Rb[0])
                for k in range(1, nframes):
                    o = orc.frame(op, Lb[k], Rb[k], state=(o["d"], o["p"]),
                                  motion=(x["Rm"][b, k].numpy(), x["t"][b, k].numpy(), x["K"].numpy(), 0.54))
                stats = compare_stream(g, b, o, H, W)
                assert stats["bit_equal_f32"]
    finally:
        rs.rsgm_group_destroy(group)
        for m in members:
            m.close()


def test_group_rejects_host_images_and_mixed_streams(rs):
    P = rs.rsgm_default_params(64, 32, max_disp=16)
    with rs.Stream(P) as a, rs.Stream(P, torch.cuda.Stream()) as b:
        with pytest.raises(rs.RsgmError) as e:
            rs.rsgm_group_create([a.handle, b.handle])
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG
        z = torch.zeros(32, 64, dtype=torch.uint8, device="cuda")
        a.full_frame(z, z)
        g = rs.rsgm_group_create([a.handle])
        try:
            zh = torch.zeros(32, 64, dtype=torch.uint8)
            K = torch.tensor([[30.0, 0, 31.5], [0, 30.0, 15.5], [0, 0, 1]])
            with pytest.raises(rs.RsgmError) as e:
                rs.rsgm_group_reduced_frame(g, [zh], [zh], [torch.eye(3)[None]], [torch.zeros(1, 3)], [K], [0.5])
            assert e.value.code == rs.RSGM_ERR_INVALID_ARG
        finally:
            rs.rsgm_group_destroy(g)


@pytest.mark.parametrize("mask", [0x01, 0x02, 0x0F])
def test_every_row_schedule_gives_the_same_aggregation(rs, mask):
    # rows per horizontal warp (8, 16, 32) and register capacities, for one
    # horizontal direction alone and for both (a row pair)
    B, W, H, D, f = 2, 240, 100, 64, 150.0
    import synth
    seqs = [synth.kitti_like_sequence(720 + b, n_frames=3, width=W, height=H, f=f, baseline=0.54) for b in range(B)]
    st = lambda k: torch.stack([q[k] for q in seqs])
    L, R, Rm, t, K = st("left"), st("right"), st("R"), st("t"), seqs[0]["K"]
    P = rs.rsgm_default_params(W, H, max_disp=D, radius=4, batch=B, path_mask=mask)
    results = {}
    for cells in (0, 2, 18):
        for rows in (0, 8, 32):
            with rs.Stream(P) as s:
                rs.rsgm_set_schedule(s.handle, cells)
                rs.rsgm_set_rows_per_warp(s.handle, rows)
                s.full_frame(L[:, 0].cuda().contiguous(), R[:, 0].cuda().contiguous())
                for k in (1, 2):
                    s.reduced_frame(L[:, k].cuda().contiguous(), R[:, k].cuda().contiguous(), Rm[:, k].contiguous(),
                                    t[:, k].contiguous(), K, 0.54)
                results[(cells, rows)] = [s.read(rs.RSGM_BUF_AGGREGATED, torch.int16)] + [x.cpu() for x in s.state()]
    base = results[(0, 0)]
    for key, got in results.items():
        for u, v in zip(base, got):
            assert torch.equal(u, v), key
    with rs.Stream(P) as s:
        with pytest.raises(rs.RsgmError) as e:
            rs.rsgm_set_rows_per_warp(s.handle, 12)
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG
        # the getter reports what later frames use
        assert rs.rsgm_get_schedule(s.handle) == (10, 0)      # radius 4: 9 cells, rounded up; row sweep
        rs.rsgm_set_rows_per_warp(s.handle, 16)
        rs.rsgm_set_schedule(s.handle, 5)                      # resets the rows to the row sweep
        assert rs.rsgm_get_schedule(s.handle) == (6, 0)
        rs.rsgm_set_rows_per_warp(s.handle, 32)
        assert rs.rsgm_get_schedule(s.handle) == (6, 32)
        s.full_frame(L[:, 0].cuda().contiguous(), R[:, 0].cuda().contiguous())
        rs.rsgm_autotune(s.handle)
        cells, rows = rs.rsgm_get_schedule(s.handle)
        assert cells in (2, 6, 10, 18) and rows in ((0, 8, 16, 32) if mask & 3 else (0,))


@pytest.mark.parametrize("radius", [2, 4, 8])
def test_every_schedule_gives_the_same_aggregation(rs, radius):
    # Eq. 1 is exact in integers, so S and the state must not depend on how
    # many path lines a warp carries; oversized requests are capped.
    B, W, H, D, f = 3, 240, 100, 64, 150.0
    import synth
    seqs = [synth.kitti_like_sequence(700 + b, n_frames=3, width=W, height=H, f=f, baseline=0.54) for b in range(B)]
    st = lambda k: torch.stack([q[k] for q in seqs])
    L, R, Rm, t, K = st("left"), st("right"), st("R"), st("t"), seqs[0]["K"]
    P = rs.rsgm_default_params(W, H, max_disp=D, radius=radius, batch=B)
    results = {}
    for sched in [0, 1, 2, 3, 5, 7, 16, 32]:
        with rs.Stream(P) as s:
            rs.rsgm_set_schedule(s.handle, sched)
            s.full_frame(L[:, 0].cuda().contiguous(), R[:, 0].cuda().contiguous())
            for k in (1, 2):
                s.reduced_frame(L[:, k].cuda().contiguous(), R[:, k].cuda().contiguous(), Rm[:, k].contiguous(),
                                t[:, k].contiguous(), K, 0.54)
            results[sched] = [s.read(rs.RSGM_BUF_AGGREGATED, torch.int16)] + [x.cpu() for x in s.state()]
    base = results[0]
    for sched, got in results.items():
        for u, v in zip(base, got):
            assert torch.equal(u, v), "schedule %d" % sched


def test_set_schedule_rejects_out_of_range(rs):
    P = rs.rsgm_default_params(64, 32, max_disp=16)
    with rs.Stream(P) as s:
        for bad in (-1, 33):
            with pytest.raises(rs.RsgmError) as e:
                rs.rsgm_set_schedule(s.handle, bad)
            assert e.value.code == rs.RSGM_ERR_INVALID_ARG
