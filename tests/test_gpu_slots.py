"""Per-slot frames (rsgm_slot_frame), the basis of continuous batching: in one
handle of B streams, each stream advances only in the frames where its slot
is active, and new streams enter with a full-range frame.  Every slot's
results must be bit-identical to the same stream run alone on a handle of its
own, whatever the roles of the other slots; idle slots keep their state; one
stream is also checked against the oracle chained over its frames."""
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


W, H, D = 200, 96, 48


def _streams(n, nframes):
    import synth
    return [synth.kitti_like_sequence(1500 + i, n_frames=nframes, width=W, height=H, f=150.0, baseline=0.54,
                                      device="cuda") for i in range(n)]


@pytest.mark.parametrize("radius_mode", [0, 2])
def test_slots_match_streams_run_alone(rs, orc, radius_mode):
    B, nframes = 3, 5
    seqs = _streams(B, nframes)
    K = seqs[0]["K"]
    # per tick, the frame each slot runs (None: idle); slot 1 starts late and
    # slot 2 sits frames out
    plan = [(0, None, 0), (1, 0, None), (2, 1, 1), (None, 2, None), (3, 3, 2), (4, None, 3)]
    P = rs.rsgm_default_params(W, H, max_disp=D, radius=4, batch=B, radius_mode=radius_mode)
    P1 = rs.rsgm_default_params(W, H, max_disp=D, radius=4, batch=1, radius_mode=radius_mode)
    alone = [rs.Stream(P1) for _ in range(B)]
    L = torch.zeros(B, H, W, dtype=torch.uint8, device="cuda")
    R = torch.zeros_like(L)
    with rs.Stream(P) as pool:
        prev = None
        for tick in plan:
            roles, Rm, tv = [], torch.eye(3).repeat(B, 1, 1), torch.zeros(B, 3)
            for b, k in enumerate(tick):
                if k is None:
                    roles.append(rs.RSGM_SLOT_IDLE)
                    continue
                roles.append(rs.RSGM_SLOT_FULL if k == 0 else rs.RSGM_SLOT_REDUCED)
                L[b], R[b] = seqs[b]["left"][k], seqs[b]["right"][k]
                Rm[b], tv[b] = seqs[b]["R"][k], seqs[b]["t"][k]
                if k == 0:
                    alone[b].full_frame(L[b], R[b])
                else:
                    alone[b].reduced_frame(L[b], R[b], Rm[b:b + 1], tv[b:b + 1], K, 0.54)
            rs.rsgm_slot_frame(pool.handle, roles, L, R, Rm, tv, K, 0.54)
            got = [x.clone() for x in pool.state()]
            for b, k in enumerate(tick):
                if k is not None:
                    for u, v in zip(got, alone[b].state()):
                        assert torch.equal(u[b], v[0]), (tick, b)
                elif prev is not None:
                    for u, v in zip(got, prev):
                        assert torch.equal(u[b], v[b]), ("idle slot changed", tick, b)
            prev = got
        # slot 0 ran frames 0..4 in ticks 0, 1, 2, 4, 5: against the oracle
        g = read_all(rs, pool)
        op = oracle_params(orc, P1)
        s0 = seqs[0]
        Ln, Rn = s0["left"].cpu().numpy(), s0["right"].cpu().numpy()
        o = orc.frame(op, Ln[0], Rn[0])
        for k in range(1, 5):
            o = orc.frame(op, Ln[k], Rn[k], state=(o["d"], o["p"]),
                          motion=(s0["R"][k].cpu().numpy(), s0["t"][k].cpu().numpy(), K.cpu().numpy(), 0.54))
        assert compare_stream(g, 0, o, H, W)["bit_equal_f32"]
    for a in alone:
        a.close()


def test_slot_frame_arguments(rs):
    P = rs.rsgm_default_params(64, 32, max_disp=16, batch=2)
    z = torch.zeros(2, 32, 64, dtype=torch.uint8, device="cuda")
    K = torch.tensor([[30.0, 0, 31.5], [0, 30.0, 15.5], [0, 0, 1]])
    eye, zero = torch.eye(3).repeat(2, 1, 1), torch.zeros(2, 3)
    with rs.Stream(P) as s:
        with pytest.raises(rs.RsgmError) as e:   # a reduced slot without a state
            rs.rsgm_slot_frame(s.handle, [rs.RSGM_SLOT_FULL, rs.RSGM_SLOT_REDUCED], z, z, eye, zero, K, 0.5)
        assert e.value.code == rs.RSGM_ERR_NO_STATE
        with pytest.raises(rs.RsgmError) as e:
            rs.rsgm_slot_frame(s.handle, [3, 0], z, z, eye, zero, K, 0.5)
        assert e.value.code == rs.RSGM_ERR_INVALID_ARG
        rs.rsgm_slot_frame(s.handle, [rs.RSGM_SLOT_IDLE] * 2, z, z, eye, zero, K, 0.5)   # nothing to do
        rs.rsgm_slot_frame(s.handle, [rs.RSGM_SLOT_FULL, rs.RSGM_SLOT_IDLE], z, z, eye, zero, K, 0.5)
        with pytest.raises(rs.RsgmError) as e:   # stream 1 has no state yet
            s.reduced_frame(z, z, eye, zero, K, 0.5)
        assert e.value.code == rs.RSGM_ERR_NO_STATE
        rs.rsgm_slot_frame(s.handle, [rs.RSGM_SLOT_REDUCED, rs.RSGM_SLOT_FULL], z, z, eye, zero, K, 0.5)
        s.reduced_frame(z, z, eye, zero, K, 0.5)
        frames = s.counters()[0]
        assert frames == 1 + 2 + 2
