"""The allocation-free offsets entry point (rsgm_window_offsets_noalloc).

It serves callers that cannot call cudaMalloc, so its scratch is a fixed
array inside the library.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run every other
test.  The check: on windows produced by a real reduced frame, two calls in a
row reproduce, exactly, the offsets the library computed for that frame
through its normal (allocating) entry points.
"""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


def _frame_buffers(rs, seeds):
    import synth
    seqs = [synth.tiny_pair(s) for s in seeds]
    L = torch.stack([q["left"] for q in seqs])
    R = torch.stack([q["right"] for q in seqs])
    Rm = torch.stack([q["R"] for q in seqs])
    tv = torch.stack([q["t"] for q in seqs])
    P = rs.rsgm_default_params(384, 128, max_disp=64, radius=4, batch=len(seeds))
    with rs.Stream(P) as gs:
        gs.full_frame(L[:, 0].cuda().contiguous(), R[:, 0].cuda().contiguous())
        gs.reduced_frame(L[:, 1].cuda().contiguous(), R[:, 1].cuda().contiguous(), Rm[:, 1].contiguous(),
                         tv[:, 1].contiguous(), seqs[0]["K"], seqs[0]["baseline"])
        win = gs.read(rs.RSGM_BUF_WINDOW, torch.int32)
        off = gs.read(rs.RSGM_BUF_OFFSET, torch.int32)
        last = gs.counters()[2]
    return win, off, last


@pytest.mark.gpu
def test_noalloc_offsets_match_the_library_on_two_calls_in_a_row(rs):
    win, off, last = _frame_buffers(rs, [11, 12])
    rows, width = 2 * 128, 384
    dwin = win.cuda()
    for call in range(2):
        out = torch.full_like(dwin, -1)
        tot = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rs.rsgm_window_offsets_noalloc(dwin, width, rows, out, tot, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(out.cpu(), off), "call %d" % call
        assert int(tot.item()) & 0xFFFFFFFF == last
    # a different input right after: no state carried between calls
    full = torch.full_like(dwin, 64 << 16)
    out = torch.empty_like(dwin)
    rs.rsgm_window_offsets_noalloc(full, width, rows, out, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    expect = np.arange(rows * width, dtype=np.int64) * 64
    assert np.array_equal(out.cpu().numpy().view(np.uint32).astype(np.int64), expect)


@pytest.mark.gpu
def test_noalloc_rejects_more_rows_than_its_scratch(rs):
    dwin = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(rs.RsgmError) as e:
        rs.rsgm_window_offsets_noalloc(dwin, 1, 65537, dwin)
    assert e.value.code == rs.RSGM_ERR_INVALID_ARG
