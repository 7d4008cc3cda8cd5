"""The request loop on the GPU: streams of different resolutions arrive as
Poisson processes; streams of one geometry share launches of a pool handle
(continuous batching) and pools overlap on the device.  Every stream's final
state is bit-identical to the same frames run alone on a handle of its own,
for the fixed and for the learned search window, and equal to the oracle's
state chained over the stream's frames (integers bit-exact, the Kalman mean
and variance within 1e-5 relative of the single-precision oracle)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_07986_gb300 import build
    build.build()
    import paper_1809_07986_gb300 as rs
    return rs


GEOMS = [(160, 120, 32, 100.0), (200, 100, 48, 150.0), (160, 120, 32, 100.0), (240, 96, 64, 200.0),
         (200, 100, 48, 150.0), (160, 120, 32, 100.0)]


def _mix(seed, geoms, frames=(4, 8), rates=(20, 60), spread=0.05):
    import synth
    from paper_1809_07986_gb300.serving import StreamSpec, poisson_arrivals
    rng = np.random.default_rng(seed)
    specs, data = [], {}
    for i, (W, H, D, f) in enumerate(geoms):
        n = int(rng.integers(frames[0], frames[1]))
        s = synth.kitti_like_sequence(800 + 10 * seed + i, n_frames=n, width=W, height=H, f=f, baseline=0.54,
                                      device="cuda")
        data[i] = dict(left=s["left"], right=s["right"], R=s["R"], t=s["t"], K=s["K"], baseline=0.54)
        start = float(rng.uniform(0.0, spread))
        specs.append(StreamSpec(i, W, H, D, start, poisson_arrivals(rng, start, float(rng.uniform(*rates)), n)))
    return specs, data


def _alone(rs, backend, spec, f):
    with rs.Stream(backend.params(spec.geometry, 1)) as st:
        if backend.cnn:
            rs.rsgm_attach_cnn(st.handle, backend.cnn)
        for k in range(len(spec.arrivals_s)):
            if k == 0:
                st.full_frame(f["left"][0], f["right"][0])
            else:
                st.reduced_frame(f["left"][k], f["right"][k], f["R"][k:k + 1], f["t"][k:k + 1], f["K"], 0.54)
        return [x[0] for x in st.state()]


@pytest.mark.parametrize("learned", [False, True])
def test_serving_results_equal_alone_results(rs, learned):
    from paper_1809_07986_gb300 import learned as LO
    from paper_1809_07986_gb300.serving import GpuBackend, serve
    specs, frames = _mix(5, GEOMS[:4])
    backend = GpuBackend(frames, network=LO.init_params(3) if learned else None)
    try:
        # room for two slots of the largest pool: some streams wait for a slot
        budget = sum(backend.footprint(g, 1) for g in {s.geometry for s in specs}) + backend.footprint(
            specs[0].geometry, 1)
        rep = serve(specs, backend, budget_bytes=budget)
        assert rep.frames == sum(len(s.arrivals_s) for s in specs) and rep.order_ok
        assert rep.pool_bytes <= budget
        for spec in specs:
            for a, b in zip(_alone(rs, backend, spec, frames[spec.sid]), backend.finals[spec.sid]):
                assert torch.equal(a, b), spec.sid
    finally:
        backend.close()


def _oracle_final(orc, spec, f):
    op = orc.Params(spec.width, spec.height, max_disp=spec.max_disp, radius=spec.radius)
    L, R = f["left"].cpu().numpy(), f["right"].cpu().numpy()
    o = orc.frame(op, L[0], R[0])
    for k in range(1, len(spec.arrivals_s)):
        o = orc.frame(op, L[k], R[k], state=(o["d"], o["p"]),
                      motion=(f["R"][k].cpu().numpy(), f["t"][k].cpu().numpy(), f["K"].cpu().numpy(), f["baseline"]))
    return o


def test_served_streams_match_the_chained_oracle(rs, orc):
    from paper_1809_07986_gb300.serving import GpuBackend, serve
    specs, frames = _mix(11, GEOMS)
    backend = GpuBackend(frames)
    rep = serve(specs, backend, budget_bytes=10 ** 11)
    assert rep.frames == sum(len(s.arrivals_s) for s in specs) and rep.order_ok
    for spec in specs:
        o = _oracle_final(orc, spec, frames[spec.sid])
        d, p, m, di = (x.cpu().numpy().reshape(spec.height, spec.width) for x in backend.finals[spec.sid])
        np.testing.assert_array_equal(di, o["d_int"], "integer disparity, stream %d" % spec.sid)
        np.testing.assert_array_equal(m, o["mask"], "moving mask, stream %d" % spec.sid)
        for got, want, what in ((d, o["d"], "mean"), (p, o["p"], "variance")):
            rel = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1e-30)
            assert rel.max() <= 1e-5, "Kalman %s of stream %d: rel err %g" % (what, spec.sid, rel.max())
