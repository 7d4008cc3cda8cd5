"""The request loop on the GPU: streams of different resolutions arrive as
Poisson processes and overlap on the device; every stream's final state is
bit-identical to the same frames run alone on a fresh handle, and equal to
the oracle's state chained over the stream's frames (integers bit-exact, the
Kalman mean and variance within 1e-5 relative of the single-precision
oracle)."""
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


def test_serving_results_equal_alone_results(rs):
    import synth
    from paper_1809_07986_gb300.serving import GpuBackend, StreamSpec, poisson_arrivals, serve
    rng = np.random.default_rng(5)
    geoms = [(160, 120, 32, 100.0), (200, 100, 48, 150.0), (240, 96, 64, 200.0), (160, 120, 32, 100.0)]
    specs, frames = [], {}
    for i, (W, H, D, f) in enumerate(geoms):
        n = 6
        s = synth.kitti_like_sequence(700 + i, n_frames=n, width=W, height=H, f=f, baseline=0.54, device="cuda")
        frames[i] = dict(left=s["left"], right=s["right"], R=s["R"], t=s["t"], K=s["K"], baseline=0.54)
        specs.append(StreamSpec(i, W, H, D, 0.02 * i, poisson_arrivals(rng, 0.02 * i, 40.0, n)))
    backend = GpuBackend(frames)
    budget = sum(backend.footprint(s) for s in specs[:2])   # forces some streams to wait
    rep = serve(specs, backend, budget_bytes=budget)
    assert rep.frames == sum(len(s.arrivals_s) for s in specs) and rep.order_ok
    assert rep.peak_bytes <= max(budget, max(backend.footprint(s) for s in specs))
    for spec in specs:
        f = frames[spec.sid]
        with rs.Stream(backend.params(spec)) as st:
            for k in range(len(spec.arrivals_s)):
                if k == 0:
                    st.full_frame(f["left"][0], f["right"][0])
                else:
                    st.reduced_frame(f["left"][k], f["right"][k], f["R"][k:k + 1], f["t"][k:k + 1], f["K"], 0.54)
            alone = st.state()
        for a, b in zip(alone, backend.finals[spec.sid]):
            assert torch.equal(a, b), spec.sid


def _oracle_final(orc, spec, f):
    op = orc.Params(spec.width, spec.height, max_disp=spec.max_disp, radius=spec.radius)
    L, R = f["left"].cpu().numpy(), f["right"].cpu().numpy()
    o = orc.frame(op, L[0], R[0])
    for k in range(1, len(spec.arrivals_s)):
        o = orc.frame(op, L[k], R[k], state=(o["d"], o["p"]),
                      motion=(f["R"][k].cpu().numpy(), f["t"][k].cpu().numpy(), f["K"].cpu().numpy(), f["baseline"]))
    return o


def test_served_streams_match_the_chained_oracle(rs, orc):
    import synth
    from paper_1809_07986_gb300.serving import GpuBackend, StreamSpec, poisson_arrivals, serve
    rng = np.random.default_rng(11)
    geoms = [(160, 120, 32, 100.0), (200, 100, 48, 150.0), (160, 120, 32, 100.0), (240, 96, 64, 200.0),
             (200, 100, 48, 150.0), (160, 120, 32, 100.0)]
    specs, frames = [], {}
    for i, (W, H, D, f) in enumerate(geoms):
        n = int(rng.integers(4, 8))
        s = synth.kitti_like_sequence(800 + i, n_frames=n, width=W, height=H, f=f, baseline=0.54, device="cuda")
        frames[i] = dict(left=s["left"], right=s["right"], R=s["R"], t=s["t"], K=s["K"], baseline=0.54)
        start = float(rng.uniform(0.0, 0.05))
        specs.append(StreamSpec(i, W, H, D, start, poisson_arrivals(rng, start, float(rng.uniform(20, 60)), n)))
    backend = GpuBackend(frames)
    rep = serve(specs, backend, budget_bytes=sum(backend.footprint(s) for s in specs))
    assert rep.frames == sum(len(s.arrivals_s) for s in specs) and rep.order_ok
    for spec in specs:
        o = _oracle_final(orc, spec, frames[spec.sid])
        d, p, m, di = (x.cpu().numpy().reshape(spec.height, spec.width) for x in backend.finals[spec.sid])
        np.testing.assert_array_equal(di, o["d_int"], "integer disparity, stream %d" % spec.sid)
        np.testing.assert_array_equal(m, o["mask"], "moving mask, stream %d" % spec.sid)
        for got, want, what in ((d, o["d"], "mean"), (p, o["p"], "variance")):
            rel = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1e-30)
            assert rel.max() <= 1e-5, "Kalman %s of stream %d: rel err %g" % (what, spec.sid, rel.max())
