"""The request loop on the GPU: streams of different resolutions arrive as
Poisson processes and overlap on the device; every stream's final state is
bit-identical to the same frames run alone on a fresh handle."""
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
