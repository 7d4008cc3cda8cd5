"""Helpers of the GPU parity tests: run frames through the C ABI and compare
every stage with the oracle on the same inputs.

Bars: bit-exact for census codes, windows, offsets, classes, costs,
aggregated costs, integer disparities, the mask, and the single-precision
decision values (prediction, measurement, innovation); the Kalman mean and
variance within 1e-5 relative of the single-precision oracle (same
operations, same order), and the difference from the double-precision oracle
reported and bounded by single-precision rounding of Eqs. 5-6.
"""
from __future__ import annotations

import numpy as np
import torch

KALMAN_RTOL = 1e-5


def oracle_params(orc, P):
    return orc.Params(P.width, P.height, max_disp=P.max_disp, census_w=P.census_w, census_h=P.census_h,
                      path_mask=P.path_mask, radius_mode=P.radius_mode, radius=P.radius, P1=P.P1, P2=P.P2,
                      q=P.q, r_meas=P.r_meas, p_reset=(P.p_reset if P.p_reset > 0 else None),
                      tau_disc=P.tau_disc, gate_gamma=P.gate_gamma)


def read_all(rs, gs):
    """Every intermediate of the handle's last frame as numpy arrays."""
    def rd(which, dt, view):
        return gs.read(which, dt).numpy().view(view)
    out = dict(
        census_l=rd(rs.RSGM_BUF_CENSUS_L, torch.int64, np.uint64),
        census_r=rd(rs.RSGM_BUF_CENSUS_R, torch.int64, np.uint64),
        win=rd(rs.RSGM_BUF_WINDOW, torch.int32, np.uint32),
        off=rd(rs.RSGM_BUF_OFFSET, torch.int32, np.uint32),
        cls=rd(rs.RSGM_BUF_CLASS, torch.uint8, np.uint8),
        d_pred=rd(rs.RSGM_BUF_D_PRED, torch.float32, np.float32),
        p_pred=rd(rs.RSGM_BUF_P_PRED, torch.float32, np.float32),
        cost=rd(rs.RSGM_BUF_COST, torch.uint8, np.uint8),
        S=rd(rs.RSGM_BUF_AGGREGATED, torch.int16, np.uint16),
        d_z=rd(rs.RSGM_BUF_D_MEAS, torch.float32, np.float32),
        nu=rd(rs.RSGM_BUF_INNOVATION, torch.float32, np.float32),
    )
    d, p, m, di = gs.state()
    out.update(d=d.cpu().numpy().ravel(), p=p.cpu().numpy().ravel(), mask=m.cpu().numpy().ravel(),
               d_int=di.cpu().numpy().ravel())
    return out


def compare_stream(g, b, o, H, W, check_prediction=True):
    """Compares stream b of the GPU frame g (read_all) with the oracle frame o."""
    n = H * W
    sl = slice(b * n, (b + 1) * n)
    eq = np.testing.assert_array_equal
    eq(g["census_l"][sl], o["census_l"].ravel(), "census (left)")
    eq(g["census_r"][sl], o["census_r"].ravel(), "census (right)")
    win = g["win"][sl]
    eq((win & 0xFFFF).astype(np.uint16), o["lo"].ravel(), "window start")
    eq((win >> 16).astype(np.uint16), o["wd"].ravel(), "window width")
    cls = g["cls"][sl]
    eq(cls, o["cls"].ravel(), "pixel class")
    known = o["cls"].ravel() != 2
    if check_prediction:
        eq(g["d_pred"][sl][known], o["d_pred"].ravel()[known], "predicted disparity")
        eq(g["p_pred"][sl][known], o["p_pred"].ravel()[known], "predicted variance")
    off = g["off"][sl].astype(np.int64)
    base = int(off[0])
    eq(off - base, o["off"].ravel().astype(np.int64), "cell offsets")
    nc = o["ncells"]
    eq(g["cost"][base: base + nc], o["cost"], "cost volume")
    eq(g["S"][base: base + nc], o["S"], "aggregated cost")
    eq(g["d_int"][sl], o["d_int"].ravel(), "integer disparity")
    eq(g["d_z"][sl], o["d_z"].ravel(), "sub-pixel measurement")
    eq(g["mask"][sl], o["mask"].ravel(), "moving mask")
    eq(g["nu"][sl], o["nu"].ravel(), "innovation")
    # Kalman mean and variance: within 1e-5 relative of the single-precision
    # oracle (the same operations in the same order; in practice bit-equal).
    d, p = g["d"][sl].astype(np.float64), g["p"][sl].astype(np.float64)
    d32, p32 = o["d"].ravel().astype(np.float64), o["p"].ravel().astype(np.float64)
    rel32_d = np.abs(d - d32) / np.maximum(np.abs(d32), 1e-30)
    rel32_p = np.abs(p - p32) / np.maximum(np.abs(p32), 1e-30)
    assert rel32_d.max() <= KALMAN_RTOL, "Kalman mean vs f32 oracle rel err %g" % rel32_d.max()
    assert rel32_p.max() <= KALMAN_RTOL, "Kalman variance vs f32 oracle rel err %g" % rel32_p.max()
    # Against the double-precision oracle the difference is single-precision
    # rounding: bounded relative to the operands of Eq. 5 (d = d_pred +
    # K (d_z - d_pred) cancels when d_z is near 0), and relative to p itself
    # for Eq. 6 (a sum of non-negative terms).
    d64, p64 = o["d64"].ravel(), o["p64"].ravel()
    scale = np.maximum.reduce([np.abs(d64), np.abs(o["d_pred"].ravel()).astype(np.float64),
                               np.abs(o["d_z"].ravel()).astype(np.float64)])
    err_d = np.abs(d - d64) / np.maximum(scale, 1e-30)
    rel64_d = np.abs(d - d64) / np.maximum(np.abs(d64), 1e-30)
    rel64_p = np.abs(p - p64) / np.maximum(np.abs(p64), 1e-30)
    assert err_d.max() <= KALMAN_RTOL, "Kalman mean vs f64 oracle (operand-relative) %g" % err_d.max()
    assert rel64_p.max() <= KALMAN_RTOL, "Kalman variance vs f64 oracle rel err %g" % rel64_p.max()
    return dict(max_rel_d_vs_f64=float(rel64_d.max()), max_operand_rel_d_vs_f64=float(err_d.max()),
                max_rel_p_vs_f64=float(rel64_p.max()), max_rel_d_vs_f32=float(rel32_d.max()),
                bit_equal_f32=bool((g["d"][sl] == o["d"].ravel()).all() and (g["p"][sl] == o["p"].ravel()).all()),
                ncells=nc)


def run_sequence(rs, orc, P, left, right, Rm, tv, K, baseline, nframes, streams_to_check=None, dev="cuda"):
    """Runs nframes (frame 0 full range, then reduced) of B streams through the
    C ABI and the oracle, comparing after every frame.  left/right: [B, F, H, W]
    uint8 tensors; Rm: [B, F, 3, 3]; tv: [B, F, 3]."""
    B, H, W = P.batch, P.height, P.width
    if streams_to_check is None:
        streams_to_check = range(B)
    op = oracle_params(orc, P)
    stats = []
    with rs.Stream(P, torch.cuda.current_stream()) as gs:
        states = {b: None for b in streams_to_check}
        for k in range(nframes):
            L = left[:, k].to(dev).contiguous()
            R = right[:, k].to(dev).contiguous()
            if k == 0:
                gs.full_frame(L, R)
            else:
                gs.reduced_frame(L, R, Rm[:, k].contiguous(), tv[:, k].contiguous(), K, baseline)
            g = read_all(rs, gs)
            for b in streams_to_check:
                lb, rb = left[b, k].cpu().numpy(), right[b, k].cpu().numpy()
                if k == 0:
                    o = orc.frame(op, lb, rb)
                else:
                    o = orc.frame(op, lb, rb, state=states[b],
                                  motion=(Rm[b, k].numpy(), tv[b, k].numpy(), K.numpy(), baseline))
                stats.append(compare_stream(g, b, o, H, W))
                states[b] = (o["d"], o["p"])
    return stats
