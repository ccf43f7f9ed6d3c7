"""End-to-end link check (downlink, perfect CSI; Sec. II and the simulations
of Sec. III-E): the GPU precoder's X goes through y = H x + n, each user
applies one common receive gain (the least-squares one, the same for every
precoder) and slices to the constellation.  Two checks:

* the link-level MSE and symbol error rate of the GPU outputs equal those of
  the FP64 oracle's outputs on the same channel, symbols and noise;
* the paper's qualitative ordering: WF (= PD-WF) has the lowest MSE, ZF is
  close to it at high SNR when B >> U, FD-WF with clusters of B_c = 32 >= U
  stays close to it, MRT falls further behind as the SNR grows, and every
  precoder's MSE falls with the SNR.
"""
import numpy as np
import pytest

from gpu_util import gpu_precode, oracle_of
from paper_1804_10987_gb300 import synth

pytestmark = pytest.mark.gpu

U, B, C, N_SC, K, QAM = 16, 256, 8, 160, 14, 16
SNRS = (0.0, 10.0, 20.0)


def link(p, X, seed):
    """MSE and symbol error rate of s_hat = g (H x + n) with the least-squares
    common gain g; H[n][b][u] is user u's channel to antenna b."""
    g = np.random.default_rng(seed)
    y = np.einsum("nbu,nkb->nku", p.H.astype(np.complex128), X.astype(np.complex128))
    noise = (g.standard_normal(y.shape) + 1j * g.standard_normal(y.shape)) * np.sqrt(p.N0 / 2)
    y = y + noise
    s = p.S.astype(np.complex128)
    gain = np.vdot(y, s) / np.vdot(y, y)
    s_hat = gain * y
    mse = float(np.mean(np.abs(s_hat - s) ** 2))
    pts = synth.qam_constellation(QAM).astype(np.complex128)
    dec = pts[np.argmin(np.abs(s_hat[..., None] - pts) ** 2, axis=-1)]
    ser = float(np.mean(np.abs(dec - s) > 1e-6))
    return mse, ser


def problem(snr, mode="wf", tau=0.125):
    return synth.make_problem(U, B, C, N_SC, K, QAM, snr, seed=synth.seed_for(2, 900 + int(snr)),
                              mode=mode, tau=tau)


@pytest.mark.parametrize("snr", SNRS)
@pytest.mark.parametrize("mode,tau,prec", [("wf", 0.125, "fp32"), ("wf", 0.125, "fp16"),
                                           ("zf", 0.125, "fp32"), ("fdwf", 0.125, "fp16"),
                                           ("fdwf", 1.0, "fp32"), ("mrt", 0.125, "fp16")])
def test_link_metrics_match_oracle(snr, mode, tau, prec):
    p = problem(snr, mode, tau)
    Xg, st = gpu_precode(p, mode, tau, prec=prec)
    assert (st == 0).all()
    ref = oracle_of(p, mode, tau)
    mse_g, ser_g = link(p, Xg, 7)
    mse_o, ser_o = link(p, ref["X"], 7)
    assert abs(mse_g - mse_o) <= 1e-3 * mse_o, (mse_g, mse_o)
    assert abs(ser_g - ser_o) <= 3.0 / (N_SC * K * U), (ser_g, ser_o)  # at most a few symbols


def test_link_ordering_of_the_precoders():
    res = {}
    for snr in SNRS:
        for mode, tau in (("wf", 0.125), ("zf", 0.125), ("fdwf", 0.125), ("fdwf", 1.0),
                          ("mrt", 0.125)):
            p = problem(snr, mode, tau)
            Xg, _ = gpu_precode(p, mode, tau)
            res[(mode, tau, snr)] = link(p, Xg, 11)[0]
    print({f"{k[0]}{k[1]}@{k[2]}": round(v, 5) for k, v in res.items()})
    for snr in SNRS:
        wf = res[("wf", 0.125, snr)]
        # WF minimizes the MSE; sampling noise allows a 2 % margin
        for other in (("zf", 0.125), ("fdwf", 0.125), ("fdwf", 1.0), ("mrt", 0.125)):
            assert wf <= res[other + (snr,)] * 1.02, (snr, other, wf, res[other + (snr,)])
        # FD-WF with B_c = 32 >= U = 16 stays close to WF
        assert res[("fdwf", 0.125, snr)] <= 1.5 * wf, (snr, res[("fdwf", 0.125, snr)], wf)
    # with B/U = 16 ZF is within a few percent of WF at high SNR, and every
    # precoder's MSE falls with the SNR
    assert res[("zf", 0.125, 20.0)] <= 1.05 * res[("wf", 0.125, 20.0)]
    # MRT is interference-limited (Sec. I): its gap to WF grows with the SNR
    # (about 1.27x at 20 dB with B/U = 16)
    mrt_gap = [res[("mrt", 0.125, s)] / res[("wf", 0.125, s)] for s in SNRS]
    assert mrt_gap[0] <= mrt_gap[1] <= mrt_gap[2] and mrt_gap[2] >= 1.1, mrt_gap
    for key in (("wf", 0.125), ("zf", 0.125), ("fdwf", 0.125), ("fdwf", 1.0)):
        seq = [res[key + (s,)] for s in SNRS]
        assert seq[0] > seq[1] > seq[2], (key, seq)
