"""The timeout path of the bounded on-device waits.  A host-requested stall
(dp_debug_stall) makes the warp-specialized tensor-core kernel's MMA issuer
wait on a flag that nothing sets until its time limit runs out; nothing
faults, traps or hangs.  The call must then report DP_ERR_TIMEOUT for every
subcarrier with zeroed outputs, and the next call on the same plan and
stream must succeed, which shows that the kernel's copies and MMAs drained
and its TMEM was freed."""
import numpy as np
import pytest

from gpu_util import oracle_of, plan_of, rel_err_per_sc, to_dev
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("U,B,C,n_sc", [(16, 64, 2, 40), (8, 128, 4, 301)])
def test_stalled_wait_times_out_then_the_next_call_succeeds(U, B, C, n_sc):
    import torch
    p = synth.make_problem(U, B, C, n_sc, 14, 16, 10.0, seed=synth.seed_for(2, 950 + U))
    pl = plan_of(p, prec="fp16")
    H, S = to_dev(p.H), to_dev(p.S)
    X = torch.full(pl.shapes()["X"], float("nan"), dtype=torch.complex64, device="cuda")
    pl.debug_stall(20000)  # 20 ms, far below the waits' own bound
    pl.precode(H, S, X)
    st = pl.status_get()
    assert (st == dp.TIMEOUT).all(), np.unique(st)
    assert (X.cpu().numpy() == 0).all()
    # the same plan, stream and arrays, stall off: a normal call
    pl.debug_stall(0)
    X.fill_(float("nan"))
    pl.precode(H, S, X)
    st = pl.status_get()
    assert (st == dp.OK).all()
    ref = oracle_of(p)
    err = rel_err_per_sc(X.cpu().numpy(), ref["X"])
    assert err.max() <= 1e-3, err.max()
    pl.close()


def test_debug_stall_rejects_out_of_range():
    p = synth.make_problem(8, 64, 2, 4, 2, 4, 10.0, seed=1)
    pl = plan_of(p, prec="fp16")
    for bad in (-1, 1_000_001):
        with pytest.raises(dp.DPError):
            pl.debug_stall(bad)
    pl.close()
