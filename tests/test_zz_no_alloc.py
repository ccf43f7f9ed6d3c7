"""dp_precode_noalloc, the allocation-free entry point.  It serves callers that
cannot call cudaMalloc: a baseband runtime whose device memory is partitioned
once at start-up, or a real-time slot loop that cannot absorb an allocation's
latency or its implicit synchronization.  Its workspace is the library's
static device array, shared by every call.

Every case checks the precoded vectors against the FP64 oracle and against
dp_precode, the existing entry point, within the FP32 bar, and the entry point
is called several times in a row so that each call starts from what the
previous one left in the shared array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from gpu_util import TOL_FP32, gpu_precode, oracle_of, rel_err_per_sc
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu


def _setup():
    lib = dp.load()
    P = ctypes.c_void_p
    lib.dp_precode_noalloc.argtypes = [ctypes.POINTER(dp.PlanDesc), P, P, P, P, P]
    lib.dp_precode_noalloc.restype = ctypes.c_int
    return lib


def _noalloc(lib, p, H, S, X, stream, with_status=True):
    cs = (ctypes.c_int * p.C)(*p.cluster_sizes)
    d = dp.PlanDesc(p.U, p.B, p.C, ctypes.cast(cs, ctypes.POINTER(ctypes.c_int)), p.n_sc, p.K,
                    dp.MODES[p.mode], dp.PRECISIONS["fp32"], p.rho2, p.N0, p.Es, p.tau, 0)
    st = np.full(max(p.n_sc, 1), -1, np.int32)
    ptr = st.ctypes.data_as(ctypes.c_void_p) if with_status else None
    rc = lib.dp_precode_noalloc(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                ctypes.c_void_p(X.data_ptr()), ptr)
    return rc, st[: p.n_sc]


def _check(p, Xg):
    ref = oracle_of(p)
    assert (ref["status"] == 0).all()
    err = rel_err_per_sc(Xg, ref["X"])
    assert err.max() <= TOL_FP32, f"vs oracle: {err.max():.3e}"
    Xp, st = gpu_precode(p)
    assert (st == 0).all()
    err = rel_err_per_sc(Xg, Xp.astype(np.complex128))
    assert err.max() <= TOL_FP32, f"vs dp_precode: {err.max():.3e}"


CASES = [
    # c2 shape, PD-WF
    dict(U=16, B=256, C=8, n_sc=300, K=14, qam=16, snr_db=10.0, seed=900, mode="wf"),
    # FD-WF with 32-antenna clusters (U x U form)
    dict(U=32, B=128, C=4, n_sc=170, K=7, qam=64, snr_db=5.0, seed=901, mode="fdwf"),
    # ZF with a user count that is not a multiple of 8 (padded users)
    dict(U=12, B=64, C=2, n_sc=97, K=5, qam=16, snr_db=10.0, seed=902, mode="zf"),
    # MRT with an odd user count (rows not bulk-copyable)
    dict(U=7, B=48, C=3, n_sc=65, K=3, qam=4, snr_db=10.0, seed=903, mode="mrt"),
    # FD-WF with clusters smaller than the user count: the B_c x B_c form
    dict(U=24, B=64, C=4, n_sc=129, K=14, qam=64, snr_db=10.0, seed=904, mode="fdwf"),
]


def _problem(c):
    return synth.make_problem(c["U"], c["B"], c["C"], c["n_sc"], c["K"], c["qam"], c["snr_db"],
                              seed=synth.seed_for(2, c["seed"]), mode=c["mode"])


def test_noalloc_matches_oracle_and_dp_precode_on_consecutive_calls():
    import torch
    lib = _setup()
    stream = torch.cuda.current_stream()
    for c in CASES:  # calls in a row, each with another shape and mode
        p = _problem(c)
        H = torch.from_numpy(p.H).cuda()
        S = torch.from_numpy(p.S).cuda()
        X = torch.full((p.n_sc, p.K, p.B), float("nan"), dtype=torch.complex64, device="cuda")
        rc, st = _noalloc(lib, p, H, S, X, stream)
        assert rc == dp.OK, (c, dp.status_string(rc))
        assert (st == 0).all()
        _check(p, X.cpu().numpy())


def test_noalloc_two_calls_enqueued_then_one_synchronize():
    """Two calls on one stream without a status read between them (nothing
    waits on the host): the second call reuses the array the first one wrote,
    and both outputs are right after one stream synchronize."""
    import torch
    lib = _setup()
    stream = torch.cuda.current_stream()
    ps = [_problem(CASES[4]), _problem(CASES[0])]
    outs = []
    for p in ps:
        H = torch.from_numpy(p.H).cuda()
        S = torch.from_numpy(p.S).cuda()
        X = torch.full((p.n_sc, p.K, p.B), float("nan"), dtype=torch.complex64, device="cuda")
        rc, _ = _noalloc(lib, p, H, S, X, stream, with_status=False)
        assert rc == dp.OK, dp.status_string(rc)
        outs.append((H, S, X))
    stream.synchronize()
    for p, (_, _, X) in zip(ps, outs):
        _check(p, X.cpu().numpy())


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    lib = _setup()
    p = synth.make_problem(64, 64, 1, 1, 1, 4, 10.0, seed=3)
    big = synth.Problem(64, 64, [64], 4000, 14, p.H, p.S)  # 4000 * 64^2 * 8 B > 8 MiB
    H = torch.zeros(1, dtype=torch.complex64, device="cuda")
    rc, _ = _noalloc(lib, big, H, H, H, torch.cuda.current_stream())
    assert rc == dp.UNSUPPORTED
