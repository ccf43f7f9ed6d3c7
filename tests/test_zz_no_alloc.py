"""dp_precode_noalloc, the allocation-free entry point for callers that cannot
call cudaMalloc (a runtime with pre-partitioned device memory, a real-time
slot loop that cannot afford an allocation's latency): it must give the same
precoded vectors as dp_precode, call after call, with its workspace in the
library's static device array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from gpu_util import TOL_FP32, gpu_precode, rel_err_per_sc
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, p, H, S, X, stream):
    cs = (ctypes.c_int * p.C)(*p.cluster_sizes)
    d = dp.PlanDesc(p.U, p.B, p.C, ctypes.cast(cs, ctypes.POINTER(ctypes.c_int)), p.n_sc, p.K,
                    dp.MODES[p.mode], dp.PRECISIONS["fp32"], p.rho2, p.N0, p.Es, p.tau, 0)
    st = np.full(max(p.n_sc, 1), -1, np.int32)
    rc = lib.dp_precode_noalloc(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                ctypes.c_void_p(X.data_ptr()), st.ctypes.data_as(ctypes.c_void_p))
    return rc, st[: p.n_sc]


def _setup():
    lib = dp.load()
    P = ctypes.c_void_p
    lib.dp_precode_noalloc.argtypes = [ctypes.POINTER(dp.PlanDesc), P, P, P, P, P]
    lib.dp_precode_noalloc.restype = ctypes.c_int
    return lib


def test_noalloc_matches_dp_precode_on_consecutive_calls():
    import torch
    lib = _setup()
    stream = torch.cuda.current_stream()
    cases = [
        synth.make_problem(16, 256, 8, 300, 14, 16, 10.0, seed=synth.seed_for(2, 900)),
        synth.make_problem(32, 128, 4, 170, 7, 64, 5.0, seed=synth.seed_for(2, 901),
                           mode="fdwf"),
    ]
    for p in cases:  # two calls in a row, the second with another shape and mode
        H = torch.from_numpy(p.H).cuda()
        S = torch.from_numpy(p.S).cuda()
        X = torch.full((p.n_sc, p.K, p.B), float("nan"), dtype=torch.complex64, device="cuda")
        rc, st = _noalloc(lib, p, H, S, X, stream)
        assert rc == dp.OK, dp.status_string(rc)
        assert (st == 0).all()
        ref, ref_st = gpu_precode(p)
        assert (ref_st == 0).all()
        err = rel_err_per_sc(X.cpu().numpy(), ref.astype(np.complex128))
        assert err.max() <= TOL_FP32, err.max()


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    lib = _setup()
    p = synth.make_problem(64, 64, 1, 1, 1, 4, 10.0, seed=3)
    big = synth.Problem(64, 64, [64], 4000, 14, p.H, p.S)  # 4000 * 64^2 * 8 B > 8 MiB
    H = torch.zeros(1, dtype=torch.complex64, device="cuda")
    rc, _ = _noalloc(lib, big, H, H, H, torch.cuda.current_stream())
    assert rc == dp.UNSUPPORTED
