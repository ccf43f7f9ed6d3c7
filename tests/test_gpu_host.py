"""dp_precode_host: the slot in host memory, uploaded, precoded and downloaded
in overlapping chunks; the results equal dp_precode's bit for bit."""
import numpy as np
import pytest

from gpu_util import TOL_FP32, oracle_of, rel_err_per_sc, to_dev
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu


def run_both(p, prec, chunk, pinned=True, mode=None):
    import torch
    mode = mode or p.mode
    pl = dp.Plan(p.U, p.B, p.C, p.n_sc, p.K, mode=mode, prec=prec, N0=p.N0, tau=p.tau,
                 cluster_sizes=p.cluster_sizes)
    Xd = pl.empty("X")
    pl.precode(to_dev(p.H), to_dev(p.S), Xd)
    st_d = pl.status_get()
    Hh, Sh = torch.from_numpy(p.H), torch.from_numpy(p.S)
    Xh = torch.full((p.n_sc, p.K, p.B), float("nan"), dtype=torch.complex64)
    if pinned:
        Hh, Sh, Xh = Hh.pin_memory(), Sh.pin_memory(), Xh.pin_memory()
    pl.precode_host(Hh, Sh, Xh, chunk)
    st_h = pl.status_get()  # synchronizes the plan's stream
    return Xd.cpu(), st_d, Xh, st_h


@pytest.mark.parametrize("chunk", [0, 100, 1, 1203, 5000])
@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_host_chunks_equal_device_call(chunk, prec):
    import torch
    w = synth.WORKLOADS["c2"]
    n_sc = 1203 if chunk != 1 else 37
    p = synth.make_problem(w["U"], w["B"], w["C"], n_sc, w["K"], w["qam"], 10.0,
                           seed=synth.seed_for(2, 77))
    Xd, st_d, Xh, st_h = run_both(p, prec, chunk)
    assert np.array_equal(st_d, st_h) and (st_h == 0).all()
    assert torch.equal(Xd, Xh)


def test_host_fd_small_clusters_and_pageable_memory():
    import torch
    cs = [2, 30, 5, 64, 1]
    p = synth.make_problem(16, sum(cs), len(cs), 23, 7, 64, 20.0, seed=3101, mode="fdwf",
                           cluster_sizes=cs)
    Xd, st_d, Xh, st_h = run_both(p, "fp32", 5, pinned=False)
    assert np.array_equal(st_d, st_h)
    assert torch.equal(Xd, Xh)
    ref = oracle_of(p)
    assert rel_err_per_sc(Xh.numpy(), ref["X"]).max() <= TOL_FP32


def test_host_status_of_a_failed_subcarrier_in_a_later_chunk():
    p = synth.make_problem(16, 256, 8, 50, 14, 16, 10.0, seed=3102)
    p.H[37, 5, 3] = np.nan
    Xd, st_d, Xh, st_h = run_both(p, "fp16", 8)
    assert st_h[37] == dp.NONFINITE and (np.delete(st_h, 37) == 0).all()
    assert np.all(Xh[37].numpy() == 0)
    assert np.array_equal(st_d, st_h)


def test_host_repeated_calls_reuse_the_staging_ring():
    import torch
    p = synth.make_problem(8, 64, 2, 90, 14, 16, 10.0, seed=3103)
    pl = dp.Plan(p.U, p.B, p.C, p.n_sc, p.K, mode="wf", prec="fp16", N0=p.N0)
    Hh = torch.from_numpy(p.H).pin_memory()
    Sh = torch.from_numpy(p.S).pin_memory()
    outs = []
    for chunk in (10, 10, 30, 7):  # grows the ring once, then reuses it
        Xh = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64).pin_memory()
        pl.precode_host(Hh, Sh, Xh, chunk)
        outs.append(Xh)
    assert (pl.status_get() == 0).all()
    assert all(torch.equal(outs[0], o) for o in outs[1:])
