"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs.
Every call goes through the C ABI (via the ctypes binding)."""
import numpy as np
import pytest

from gpu_util import TOL_FP32, gpu_precode, oracle_of, plan_of, rel_err_per_sc, to_dev
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu


def c1(mode="wf", tau=0.125, seed=0):
    w = synth.WORKLOADS["c1"]
    return synth.make_problem(w["U"], w["B"], w["C"], w["n_sc"], w["K"], w["qam"], w["snr_db"],
                              seed=synth.seed_for(1, seed), mode=mode, tau=tau)


def c2(snr_db=10.0, mode="wf", tau=0.125, n_sc=None, seed=0):
    w = synth.WORKLOADS["c2"]
    return synth.make_problem(w["U"], w["B"], w["C"], n_sc or w["n_sc"], w["K"], w["qam"],
                              snr_db, seed=synth.seed_for(2, seed), mode=mode, tau=tau)


def check(p, mode=None, tau=None, tol=TOL_FP32):
    Xg, st = gpu_precode(p, mode, tau)
    ref = oracle_of(p, mode, tau)
    assert np.array_equal(st, ref["status"]), (st, ref["status"])
    err = rel_err_per_sc(Xg, ref["X"])
    assert err.max() <= tol, f"max rel err {err.max():.3e} (median {np.median(err):.3e})"
    return err


# --- workload c1: centralized WF through the decentralized Gram sum --------------

@pytest.mark.parametrize("mode", ["wf", "fdwf"])
def test_c1_fused(mode):
    check(c1(mode))


def test_c1_split_steps_match_oracle():
    """dp_gram_local -> dp_gram_reduce -> dp_solve -> dp_precode_apply, each
    intermediate against the oracle's."""
    import torch
    p = c1("wf")
    ref = oracle_of(p)
    pl = plan_of(p)
    H, S = to_dev(p.H), to_dev(p.S)
    Gloc, G, Z, sc, X = (pl.empty(k) for k in ("Gloc", "G", "Z", "scale", "X"))
    pl.gram_local(H, Gloc)
    pl.gram_reduce(Gloc, G)
    pl.solve(G, S, Z, sc)
    pl.precode_apply(H, Z, sc, X)
    assert (pl.status_get() == 0).all()
    torch.cuda.synchronize()
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(Gloc.cpu().numpy(), ref["Gloc"]) < 1e-6
    assert rel(G.cpu().numpy(), ref["G"]) < 1e-6
    assert rel(Z.cpu().numpy(), ref["Z"]) < 1e-5
    np.testing.assert_allclose(sc.cpu().numpy(), ref["scale"], rtol=1e-5)
    assert rel_err_per_sc(X.cpu().numpy(), ref["X"]).max() < TOL_FP32


def test_split_fd_steps():
    import torch
    p = c1("fdwf")
    ref = oracle_of(p)
    pl = plan_of(p)
    H, S = to_dev(p.H), to_dev(p.S)
    Gloc, Z, sc, X = (pl.empty(k) for k in ("Gloc", "Z", "scale", "X"))
    pl.gram_local(H, Gloc)
    pl.solve(Gloc, S, Z, sc)
    pl.precode_apply(H, Z, sc, X)
    torch.cuda.synchronize()
    np.testing.assert_allclose(sc.cpu().numpy(), ref["scale"], rtol=1e-5)
    assert np.abs(Z.cpu().numpy() - ref["Z"]).max() / np.abs(ref["Z"]).max() < 1e-5
    assert rel_err_per_sc(X.cpu().numpy(), ref["X"]).max() < TOL_FP32


# --- workload c2: ZF, WF and both FD-WF variants over the SNR sweep (full size) ---

@pytest.mark.parametrize("snr", synth.C2_SNRS)
@pytest.mark.parametrize("mode,tau", [("zf", 0.125), ("wf", 0.125), ("fdwf", 0.125),
                                      ("fdwf", 1.0)])
def test_c2_full(snr, mode, tau):
    check(c2(snr, mode, tau), mode, tau)


# --- shapes: ragged tails, odd / non-multiple-of-8 users, uneven clusters ---------

@pytest.mark.parametrize("U,cs,n_sc,K,mode", [
    (5, [3, 7, 22], 3, 4, "wf"),       # odd U: plain-load path, uneven clusters
    (6, [40, 1, 9], 2, 1, "fdwf"),     # B_c < U cluster (push-through form), K = 1
    (12, [100, 200], 5, 3, "wf"),      # U pads to 16
    (1, [4], 7, 2, "wf"),              # one user
    (64, [300], 2, 14, "wf"),          # largest U, streaming form if it does not fit
    (64, [1024], 1, 14, "wf"),         # U = 64, B = 1024: streaming Gram/solve/apply
    (48, [128, 128, 256], 2, 14, "fdwf"),
    (24, [512], 3, 14, "zf"),
    (40, [96, 100], 2, 5, "wf"),
    (8, [4096], 1, 2, "wf"),           # largest B
])
def test_shapes(U, cs, n_sc, K, mode):
    p = synth.make_problem(U, sum(cs), len(cs), n_sc, K, 16, 8.0, seed=1000 + U + n_sc,
                           mode=mode, cluster_sizes=cs)
    check(p)


def test_k_zero_and_empty():
    p = synth.make_problem(8, 64, 2, 3, 0, 4, 10.0, seed=5)
    Xg, st = gpu_precode(p)
    assert Xg.shape == (3, 0, 64) and (st == 0).all()
    p0 = synth.make_problem(8, 64, 2, 0, 4, 4, 10.0, seed=5)
    Xg, st = gpu_precode(p0)
    assert Xg.shape == (0, 4, 64)


def test_split_path_large_streaming():
    """The Gram / apply kernels stream antenna chunks with a ragged tail."""
    import torch
    cs = [130, 170]
    p = synth.make_problem(32, 300, 2, 4, 6, 16, 10.0, seed=77, cluster_sizes=cs)
    ref = oracle_of(p)
    pl = plan_of(p)
    H, S = to_dev(p.H), to_dev(p.S)
    Gloc, G, Z, sc, X = (pl.empty(k) for k in ("Gloc", "G", "Z", "scale", "X"))
    pl.gram_local(H, Gloc)
    pl.gram_reduce(Gloc, G)
    pl.solve(G, S, Z, sc)
    pl.precode_apply(H, Z, sc, X)
    torch.cuda.synchronize()
    assert np.abs(G.cpu().numpy() - ref["G"]).max() / np.abs(ref["G"]).max() < 1e-6
    assert rel_err_per_sc(X.cpu().numpy(), ref["X"]).max() < TOL_FP32


# --- status: numerical failures are reported, never trapped -------------------------

def test_nonfinite_subcarrier_is_flagged_and_zeroed():
    p = c1()
    p.H[5, 3, 2] = np.nan
    p.S[9, 1, 0] = np.inf
    Xg, st = gpu_precode(p)
    assert st[5] == dp.NONFINITE and st[9] == dp.NONFINITE
    assert np.all(Xg[5] == 0) and np.all(Xg[9] == 0)
    ok = np.ones(p.n_sc, bool)
    ok[[5, 9]] = False
    ref = oracle_of(p)
    assert rel_err_per_sc(Xg[ok], ref["X"][ok]).max() < TOL_FP32


def test_rank_deficient_zf_subcarrier_is_flagged():
    """ZF on an all-zero channel: G = 0 is singular."""
    p = c1()
    p.H[2] = 0
    Xg, st = gpu_precode(p, "zf")
    assert st[2] == dp.NOT_PD and np.all(Xg[2] == 0)
    assert (np.delete(st, 2) == 0).all()


def test_deterministic_bitwise():
    p = c2(n_sc=64)
    a, _ = gpu_precode(p)
    b, _ = gpu_precode(p)
    assert np.array_equal(a, b)


def test_result_independent_of_batch():
    """A subcarrier's output does not depend on which other subcarriers share
    the call."""
    p = c2(n_sc=40)
    full, _ = gpu_precode(p)
    sub = synth.Problem(p.U, p.B, p.cluster_sizes, 7, p.K, p.H[10:17].copy(), p.S[10:17].copy(),
                        p.rho2, p.N0, p.Es, p.tau, p.mode)
    part, _ = gpu_precode(sub)
    assert np.array_equal(full[10:17], part)


def test_power_normalization_on_gpu():
    """||P||_F^2 Es = rho^2 (Eq. (3)) for the GPU precoder, probed with s = e_k."""
    import torch
    p = c2(n_sc=16)
    U = p.U
    S = np.broadcast_to(np.eye(U, dtype=np.complex64), (p.n_sc, U, U)).copy()
    q = synth.Problem(p.U, p.B, p.cluster_sizes, p.n_sc, U, p.H, S, p.rho2, p.N0, p.Es)
    for mode in ("wf", "zf", "fdwf"):
        Xg, _ = gpu_precode(q, mode)
        pw = np.sum(np.abs(Xg.astype(np.complex128)) ** 2, axis=(1, 2))
        np.testing.assert_allclose(pw, p.rho2, rtol=2e-5)
    _ = torch


# --- FD-WF clusters with B_c < U: the paper's B_c x B_c form -----------------------

@pytest.mark.parametrize("U,cs,n_sc,K,snr", [
    (64, [8] * 32, 20, 14, 10.0),           # all clusters small (B_c = 8 < U = 64)
    (48, [32] * 8, 9, 14, 0.0),             # B_c = 32 < U = 48, low SNR
    (16, [2, 30, 5, 64, 1], 11, 7, 20.0),   # mixed: small and U x U clusters
    (64, [16, 16, 32, 64, 128], 4, 3, 10.0),
    (33, [32, 32, 1], 6, 14, 5.0),          # B_c = 32 at the kernel's limit, U odd
])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_fd_small_clusters(U, cs, n_sc, K, snr, prec):
    p = synth.make_problem(U, sum(cs), len(cs), n_sc, K, 64, snr, seed=3000 + U + len(cs),
                           mode="fdwf", cluster_sizes=cs)
    Xg, st = gpu_precode(p, prec=prec)
    ref = oracle_of(p)  # the oracle takes the B_c x B_c form for B_c < U
    assert np.array_equal(st, ref["status"])
    err = rel_err_per_sc(Xg, ref["X"])
    tol = TOL_FP32 if prec == "fp32" else 1e-3
    assert err.max() <= tol, err.max()


# --- MRT: the fully distributed baseline (no inverse; t = tr(G)) ------------------

@pytest.mark.parametrize("U,cs,n_sc,K,prec", [
    (16, [32] * 8, 300, 14, "fp32"),     # FP32 fused kernel
    (16, [32] * 8, 300, 14, "fp16"),     # warp-specialized tensor-core kernel
    (24, [100, 200], 5, 7, "bf16"),      # tensor-core group kernel, warp solve
    (48, [128, 128, 256], 3, 14, "fp32"),  # FP32 fused kernel, CTA solve
    (48, [128, 128, 256], 3, 14, "fp16"),  # tensor-core group kernel, U > 32
    (64, [1024], 1, 14, "fp32"),         # streaming form
])
def test_mrt(U, cs, n_sc, K, prec):
    p = synth.make_problem(U, sum(cs), len(cs), n_sc, K, 16, 10.0, seed=6000 + U + n_sc,
                           cluster_sizes=cs)
    Xg, st = gpu_precode(p, "mrt", prec=prec)
    ref = oracle_of(p, "mrt")
    assert np.array_equal(st, ref["status"]) and (st == 0).all()
    err = rel_err_per_sc(Xg, ref["X"])
    assert err.max() <= (TOL_FP32 if prec == "fp32" else 1e-3), err.max()


def test_mrt_split_steps():
    """dp_solve returns Z = S and the MRT scale; the apply gives X."""
    import torch
    p = c1()
    ref = oracle_of(p, "mrt")
    pl = plan_of(p, "mrt")
    H, S = to_dev(p.H), to_dev(p.S)
    G, Z, sc, X = (pl.empty(k) for k in ("G", "Z", "scale", "X"))
    Gloc = pl.empty("Gloc")
    pl.gram_local(H, Gloc)
    pl.gram_reduce(Gloc, G)
    pl.solve(G, S, Z, sc)
    pl.precode_apply(H, Z, sc, X)
    torch.cuda.synchronize()
    assert torch.equal(Z, S)
    np.testing.assert_allclose(sc.cpu().numpy(), ref["scale"], rtol=1e-5)
    assert rel_err_per_sc(X.cpu().numpy(), ref["X"]).max() < TOL_FP32
