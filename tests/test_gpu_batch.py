"""Batched uneven precoding (persistent launches over work-item queues, CUDA
graph replay, autotuner) against the FP64 oracle and against the single-plan
path: bit-identical where both run the same device code (FP32, and reduced
precision up to 16 users), within 1e-5 where the batch runs the split form
(reduced precision above 16 users)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_FP32, rel_err_per_sc
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu
TOL_LP = 1e-3


def make_instances(n, seed, nsc_range=(3, 40), big=False):
    """Seeded uneven instances drawn from the batched workload's sets."""
    g = synth.rng(seed)
    out = []
    for i in range(n):
        U = int(g.choice(synth.C4_U))
        B = int(g.choice(synth.C4_B if big else (64, 128, 256, 512)))
        C = int(g.choice([c for c in synth.C4_C if B % c == 0]))
        mode = ("wf", "fdwf", "zf")[int(g.integers(0, 3))]
        prec = ("bf16", "fp16", "fp32")[int(g.integers(0, 3))]
        # ZF has no regularizer and needs B > U; cond(G) grows as B/U shrinks,
        # which the automatic refinement of the 16-bit Gram takes care of
        if mode == "zf" and B < 2 * U:
            mode = "wf"
        chan = "iid" if g.integers(0, 2) == 0 else "kron"
        n_sc = int(g.integers(nsc_range[0], nsc_range[1] + 1))
        K = int(g.choice([1, 7, 14]))
        p = synth.make_problem(U, B, C, n_sc, K, 64, 10.0, seed=seed * 1000 + i, mode=mode,
                               channel=chan)
        out.append((p, prec))
    return out


def desc_of(p, prec):
    return dict(U=p.U, B=p.B, C=p.C, n_sc=p.n_sc, K=p.K, mode=p.mode, prec=prec, rho2=p.rho2,
                N0=p.N0, Es=p.Es, tau=p.tau, cluster_sizes=p.cluster_sizes)


def run_batch(insts, tune=False):
    import torch
    b = dp.Batch([desc_of(p, prec) for p, prec in insts])
    Hs = [torch.from_numpy(p.H).cuda() for p, _ in insts]
    Ss = [torch.from_numpy(p.S).cuda() for p, _ in insts]
    Xs = [torch.full((p.n_sc, p.K, p.B), float("nan"), dtype=torch.complex64, device="cuda")
          for p, _ in insts]
    if tune:
        b.tune(Hs, Ss, Xs, trials=2)
    b.precode(Hs, Ss, Xs)
    st = b.status_get()
    return b, Hs, Ss, Xs, st


def test_batch_matches_oracle_and_single_plans():
    import torch
    insts = make_instances(14, 41)
    b, Hs, Ss, Xs, st = run_batch(insts)
    info = b.describe()
    assert info["buckets"], info
    for i, (p, prec) in enumerate(insts):
        assert (st[i] == 0).all(), (i, st[i])
        ref = oracle.precode(p.H, p.S, p.cluster_sizes, p.mode, N0=p.N0, tau=p.tau, nthreads=8)
        Xg = Xs[i].cpu().numpy()
        tol = TOL_FP32 if prec == "fp32" else TOL_LP
        err = rel_err_per_sc(Xg, ref["X"])
        assert err.max() <= tol, (i, p.U, p.B, p.C, p.mode, prec, err.max())
        # the single-plan path runs the same device code -- except for more
        # than 16 users in reduced precision, where the batch runs the split
        # form (Gram, blocked solve with one row per thread, apply): the same
        # elimination with its sums in another order
        pl = dp.Plan(p.U, p.B, p.C, p.n_sc, p.K, mode=p.mode,
                     prec=prec, N0=p.N0, tau=p.tau,
                     cluster_sizes=p.cluster_sizes)
        X1 = torch.empty_like(Xs[i])
        pl.precode(Hs[i], Ss[i], X1)
        torch.cuda.synchronize()
        if prec != "fp32" and p.U > 16:
            d = rel_err_per_sc(X1.cpu().numpy(), Xs[i].cpu().numpy().astype(np.complex128))
            assert d.max() <= 1e-5, (i, d.max())
        else:
            assert torch.equal(X1, Xs[i]), i
    b.close()


def test_graph_replay_and_tuner_keep_results():
    import torch
    insts = make_instances(9, 42)
    b, Hs, Ss, Xs, _ = run_batch(insts)
    first = [x.clone() for x in Xs]
    for x in Xs:
        x.fill_(float("nan"))
    b.precode(Hs, Ss, Xs)  # graph replay
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(first, Xs))
    b.tune(Hs, Ss, Xs, trials=1)
    info = b.describe()
    assert all(bk["ctas_per_sm"] >= 1 and bk["tuned_ms"] >= 0 for bk in info["buckets"])
    for x in Xs:
        x.fill_(float("nan"))
    b.precode(Hs, Ss, Xs)
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(first, Xs))
    # new arrays (same shapes): the graph reads the new pointers
    Xs2 = [torch.empty_like(x) for x in Xs]
    b.precode(Hs, Ss, Xs2)
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(first, Xs2))
    b.close()


def test_batch_status_isolated():
    insts = make_instances(5, 43)
    insts[2][0].H[1, 0, 0] = np.nan
    b, Hs, Ss, Xs, st = run_batch(insts)
    assert st[2][1] == dp.NONFINITE
    for i in range(5):
        ok = st[i] == 0
        if i == 2:
            assert ok.sum() == insts[2][0].n_sc - 1
        else:
            assert ok.all()
    assert np.all(Xs[2][1].cpu().numpy() == 0)
    b.close()


def test_full_size_batched_workload_sampled():
    """512 instances with the batched workload's size distributions (U, B, C,
    n_sc in [72, 3300], K = 14, 64-QAM, mixed i.i.d. / Kronecker channels, WF
    and FD-WF, FP16 Gram on the tensor cores), drawn on the GPU; two
    subcarriers per instance are recomputed by the oracle.  (A BF16 Gram
    reaches ~1.5e-3 on the worst-conditioned correlated instances of this mix,
    above the 1e-3 bar: FP16 carries 3 more mantissa bits at the same cost.)"""
    import torch
    shapes = synth.c4_instance_shapes(512, synth.seed_for(4))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.seed_for(4, 1))
    descs, Hs, Ss, Xs = [], [], [], []
    N0 = synth.n0_from_snr(10.0)
    for sh in shapes:
        Hs.append(synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda"))
        Ss.append(synth.torch_symbols(64, (sh["n_sc"], 14, sh["U"]), gen, "cuda"))
        Xs.append(torch.empty((sh["n_sc"], 14, sh["B"]), dtype=torch.complex64, device="cuda"))
        descs.append(dict(U=sh["U"], B=sh["B"], C=sh["C"], n_sc=sh["n_sc"], K=14,
                          mode=sh["mode"], prec="fp16", N0=N0, tau=0.125))
    b = dp.Batch(descs)
    b.precode(Hs, Ss, Xs)
    st = b.status_get()
    assert all((s == 0).all() for s in st)
    g = np.random.default_rng(4)
    worst = 0.0
    for i, sh in enumerate(shapes):
        idx = np.sort(g.choice(sh["n_sc"], 2, replace=False))
        H = Hs[i][idx].cpu().numpy()
        S = Ss[i][idx].cpu().numpy()
        ref = oracle.precode(H, S, [sh["B"] // sh["C"]] * sh["C"], sh["mode"], N0=N0,
                             tau=0.125, nthreads=8)
        err = rel_err_per_sc(Xs[i][idx].cpu().numpy(), ref["X"])
        worst = max(worst, float(err.max()))
    assert worst <= TOL_LP, worst
    b.close()
