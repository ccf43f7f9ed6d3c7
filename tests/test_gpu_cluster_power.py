"""FD-WF with per-cluster power (Sec. III-D: rho_c^2 = rho^2 w_c / sum w,
kappa_c = tau U N0 / rho_c^2) on every kernel family, against the FP64
oracle's weighted FD-WF, element by element (per-subcarrier relative error of
the B x K block): single plans in FP32 and FP16, the B_c x B_c kernel for
clusters with B_c < U, the batch (pipelined, group, split and small-cluster
buckets) and the server (uncached and solve-cached)."""
import numpy as np
import pytest

from gpu_util import TOL_FP32, gpu_precode, oracle_of, plan_of, rel_err_per_sc, to_dev
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu
TOL_LP = 1e-3


def weights(C, seed):
    return list(np.random.default_rng(seed).uniform(0.2, 3.0, C))


def weighted(p, prec, w):
    import torch
    pl = plan_of(p, prec=prec, cluster_power=w)
    X = torch.full(pl.shapes()["X"], float("nan"), dtype=torch.complex64, device="cuda")
    pl.precode(to_dev(p.H), to_dev(p.S), X)
    st = pl.status_get()
    pl.close()
    return X.cpu().numpy(), st


CASES = [
    # (U, B, C, cluster sizes or None, n_sc, K, prec)
    (16, 256, 8, None, 40, 14, "fp32"),           # FP32 fused kernel
    (16, 256, 8, None, 40, 14, "fp16"),           # warp-specialized kernel (U x U form)
    (32, 256, 4, None, 24, 14, "bf16"),           # group kernel, two systems per tile
    (48, 384, 4, None, 12, 14, "fp16"),           # group kernel, quad-row solve
    (24, 64, 4, None, 30, 14, "fp32"),            # B_c x B_c kernel (B_c = 16 < U)
    (16, 64, 3, [8, 24, 32], 30, 7, "fp16"),      # small and U x U clusters together
    (64, 2048, 2, None, 3, 5, "fp32"),            # streaming FP32 form (block > shared)
]


@pytest.mark.parametrize("U,B,C,cs,n_sc,K,prec", CASES)
def test_weighted_fdwf_matches_oracle(U, B, C, cs, n_sc, K, prec):
    p = synth.make_problem(U, B, C, n_sc, K, 64, 10.0, seed=9100 + U + B + C, mode="fdwf",
                           cluster_sizes=cs)
    w = weights(C, U + C)
    ref = oracle_of(p, cluster_power=w)
    Xg, st = weighted(p, prec, w)
    assert (st == 0).all()
    err = rel_err_per_sc(Xg, ref["X"]).max()
    assert err <= (TOL_FP32 if prec == "fp32" else TOL_LP), err
    # the weights take effect: the unweighted output is far from the weighted one
    Xu, _ = gpu_precode(p, prec=prec)
    assert rel_err_per_sc(Xu, ref["X"]).max() > 1e-2


def test_equal_weights_are_bit_identical_to_the_default():
    """w_c equal (any value) gives the default rho^2 / C split bit for bit."""
    p = synth.make_problem(16, 128, 4, 20, 14, 64, 10.0, seed=9200, mode="fdwf")
    for prec in ("fp32", "fp16"):
        X0, _ = gpu_precode(p, prec=prec)
        X1, _ = weighted(p, prec, [2.0] * 4)
        assert np.array_equal(X0, X1), prec


def test_weighted_batch_matches_oracle():
    import torch
    shapes = [(16, 256, 8, None, 30), (64, 512, 4, None, 6), (48, 256, 2, None, 8),
              (24, 96, 6, None, 20), (8, 64, 2, None, 40), (32, 128, 4, [16, 40, 40, 32], 10)]
    probs, descs, ws = [], [], []
    for i, (U, B, C, cs, n_sc) in enumerate(shapes):
        p = synth.make_problem(U, B, C, n_sc, 14, 64, 10.0, seed=9300 + i, mode="fdwf",
                               cluster_sizes=cs)
        w = weights(C, 40 + i)
        probs.append(p)
        ws.append(w)
        descs.append(dict(U=U, B=B, C=C, n_sc=n_sc, K=14, mode="fdwf", prec="fp16", N0=p.N0,
                          tau=p.tau, cluster_sizes=cs, cluster_power=w))
    b = dp.Batch(descs)
    Hs = [to_dev(p.H) for p in probs]
    Ss = [to_dev(p.S) for p in probs]
    Xs = [torch.full((p.n_sc, p.K, p.B), float("nan"), dtype=torch.complex64, device="cuda")
          for p in probs]
    b.precode(Hs, Ss, Xs)
    st = b.status_get()
    b.close()
    for p, w, X, s in zip(probs, ws, Xs, st):
        assert (s == 0).all()
        ref = oracle_of(p, cluster_power=w)
        err = rel_err_per_sc(X.cpu().numpy(), ref["X"]).max()
        assert err <= TOL_LP, (p.U, p.B, err)


@pytest.mark.parametrize("cache", [False, True])
def test_weighted_server_cell_matches_oracle(cache):
    import torch
    p = synth.make_problem(24, 192, 6, 16, 14, 64, 10.0, seed=9400, mode="fdwf",
                           cluster_sizes=[16, 32, 48, 32, 48, 16])
    w = weights(6, 9)
    ref = oracle_of(p, cluster_power=w)
    srv = dp.Server(streams=2, max_inflight=4, arena_bytes=1 << 26, auto_release=False,
                    cache_solve=cache)
    prec = "fp32" if cache else "fp16"
    cid = srv.add_cell(dict(U=p.U, B=p.B, C=p.C, n_sc=p.n_sc, K=p.K, mode="fdwf", prec=prec,
                            N0=p.N0, tau=p.tau, cluster_sizes=p.cluster_sizes,
                            cluster_power=w), to_dev(p.H))
    rid = srv.submit(cid, to_dev(p.S))
    srv.drain()
    X = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
    srv.copy_result(rid, X)
    assert srv.result(rid) == 0
    srv.close()
    err = rel_err_per_sc(X.cpu().numpy(), ref["X"]).max()
    assert err <= (TOL_FP32 if cache else TOL_LP), err
