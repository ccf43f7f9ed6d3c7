"""Continuous-batching server: results identical alone and in a concurrent
mix, admission bounded by the arena, channel switches, latency accounting,
and the per-channel solve cache (outputs against the oracle across channel
switches, overlapping requests of one cell, a bad request flagged alone)."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_FP32, rel_err_per_sc
from paper_1804_10987_gb300 import dp, synth

pytestmark = pytest.mark.gpu
TOL_LP = 1e-3


def make_cells(n, seed, prec_cycle=("fp16", "bf16", "fp32")):
    import torch
    g = synth.rng(seed)
    cells = []
    for i in range(n):
        U = int(g.choice((8, 16, 24, 32, 48)))
        B = int(g.choice((64, 128, 256)))
        C = int(g.choice([c for c in (1, 2, 4, 8) if B % c == 0]))
        n_sc = int(g.integers(8, 80))
        mode = "wf" if i % 2 == 0 else "fdwf"
        p = synth.make_problem(U, B, C, n_sc, 14, 64, 10.0, seed=seed * 100 + i, mode=mode)
        prec = prec_cycle[i % len(prec_cycle)]
        desc = dict(U=U, B=B, C=C, n_sc=n_sc, K=14, mode=mode, prec=prec, N0=p.N0, tau=0.125)
        cells.append((p, desc, torch.from_numpy(p.H).cuda()))
    return cells


def symbols(p, seed):
    import torch
    return torch.from_numpy(synth.qam_symbols(64, (p.n_sc, p.K, p.U), synth.rng(seed))).cuda()


def test_alone_equals_mix_and_matches_oracle():
    import torch
    cells = make_cells(6, 51)
    srv = dp.Server(streams=4, max_inflight=16, arena_bytes=256 << 20)
    ids = [srv.add_cell(desc, H) for _, desc, H in cells]
    g = np.random.default_rng(5)
    reqs = [(int(g.integers(0, len(cells))), 1000 + i) for i in range(40)]
    S = [symbols(cells[c][0], s) for c, s in reqs]
    # alone: one request at a time
    alone = []
    for (c, _), s in zip(reqs, S):
        rid = srv.submit(ids[c], s)
        srv.drain()
        p = cells[c][0]
        x = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
        srv.copy_result(rid, x)
        assert srv.result(rid) == 0
        srv.release(rid)
        alone.append(x)
    # in the mix: everything submitted at once, overlapping on the GPU
    srv.reset_stats()
    rids = [srv.submit(ids[c], s) for (c, _), s in zip(reqs, S)]
    srv.drain()
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["inflight_peak"] > 1
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for i, rid in enumerate(rids):
        c = reqs[i][0]
        p = cells[c][0]
        x = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
        srv.copy_result(rid, x)
        srv.release(rid)
        assert torch.equal(x, alone[i]), i
    # a few against the oracle
    for i in range(0, len(reqs), 7):
        c = reqs[i][0]
        p, desc, _ = cells[c]
        ref = oracle.precode(p.H, S[i].cpu().numpy(), p.cluster_sizes, desc["mode"], N0=p.N0,
                             tau=0.125, nthreads=8)
        tol = TOL_FP32 if desc["prec"] == "fp32" else TOL_LP
        assert rel_err_per_sc(alone[i].cpu().numpy(), ref["X"]).max() <= tol
    srv.close()


def test_admission_by_memory_and_poisson_replay():
    import torch
    cells = make_cells(4, 52, prec_cycle=("fp16",))
    biggest = max(p.n_sc * p.K * p.B * 8 for p, _, _ in cells)
    # room for about two requests at a time
    srv = dp.Server(streams=4, max_inflight=64, arena_bytes=2 * biggest + (1 << 16),
                    auto_release=True)
    ids = [srv.add_cell(desc, H) for _, desc, H in cells]
    g = np.random.default_rng(6)
    n = 200
    cell_of = g.integers(0, len(cells), n)
    S = [symbols(cells[c][0], 3000 + i) for i, c in enumerate(cell_of)]
    t = np.cumsum(g.exponential(1 / 20000.0, n))
    srv.replay([ids[c] for c in cell_of], S, t)
    st = srv.stats()
    assert st["completed"] == n and st["failed"] == 0
    assert st["arena_high_water"] <= 2 * biggest + (1 << 16)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_channel_switch_applies_to_later_requests():
    import torch
    cells = make_cells(1, 53, prec_cycle=("fp32",))
    p, desc, H = cells[0]
    H2np = synth.rayleigh(p.n_sc, p.B, p.U, synth.rng(99))
    H2 = torch.from_numpy(H2np).cuda()
    srv = dp.Server(streams=1, max_inflight=4, arena_bytes=64 << 20)
    cid = srv.add_cell(desc, H)
    s = symbols(p, 7)
    r1 = srv.submit(cid, s)
    srv.set_channel(cid, H2)
    r2 = srv.submit(cid, s)
    srv.drain()
    x1 = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    srv.copy_result(r1, x1)
    srv.copy_result(r2, x2)
    ref1 = oracle.precode(p.H, s.cpu().numpy(), p.cluster_sizes, desc["mode"], N0=p.N0, tau=0.125)
    ref2 = oracle.precode(H2np, s.cpu().numpy(), p.cluster_sizes, desc["mode"], N0=p.N0, tau=0.125)
    assert rel_err_per_sc(x1.cpu().numpy(), ref1["X"]).max() <= TOL_FP32
    assert rel_err_per_sc(x2.cpu().numpy(), ref2["X"]).max() <= TOL_FP32
    srv.close()


def test_server_rejects_bad_cells():
    import torch
    srv = dp.Server(streams=1, max_inflight=1, arena_bytes=1 << 16)
    H = torch.zeros(4, 64, 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(dp.DPError):  # one request would not fit the arena
        srv.add_cell(dict(U=8, B=64, C=2, n_sc=4000, K=14), H)
    with pytest.raises(dp.DPError):
        srv.add_cell(dict(U=8, B=64, C=3, n_sc=4, K=14), H)
    srv.close()


def test_cached_solve_across_channel_switches():
    """cache_solve: the Gram, inverse and scale are computed once per channel
    (FP32) and reused; requests before and after each switch match the oracle
    on the channel they were submitted on."""
    import torch
    cells = make_cells(6, 61)
    p_mrt = synth.make_problem(16, 128, 4, 24, 14, 64, 10.0, seed=6161, mode="wf")
    cells.append((p_mrt, dict(U=16, B=128, C=4, n_sc=24, K=14, mode="mrt", prec="fp16",
                              N0=p_mrt.N0, tau=0.125), torch.from_numpy(p_mrt.H).cuda()))
    cs = [3, 40, 5, 80]  # FD-WF with B_c < U clusters (those stay per request)
    p_fd = synth.make_problem(16, sum(cs), len(cs), 20, 14, 64, 10.0, seed=6162, mode="fdwf",
                              cluster_sizes=cs)
    cells.append((p_fd, dict(U=16, B=sum(cs), C=len(cs), n_sc=20, K=14, mode="fdwf", prec="bf16",
                             N0=p_fd.N0, tau=0.125, cluster_sizes=cs),
                  torch.from_numpy(p_fd.H).cuda()))
    srv = dp.Server(streams=3, max_inflight=8, arena_bytes=256 << 20, cache_solve=True)
    ids = [srv.add_cell(desc, H) for _, desc, H in cells]
    H2 = [synth.rayleigh(p.n_sc, p.B, p.U, synth.rng(700 + i)) for i, (p, _, _) in enumerate(cells)]
    H2d = [torch.from_numpy(h).cuda() for h in H2]
    plan = []  # (cell, channel index) in submission order
    for c in range(len(cells)):
        plan += [(c, 0)] * 3 + [(c, 1)] * 2 + [(c, 0)]
    order = np.random.default_rng(7).permutation(len(cells))  # interleave the cells
    seq = [x for k in range(6) for c in order for x in [plan[c * 6 + k]]]
    S, rids = [], []
    for c, ch in seq:
        p, _, H = cells[c]
        srv.set_channel(ids[c], H if ch == 0 else H2d[c])
        s = symbols(p, 5000 + len(S))
        S.append(s)
        rids.append(srv.submit(ids[c], s))
    srv.drain()
    for (c, ch), s, rid in zip(seq, S, rids):
        p, desc, _ = cells[c]
        x = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
        srv.copy_result(rid, x)
        assert srv.result(rid) == 0
        srv.release(rid)
        ref = oracle.precode(p.H if ch == 0 else H2[c], s.cpu().numpy(), p.cluster_sizes,
                             desc["mode"], N0=p.N0, tau=0.125, nthreads=8)
        err = rel_err_per_sc(x.cpu().numpy(), ref["X"]).max()
        assert err <= TOL_FP32, (c, ch, desc["mode"], desc["prec"], err)
    srv.close()


def test_cached_solve_flags_a_bad_request_only():
    import torch
    cells = make_cells(1, 62, prec_cycle=("fp16",))
    p, desc, H = cells[0]
    srv = dp.Server(streams=1, max_inflight=4, arena_bytes=64 << 20, cache_solve=True)
    cid = srv.add_cell(desc, H)
    good = symbols(p, 1)
    bad = good.clone()
    bad[3, 2, 1] = float("nan")
    rids = [srv.submit(cid, s) for s in (good, bad, good)]
    srv.drain()
    outs = []
    for rid in rids:
        x = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
        srv.copy_result(rid, x)
        outs.append((srv.result(rid), x))
    assert outs[0][0] == 0 and outs[2][0] == 0 and outs[1][0] == dp.NONFINITE
    assert torch.equal(outs[0][1], outs[2][1])
    assert torch.all(outs[1][1][3] == 0)
    assert torch.equal(outs[1][1][:3], outs[0][1][:3])
    srv.close()


def test_one_cell_overlaps_and_recomputes_in_order():
    """Requests of one cell overlap on the GPU; each channel switch recomputes
    the cell's cached solve only after the requests still reading the old one,
    so every output matches the oracle on its own channel."""
    import torch
    p = synth.make_problem(32, 256, 4, 96, 14, 64, 10.0, seed=6301, mode="wf")
    desc = dict(U=32, B=256, C=4, n_sc=96, K=14, mode="wf", prec="fp32", N0=p.N0, tau=0.125)
    Hs = [p.H] + [synth.rayleigh(p.n_sc, p.B, p.U, synth.rng(6310 + i)) for i in range(2)]
    Hd = [torch.from_numpy(h).cuda() for h in Hs]
    srv = dp.Server(streams=4, max_inflight=16, arena_bytes=256 << 20, cache_solve=True)
    cid = srv.add_cell(desc, Hd[0])
    seq = [0, 0, 0, 1, 1, 2, 2, 2, 0, 1, 1, 0]
    S, rids = [], []
    for i, ch in enumerate(seq):
        srv.set_channel(cid, Hd[ch])
        S.append(symbols(p, 6400 + i))
        rids.append(srv.submit(cid, S[-1]))
    srv.drain()
    for ch, s, rid in zip(seq, S, rids):
        x = torch.empty((p.n_sc, p.K, p.B), dtype=torch.complex64, device="cuda")
        srv.copy_result(rid, x)
        assert srv.result(rid) == 0
        srv.release(rid)
        ref = oracle.precode(Hs[ch], s.cpu().numpy(), p.cluster_sizes, "wf", N0=p.N0, tau=0.125,
                             nthreads=8)
        assert rel_err_per_sc(x.cpu().numpy(), ref["X"]).max() <= TOL_FP32, ch
    srv.close()
