"""Cluster-sharded PD-WF (Sec. IV-A/IV-B: each rank holds a group of clusters;
local Grams reduced to a root, z and the precoding factor broadcast back): the
host logic on CPU with two and three gloo ranks, the three compute steps
supplied by the FP64 oracle's routines.  The assembled output must equal the
oracle's centralized WF of the full channel (Thm. 1) -- PD-WF is exact
(Sec. III-B) -- up to the FP32 precoding factor the sharded precoder carries."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """Steps 1, 3 and 5 from the oracle's FP64 routines (test infrastructure)."""

    def __init__(self, U, N0, rho2=1.0, Es=1.0):
        self.U, self.kappa, self.rho2, self.Es = U, U * N0 / rho2, rho2, Es

    def gram(self, H_r):
        import torch

        import oracle
        G = np.stack([oracle.gram(h) for h in H_r.numpy()])
        return torch.from_numpy(G)

    def solve(self, G, S):
        import torch

        import oracle
        Gn, Sn = G.numpy(), S.numpy()
        Z = np.zeros_like(Sn)
        scale = np.zeros(Gn.shape[0], np.float32)
        for n in range(Gn.shape[0]):
            A = Gn[n] + self.kappa * np.eye(self.U)
            st, L = oracle.cholesky(A)
            assert st == 0
            T = oracle.inverse_from_cholesky(L)
            t = oracle.t_direct(T, Gn[n])
            scale[n] = np.sqrt(self.rho2 / (self.Es * t))
            Z[n] = (T @ Sn[n].T).T
        return torch.from_numpy(Z), torch.from_numpy(scale)

    def apply(self, H_r, Z, scale):
        import torch
        Hn, Zn, sc = H_r.numpy(), Z.numpy(), scale.numpy().astype(np.float64)
        X = np.einsum("nbu,nku->nkb", np.conj(Hn), Zn) * sc[:, None, None]
        return torch.from_numpy(X)


def _rank(rank, world, port, cs, U, n_sc, K, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1804_10987_gb300 import sharded, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.make_problem(U, sum(cs), len(cs), n_sc, K, 16, 10.0, seed=8100,
                               cluster_sizes=cs)
        c0, nc, a0, ants = sharded.split_clusters(cs, world)[rank]
        H_r = torch.from_numpy(p.H[:, a0:a0 + ants].astype(np.complex128).copy())
        S = torch.from_numpy(p.S.astype(np.complex128))
        drv = sharded.ShardedPDWF(U, ants, n_sc, K, p.N0, ops=OracleOps(U, p.N0))
        X_r = drv.precode(H_r, S)
        q.put((rank, a0, X_r.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,cs", [(2, [32, 32, 16, 48]), (3, [8, 24, 24, 8, 40])])
def test_sharded_pdwf_equals_centralized_wf(world, cs):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1804_10987_gb300 import synth
    U, n_sc, K = 8, 5, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cs, U, n_sc, K, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    try:
        res = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for pr in procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.kill()
    assert [pr.exitcode for pr in procs] == [0] * world
    X = np.concatenate([x for _, _, x in res], axis=2)
    p = synth.make_problem(U, sum(cs), len(cs), n_sc, K, 16, 10.0, seed=8100, cluster_sizes=cs)
    ref = oracle.precode(p.H, p.S, cs, "wf", N0=p.N0)["X"]
    rel = np.linalg.norm((X - ref).reshape(n_sc, -1), axis=1) / np.linalg.norm(
        ref.reshape(n_sc, -1), axis=1)
    assert rel.max() < 1e-6, rel.max()


def test_split_clusters_covers_every_cluster_once():
    sys.path.insert(0, ROOT)
    from paper_1804_10987_gb300 import sharded
    for cs in ([32] * 8, [8, 24, 24, 8, 40], [1, 1, 100, 1], [64, 64]):
        for world in range(1, len(cs) + 1):
            parts = sharded.split_clusters(cs, world)
            assert len(parts) == world
            assert all(n >= 1 for _, n, _, _ in parts)
            assert parts[0][0] == 0 and parts[0][2] == 0
            for (c0, n, a0, ants), (c1, _, a1, _) in zip(parts, parts[1:]):
                assert c1 == c0 + n and a1 == a0 + ants
            c0, n, a0, ants = parts[-1]
            assert c0 + n == len(cs) and a0 + ants == sum(cs)
            assert [sum(cs[c0:c0 + n]) for c0, n, _, _ in parts] == [a for *_, a in parts]
    with pytest.raises(ValueError):
        sharded.split_clusters([4, 4], 3)
    # eight equal clusters over eight ranks: one cluster each (the paper's C = 8 GPUs)
    assert [n for _, n, _, _ in sharded.split_clusters([32] * 8, 8)] == [1] * 8
