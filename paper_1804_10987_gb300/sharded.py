"""PD-WF with the antenna clusters sharded over the GPUs of one node (the
paper's own mapping, Sec. IV-A and IV-B: one cluster group per GPU, the local
Grams reduced to a master, the whitened symbols broadcast back).

Per slot, rank r holds the contiguous antenna block of its clusters, H_r
[n_sc][B_r][U], and:
  1. forms its local Gram G_r = sum over its clusters of H_c H_c^H (step a1 and
     its share of the adder tree a2, on its GPU),
  2. the G_r are summed onto the root rank (a reduce: the rest of a2),
  3. the root solves the regularized system (a3-a5): z = A^{-1} s and the
     precoding factor, from the summed Gram,
  4. z and the factor are broadcast to every rank,
  5. each rank applies x_c = scale H_c^H z to its own antennas (a6).
The concatenation of the ranks' X_r (in rank order) is the centralized WF of
Thm. 1, computed the partially decentralized way (Sec. III-B).

The collectives move n_sc U^2 complex values (the reduce) and n_sc (K U + 1)
values (the broadcast) per slot; they go through torch.distributed (NCCL on
GPUs), as real views of the complex arrays.  The arithmetic of steps 1, 3 and
5 is the CUDA library's (dp_gram_local, dp_solve, dp_precode_apply); `ops`
lets a caller substitute other implementations of those three steps (the CPU
tests of the host logic do).
"""
from __future__ import annotations

from dataclasses import dataclass


def split_clusters(cluster_sizes, world: int):
    """Contiguous runs of clusters per rank, as even in antennas as the
    cluster boundaries allow: returns [(first cluster, cluster count, first
    antenna, antennas)] for ranks 0..world-1.  Every rank gets >= 1 cluster."""
    C = len(cluster_sizes)
    if world < 1 or world > C:
        raise ValueError(f"{world} ranks cannot share {C} clusters")
    B = sum(cluster_sizes)
    out, c0, a0 = [], 0, 0
    for r in range(world):
        left = world - r
        if left == 1:
            n = C - c0
        else:
            target = (B - a0) / left
            n, acc = 0, 0
            while c0 + n < C - (left - 1) and (n == 0 or acc + cluster_sizes[c0 + n] / 2 <= target):
                acc += cluster_sizes[c0 + n]
                n += 1
        ants = sum(cluster_sizes[c0:c0 + n])
        out.append((c0, n, a0, ants))
        c0, a0 = c0 + n, a0 + ants
    return out


@dataclass
class CudaOps:
    """Steps 1, 3 and 5 on this rank's GPU through the C ABI: a plan over the
    rank's antennas (one cluster: its Gram is the local sum) for the Gram and
    the apply, and the same plan's dp_solve on the summed Gram (kappa depends
    on U, N0 and rho^2 only)."""
    plan: object

    def gram(self, H_r):
        G = self.plan.empty("Gloc")  # [1][n_sc][U][U]
        self.plan.gram_local(H_r, G)
        return G[0]

    def solve(self, G, S):
        Z, scale = self.plan.empty("Z"), self.plan.empty("scale")
        self.plan.solve(G, S, Z, scale)
        return Z, scale

    def apply(self, H_r, Z, scale):
        X = self.plan.empty("X")
        self.plan.precode_apply(H_r, Z, scale, X)
        return X


class ShardedPDWF:
    """One rank's part of a cluster-sharded PD-WF precoder.

    U users; this rank's antennas B_r (its clusters' contiguous block); n_sc
    subcarriers and K symbols per slot; N0, rho2, Es as in dp_plan_desc.
    group: a torch.distributed process group (None: the default one); root:
    the rank that solves.  ops: the three steps (default: CudaOps on the
    current GPU, FP32)."""

    def __init__(self, U: int, B_r: int, n_sc: int, K: int, N0: float, rho2: float = 1.0,
                 Es: float = 1.0, group=None, root: int = 0, ops=None, stream=None):
        import torch.distributed as dist
        self.U, self.B_r, self.n_sc, self.K = U, B_r, n_sc, K
        self.group, self.root = group, root
        self.rank = dist.get_rank(group)
        if ops is None:
            from . import dp
            ops = CudaOps(dp.Plan(U, B_r, 1, n_sc, K, mode="wf", prec="fp32", rho2=rho2, N0=N0,
                                  Es=Es, stream=stream))
        self.ops = ops

    def precode(self, H_r, S):
        """H_r [n_sc][B_r][U] (this rank's antennas), S [n_sc][K][U] (the same
        symbols on every rank); returns X_r [n_sc][K][B_r]."""
        import torch
        import torch.distributed as dist
        G = self.ops.gram(H_r)                                          # 1
        Gr = torch.view_as_real(G.contiguous())
        dist.reduce(Gr, dst=self.root, op=dist.ReduceOp.SUM, group=self.group)  # 2
        G = torch.view_as_complex(Gr)
        if self.rank == self.root:
            Z, scale = self.ops.solve(G, S)                             # 3
        else:
            Z = torch.empty((self.n_sc, self.K, self.U), dtype=S.dtype, device=S.device)
            scale = torch.empty((self.n_sc,), dtype=torch.float32, device=S.device)
        Zr = torch.view_as_real(Z.contiguous())
        dist.broadcast(Zr, src=self.root, group=self.group)             # 4
        dist.broadcast(scale, src=self.root, group=self.group)
        return self.ops.apply(H_r, torch.view_as_complex(Zr), scale)    # 5
