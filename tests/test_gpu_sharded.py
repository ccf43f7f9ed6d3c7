"""The cluster-sharded PD-WF driver with the CUDA library's steps (dp_gram_local,
dp_solve, dp_precode_apply) on one GPU: a one-rank NCCL group, whose reduce
and broadcast pass through, against the FP64 oracle's centralized WF.  The
multi-rank host logic is tested on CPU (test_sharded.py)."""
import os
import socket

import numpy as np
import pytest

from gpu_util import TOL_FP32, oracle_of, rel_err_per_sc, to_dev
from paper_1804_10987_gb300 import sharded, synth

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_driver_on_one_gpu_matches_oracle():
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        p = synth.make_problem(16, 256, 8, 120, 14, 16, 10.0, seed=synth.seed_for(2, 960))
        (c0, nc, a0, ants), = sharded.split_clusters(p.cluster_sizes, 1)
        drv = sharded.ShardedPDWF(p.U, ants, p.n_sc, p.K, p.N0)
        X = drv.precode(to_dev(p.H[:, a0:a0 + ants].copy()), to_dev(p.S))
        torch.cuda.synchronize()
        err = rel_err_per_sc(X.cpu().numpy(), oracle_of(p)["X"])
        assert err.max() <= TOL_FP32, err.max()
        assert np.isfinite(X.cpu().numpy()).all()
    finally:
        dist.destroy_process_group()
