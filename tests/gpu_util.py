"""Helpers shared by the GPU tests: run a synthetic problem through the CUDA
library (via the binding) and through the FP64 oracle, and compare."""
import numpy as np

import oracle
from paper_1804_10987_gb300 import dp, synth

# Relative error bar of the FP32 path against the FP64 oracle (per subcarrier,
# ||X_gpu - X_ref||_F / ||X_ref||_F over the B x K block).
TOL_FP32 = 1e-5


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err_per_sc(Xg: np.ndarray, Xr: np.ndarray) -> np.ndarray:
    n = Xr.shape[0]
    d = np.linalg.norm((Xg.astype(np.complex128) - Xr).reshape(n, -1), axis=1)
    r = np.linalg.norm(Xr.reshape(n, -1), axis=1)
    return d / np.where(r > 0, r, 1.0)


def entry_err_per_sc(Xg: np.ndarray, Xr: np.ndarray) -> np.ndarray:
    """Per subcarrier: the largest entry error over the B x K block, relative
    to the block's largest entry (catches a few bad entries that the
    Frobenius norm would average away)."""
    n = Xr.shape[0]
    d = np.abs(Xg.astype(np.complex128) - Xr).reshape(n, -1).max(axis=1)
    r = np.abs(Xr).reshape(n, -1).max(axis=1)
    return d / np.where(r > 0, r, 1.0)


def oracle_of(p: synth.Problem, mode=None, tau=None, nthreads=8, **kw):
    mode = mode or p.mode
    return oracle.precode(p.H, p.S, p.cluster_sizes, mode, rho2=p.rho2, N0=p.N0, Es=p.Es,
                          tau=p.tau if tau is None else tau, nthreads=nthreads, **kw)


def plan_of(p: synth.Problem, mode=None, tau=None, prec="fp32", refine=0, **kw):
    """A plan for problem p; refine follows the ABI (0 automatic, 1 always,
    -1 never)."""
    mode = mode or p.mode
    return dp.Plan(p.U, p.B, p.C, p.n_sc, p.K, mode=mode, prec=prec, rho2=p.rho2, N0=p.N0,
                   Es=p.Es, tau=p.tau if tau is None else tau, refine=refine,
                   cluster_sizes=p.cluster_sizes, **kw)


def gpu_precode(p: synth.Problem, mode=None, tau=None, prec="fp32", refine=0):
    import torch
    pl = plan_of(p, mode, tau, prec, refine)
    H, S = to_dev(p.H), to_dev(p.S)
    X = torch.full(pl.shapes()["X"], float("nan"), dtype=torch.complex64, device="cuda")
    pl.precode(H, S, X)
    st = pl.status_get()
    Xh = X.cpu().numpy()
    pl.close()
    return Xh, st
