"""Seeded synthetic inputs for the precoding path: channels, symbols, noise
levels and the named workloads.

This module holds none of the precoder's arithmetic.  It is the one module the
CUDA path's tests and benchmark share with the FP64 oracle's tests: both sides
draw the same arrays from here and compute from them independently.

Recipe (the paper's simulation setting, Sec. III-E and Sec. IV-C):
* channel: i.i.d. Rayleigh, H[u][b] ~ CN(0, 1/B), independent per subcarrier,
  constant over the K OFDM symbols of a slot (block fading, Eq. (1));
  or Kronecker exponential correlation H = R_U^{1/2} H_w R_B^{1/2} with
  [R]_{ij} = r^{|i-j|} (r_B = 0.7 over the antenna index, r_U = 0.3 over the
  user index), which keeps E|H[u][b]|^2 = 1/B;
* symbols: square QAM with Gray labels, normalized to Es = E|s|^2 = 1;
* noise: SNR = rho^2 / N0, so N0 = rho^2 10^(-SNR/10) with rho^2 = 1.
Storage: H [n_sc][B][U] complex64 (user index fastest), S [n_sc][K][U].

CPU draws use numpy's Philox generator, whose streams are identical on every
host; large workloads draw on the GPU with torch's Philox generator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1804_10987


def seed_for(config: int, i: int = 0) -> int:
    """Seed of draw i of workload `config` (1-based workload number)."""
    return SEED_BASE + 1000 * config + i


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def n0_from_snr(snr_db: float, rho2: float = 1.0) -> float:
    return rho2 * 10.0 ** (-snr_db / 10.0)


def gray_pam_levels(m: int) -> np.ndarray:
    """Amplitudes of an m-level PAM indexed by Gray label (unnormalized, odd
    integers -(m-1)..(m-1))."""
    bits = int(round(math.log2(m)))
    assert 1 << bits == m
    levels = np.zeros(m)
    for pos in range(m):
        gray = pos ^ (pos >> 1)
        levels[gray] = 2 * pos - (m - 1)
    return levels


def qam_constellation(order: int) -> np.ndarray:
    """Square QAM of `order` points, index = (Gray label of I) * sqrt(order) +
    (Gray label of Q), normalized to unit average energy."""
    m = int(round(math.sqrt(order)))
    assert m * m == order and order >= 4
    lv = gray_pam_levels(m)
    pts = (lv[:, None] + 1j * lv[None, :]).reshape(-1)
    return pts / math.sqrt(np.mean(np.abs(pts) ** 2))


def qam_symbols(order: int, shape, g: np.random.Generator) -> np.ndarray:
    idx = g.integers(0, order, size=shape)
    return qam_constellation(order)[idx].astype(np.complex64)


def rayleigh(n_sc: int, B: int, U: int, g: np.random.Generator) -> np.ndarray:
    """i.i.d. CN(0, 1/B) channel, stored [n_sc][B][U] complex64."""
    sd = math.sqrt(0.5 / B)
    re = g.standard_normal((n_sc, B, U)) * sd
    im = g.standard_normal((n_sc, B, U)) * sd
    return (re + 1j * im).astype(np.complex64)


def exp_corr(n: int, r: float) -> np.ndarray:
    i = np.arange(n)
    return r ** np.abs(i[:, None] - i[None, :])


def kronecker(n_sc: int, B: int, U: int, r_B: float, r_U: float,
              g: np.random.Generator) -> np.ndarray:
    """Kronecker-correlated channel with exponential correlation at both ends,
    stored [n_sc][B][U] complex64.  With H stored transposed (Ht = H^T, B x U),
    Ht = L_B Hw^T L_U^T where R = L L^T."""
    LB = np.linalg.cholesky(exp_corr(B, r_B))
    LU = np.linalg.cholesky(exp_corr(U, r_U))
    hw = rayleigh(n_sc, B, U, g).astype(np.complex128)
    out = np.empty((n_sc, B, U), np.complex64)
    step = max(1, (1 << 22) // max(1, B * U))
    for lo in range(0, n_sc, step):
        out[lo:lo + step] = (LB @ hw[lo:lo + step] @ LU.T).astype(np.complex64)
    return out


def equal_clusters(B: int, C: int) -> list[int]:
    assert B % C == 0
    return [B // C] * C


@dataclasses.dataclass
class Problem:
    """One precoding problem: a slot of n_sc subcarriers x K OFDM symbols."""
    U: int
    B: int
    cluster_sizes: list
    n_sc: int
    K: int
    H: np.ndarray          # [n_sc][B][U] complex64
    S: np.ndarray          # [n_sc][K][U] complex64
    rho2: float = 1.0
    N0: float = 0.1
    Es: float = 1.0
    tau: float = 0.125
    mode: str = "wf"

    @property
    def C(self) -> int:
        return len(self.cluster_sizes)


def make_problem(U: int, B: int, C: int, n_sc: int, K: int, qam: int, snr_db: float,
                 seed: int, mode: str = "wf", tau: float = 0.125, channel: str = "iid",
                 r_B: float = 0.7, r_U: float = 0.3, cluster_sizes=None) -> Problem:
    g = rng(seed)
    if channel == "iid":
        H = rayleigh(n_sc, B, U, g)
    elif channel == "kron":
        H = kronecker(n_sc, B, U, r_B, r_U, g)
    else:
        raise ValueError(channel)
    S = qam_symbols(qam, (n_sc, K, U), g)
    cs = list(cluster_sizes) if cluster_sizes is not None else equal_clusters(B, C)
    return Problem(U, B, cs, n_sc, K, H, S, 1.0, n0_from_snr(snr_db), 1.0, tau, mode)


# --- the named workloads ---------------------------------------------------------

WORKLOADS = {
    # plain centralized WF through the decentralized Gram sum
    "c1": dict(U=8, B=64, C=2, n_sc=64, K=14, qam=4, snr_db=10.0),
    # ZF, centralized (= PD) WF and FD-WF (tau = 0.125 and 1), SNR 0..20 dB
    "c2": dict(U=16, B=256, C=8, n_sc=1200, K=14, qam=16, snr_db=10.0),
    # reduced-precision Gram; i.i.d. and Kronecker-correlated channels
    "c3": dict(U=32, B=512, C=16, n_sc=3300, K=14, qam=64, snr_db=10.0),
}
C2_SNRS = (0.0, 5.0, 10.0, 15.0, 20.0)

# batched uneven workload: per-instance size distributions
C4_U = (8, 16, 24, 32, 48, 64)
C4_B = (64, 128, 256, 512, 1024)
C4_C = (1, 2, 4, 8, 16, 32)
C4_NSC = (72, 3300)


def c4_instance_shapes(n_inst: int, seed: int) -> list[dict]:
    """Sizes of the batched uneven workload: U, B uniform over their sets, C
    uniform over the listed values that divide B, n_sc uniform in [72, 3300],
    channel i.i.d. or Kronecker with equal odds, mode WF or FD-WF (tau 0.125)
    with equal odds, 64-QAM, 10 dB, K = 14."""
    g = rng(seed)
    out = []
    for _ in range(n_inst):
        U = int(g.choice(C4_U))
        B = int(g.choice(C4_B))
        Cs = [c for c in C4_C if B % c == 0]
        C = int(g.choice(Cs))
        n_sc = int(g.integers(C4_NSC[0], C4_NSC[1] + 1))
        chan = "iid" if g.integers(0, 2) == 0 else "kron"
        mode = "wf" if g.integers(0, 2) == 0 else "fdwf"
        out.append(dict(U=U, B=B, C=C, n_sc=n_sc, K=14, qam=64, snr_db=10.0,
                        channel=chan, mode=mode, tau=0.125))
    return out


def torch_channel(n_sc: int, B: int, U: int, channel: str, gen, device,
                  r_B: float = 0.7, r_U: float = 0.3):
    """The same channel recipe drawn on a torch device (for workloads too large
    to draw on the host).  Returns a complex64 tensor [n_sc][B][U]."""
    import torch
    sd = math.sqrt(0.5 / B)
    h = torch.complex(torch.randn((n_sc, B, U), generator=gen, device=device) * sd,
                      torch.randn((n_sc, B, U), generator=gen, device=device) * sd)
    if channel == "kron":
        # the factors on the host (numpy), so that the draw needs no device
        # linear-algebra library
        LB = torch.tensor(np.linalg.cholesky(exp_corr(B, r_B)), dtype=torch.complex64,
                          device=device)
        LU = torch.tensor(np.linalg.cholesky(exp_corr(U, r_U)), dtype=torch.complex64,
                          device=device)
        h = LB @ h @ LU.T
    return h.contiguous()


def torch_symbols(order: int, shape, gen, device):
    import torch
    pts = torch.tensor(qam_constellation(order), dtype=torch.complex64, device=device)
    idx = torch.randint(0, order, shape, generator=gen, device=device)
    return pts[idx].contiguous()
