// dp_fdsmall.cu -- FD-WF clusters with fewer antennas than users, in the
// paper's B_c x B_c form (Sec. III-D): for B_c < U,
//   Q_c = (H_c^H H_c + kappa_c I_{B_c})^{-1} H_c^H,
//   x_c = sqrt(rho_c^2 / (tr(Q_c^H Q_c) Es)) Q_c s,
// which replaces the U x U inverse by a B_c x B_c one.  One warp per
// cluster system (B_c <= BCP <= 32).  Lane (a, part) = (lane % BCP,
// lane / BCP) works on antenna a of the cluster and on the users
// u = part (mod 32 / BCP) of every chunk, so that all 32 lanes share the
// user loops when BCP < 32:
//   1. G'[a][b] = sum_u conj(H[a][u]) H[b][u] over user chunks of 16 staged in
//      shared memory; the parts' partial rows are summed by shuffles, after
//      which every part holds row a of G' in registers,
//   2. in-place Gauss-Jordan inverse of A' = G' + kappa_c I in registers
//      (row a of every part, identical across the parts),
//   3. Q[a][u] = sum_b T'[a][b] conj(H[b][u]) chunk by chunk; tr(Q^H Q) is
//      accumulated as the definition (no Lemma 1 subtraction to cancel) and
//      x[k][a] += sum_u Q[a][u] s_k[u] into per-part shared accumulators,
//   4. scale = sqrt(rho_c^2 / (Es tr(Q^H Q))), X[k][lo + a] = scale times the
//      sum of the parts' accumulators, in part order.
#include "dp_blocks.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

constexpr int UC = 16;          // users per staged chunk
constexpr int FD_WARPS = 4;     // warps (systems in flight) per CTA

__host__ __device__ constexpr size_t fd_warp_floats(int BCP, int K) {
  // H chunk [BCP][UC] + S chunk [K][UC] + x accumulators [32 / BCP][K][BCP]
  // (complex)
  return 2 * ((size_t)BCP * UC + (size_t)K * UC + (size_t)K * 32);
}

template <int BCP>
__device__ void fd_small_system(const InstDesc &in, int sys, float2 *ws, int lane) {
  constexpr int PARTS = 32 / BCP;  // lanes sharing one antenna row
  constexpr int UPL = UC / PARTS;  // users of a chunk per lane
  static_assert(32 % BCP == 0 && UC % PARTS == 0, "lane split");
  const SysDesc &d = in.d;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  int lo, hi;
  sys_rows(d, g, lo, hi);
  const int nb = hi - lo, U = d.U, K = d.K;
  if (!(nb < U && nb <= BCP)) return;  // not a small-cluster system
  const int a = lane % BCP, part = lane / BCP;
  float2 *Hc = ws;                      // [BCP][UC]
  float2 *Sc = Hc + BCP * UC;           // [K][UC]
  float2 *Xa = Sc + K * UC;             // [PARTS][K][BCP]
  const float2 *Hn = in.H + ((size_t)n * d.B + lo) * U;
  const float2 *Sn = in.S + (size_t)n * K * U;
  bool fin = true;

  // 1. antenna-side Gram, row a (this part's users)
  float2 row[BCP];
#pragma unroll
  for (int b = 0; b < BCP; ++b) row[b] = make_float2(0.f, 0.f);
  for (int u0 = 0; u0 < U; u0 += UC) {
    const int uc = min(UC, U - u0);
    __syncwarp();
    for (int e = lane; e < BCP * UC; e += 32) {
      const int b = e / UC, u = e - b * UC;
      float2 v = make_float2(0.f, 0.f);
      if (b < nb && u < uc) {
        v = __ldg(Hn + (size_t)b * U + u0 + u);
        fin = fin && cfinite(v);
      }
      Hc[e] = v;
    }
    __syncwarp();
    float2 my[UPL];
#pragma unroll
    for (int uu = 0; uu < UPL; ++uu) my[uu] = Hc[a * UC + part + uu * PARTS];
#pragma unroll
    for (int b = 0; b < BCP; ++b) {
      if (b < nb) {
#pragma unroll
        for (int uu = 0; uu < UPL; ++uu) cmac_cj(row[b], my[uu], Hc[b * UC + part + uu * PARTS]);
      }
    }
  }
  // the parts' partial rows: a butterfly over the lanes a, a + BCP, ...
#pragma unroll
  for (int o = BCP; o < 32; o <<= 1) {
#pragma unroll
    for (int b = 0; b < BCP; ++b) {
      row[b].x += __shfl_xor_sync(FULL, row[b].x, o);
      row[b].y += __shfl_xor_sync(FULL, row[b].y, o);
    }
  }
  for (int e = lane; e < K * U; e += 32) fin = fin && cfinite(__ldg(Sn + e));
  fin = __all_sync(FULL, fin);
  if (a >= nb) {
#pragma unroll
    for (int b = 0; b < BCP; ++b) row[b] = make_float2(0.f, 0.f);
  }
  // this cluster's regularizer (read where it is used: short live range)
  const float kap = d.ckr ? __ldg(&d.ckr[g].x) : d.kappa;
#pragma unroll
  for (int b = 0; b < BCP; ++b)
    if (b == a) {
      row[b].y = 0.f;
      row[b].x += kap;  // A' = G' + kappa_c I
    }

  // 2. T' = A'^{-1} (pivot rows come from the lanes of part 0)
  int st = fin ? ST_OK : ST_NONFINITE;
  if (st == ST_OK && !warp_gj_inverse<BCP>(row, a, nb)) st = ST_NOT_PD;

  // 3. Q = T' H_c^H by user chunks; t = ||Q||_F^2; x accumulators
  float2 *Xp = Xa + part * K * BCP;  // this part's accumulators
  for (int e = lane; e < PARTS * K * BCP; e += 32) Xa[e] = make_float2(0.f, 0.f);
  float tq = 0.f;
  if (st == ST_OK) {
    for (int u0 = 0; u0 < U; u0 += UC) {
      const int uc = min(UC, U - u0);
      __syncwarp();
      for (int e = lane; e < BCP * UC; e += 32) {
        const int b = e / UC, u = e - b * UC;
        Hc[e] = (b < nb && u < uc) ? __ldg(Hn + (size_t)b * U + u0 + u) : make_float2(0.f, 0.f);
      }
      for (int e = lane; e < K * UC; e += 32) {
        const int k = e / UC, u = e - k * UC;
        Sc[e] = u < uc ? __ldg(Sn + (size_t)k * U + u0 + u) : make_float2(0.f, 0.f);
      }
      __syncwarp();
      float2 q[UPL];
#pragma unroll
      for (int uu = 0; uu < UPL; ++uu) q[uu] = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < BCP; ++b) {
        if (b < nb) {
#pragma unroll
          for (int uu = 0; uu < UPL; ++uu)
            cmac(q[uu], row[b], cconj(Hc[b * UC + part + uu * PARTS]));
        }
      }
      if (a < nb) {
#pragma unroll
        for (int uu = 0; uu < UPL; ++uu) tq = fmaf(q[uu].x, q[uu].x, fmaf(q[uu].y, q[uu].y, tq));
        for (int k = 0; k < K; ++k) {
          float2 acc = Xp[k * BCP + a];
#pragma unroll
          for (int uu = 0; uu < UPL; ++uu) cmac(acc, q[uu], Sc[k * UC + part + uu * PARTS]);
          Xp[k * BCP + a] = acc;
        }
      }
    }
  }
  const float t = warp_sum(a < nb ? tq : 0.f);
  float sc = 0.f;
  if (st == ST_OK) {
    if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
    else sc = sqrtf((d.ckr ? __ldg(&d.ckr[g].y) : d.rho2_sys) / (d.Es * t));
  }
  __syncwarp();
  // 4. x_c = scale Q_c s, the parts summed in order
  if (part == 0 && a < nb) {
    float2 *Xn = in.X + (size_t)n * K * d.B + lo + a;
    for (int k = 0; k < K; ++k) {
      float2 v = Xa[k * BCP + a];
#pragma unroll
      for (int pp = 1; pp < PARTS; ++pp) {
        const float2 w = Xa[(pp * K + k) * BCP + a];
        v.x += w.x;
        v.y += w.y;
      }
      Xn[(size_t)k * d.B] = st == ST_OK ? cscale(v, sc) : make_float2(0.f, 0.f);
    }
  }
  if (lane == 0) {
    in.status[sys] = st;
    if (in.scale_out) in.scale_out[sys] = sc;
  }
}

// BCP = 32 is capped at 128 registers for a fourth CTA per SM (measured
// 12 % faster despite a few spilled words); the narrower forms keep their
// natural register count (no minimum, 0).
template <int BCP>
__global__ void __launch_bounds__(32 * FD_WARPS, BCP == 32 ? 4 : 0) k_fd_small(InstDesc in) {
  extern __shared__ __align__(16) float2 fd_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sys = blockIdx.x * FD_WARPS + w;
  if (sys >= in.d.n_sc * in.d.nsys) return;  // warp-uniform, no CTA barriers below
  float2 *ws = fd_smem + (size_t)w * fd_warp_floats(BCP, in.d.K) / 2;
  fd_small_system<BCP>(in, sys, ws, lane);
}

// Persistent form: every warp pulls items (one system each) from the queue
// (the same register cap as above for BCP = 32).
template <int BCP>
__global__ void __launch_bounds__(32 * FD_WARPS, BCP == 32 ? 4 : 0)
    k_batch_fd_small(const InstDesc *__restrict__ insts, const WorkItem *__restrict__ items,
                     int n_items, int *__restrict__ queue, int Kmax) {
  extern __shared__ __align__(16) float2 fd_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 *ws = fd_smem + (size_t)w * fd_warp_floats(BCP, Kmax) / 2;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(queue, 1);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    const WorkItem wi = items[it];
    fd_small_system<BCP>(insts[wi.inst], wi.sys0, ws, lane);
  }
}

template <int BCP>
cudaError_t launch_fd_small_t(const InstDesc &in, cudaStream_t s) {
  const size_t bytes = FD_WARPS * fd_warp_floats(BCP, in.d.K) * 4;
  cudaFuncSetAttribute(k_fd_small<BCP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fd_small<BCP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  const int total = in.d.n_sc * in.d.nsys;
  k_fd_small<BCP><<<(total + FD_WARPS - 1) / FD_WARPS, 32 * FD_WARPS, bytes, s>>>(in);
  return cudaGetLastError();
}

template <int BCP>
cudaError_t launch_batch_fd_small_t(const InstDesc *insts, const WorkItem *items, int n_items,
                                    int *queue, int Kmax, int grid, cudaStream_t s) {
  const size_t bytes = FD_WARPS * fd_warp_floats(BCP, Kmax) * 4;
  cudaFuncSetAttribute(k_batch_fd_small<BCP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_fd_small<BCP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  k_batch_fd_small<BCP><<<grid, 32 * FD_WARPS, bytes, s>>>(insts, items, n_items, queue, Kmax);
  return cudaGetLastError();
}

template <int BCP>
int fd_small_blocks_t(int Kmax) {
  const size_t bytes = FD_WARPS * fd_warp_floats(BCP, Kmax) * 4;
  if (bytes > 48 * 1024 &&
      cudaFuncSetAttribute(k_batch_fd_small<BCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 0;
  return resident_blocks((const void *)k_batch_fd_small<BCP>, 32 * FD_WARPS, bytes, 0);
}

}  // namespace

int fd_small_bcp(int maxbc) { return maxbc <= 8 ? 8 : (maxbc <= 16 ? 16 : (maxbc <= 32 ? 32 : 0)); }

cudaError_t launch_fd_small(const InstDesc &in, int bcp, cudaStream_t s) {
  switch (bcp) {
    case 8: return launch_fd_small_t<8>(in, s);
    case 16: return launch_fd_small_t<16>(in, s);
    case 32: return launch_fd_small_t<32>(in, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_fd_small(int bcp, const InstDesc *insts, const WorkItem *items,
                                  int n_items, int *queue, int Kmax, int grid, cudaStream_t s) {
  switch (bcp) {
    case 8: return launch_batch_fd_small_t<8>(insts, items, n_items, queue, Kmax, grid, s);
    case 16: return launch_batch_fd_small_t<16>(insts, items, n_items, queue, Kmax, grid, s);
    case 32: return launch_batch_fd_small_t<32>(insts, items, n_items, queue, Kmax, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int fd_small_max_blocks_per_sm(int bcp, int Kmax) {
  switch (bcp) {
    case 8: return fd_small_blocks_t<8>(Kmax);
    case 16: return fd_small_blocks_t<16>(Kmax);
    case 32: return fd_small_blocks_t<32>(Kmax);
    default: return 0;
  }
}

}  // namespace dp
