// dp_fp32_impl.cuh -- FP32 kernels of the precoding path (steps a1-a6) and
// their launchers, instantiated per padded user count by dp_fp32_u*.cu
// (dp_fp32.cu dispatches on the user count).
//
//   k_gram        a1 (+ a2 when one system spans all clusters): per-system
//                 Gram, antenna rows streamed through shared memory by 1-D
//                 bulk copies (Sec. III-B, G_c = H_c H_c^H)
//   k_solve_warp  a3-a5, one warp per system, the U x U matrix held in
//                 registers (one row per lane): Gauss-Jordan inverse, the
//                 precoding factor (Thm. 1 / Lemma 1) and z = A^{-1} s
//   k_solve_cta   a3-a5 for U > 32, one CTA per system, matrix in shared memory
//   k_apply       a6: x_c = scale H_c^H z (Sec. III-B local precoding)
//   k_fused       a1-a6 in one CTA per system with the antenna block resident
//                 in shared memory: H is read from HBM once.
#pragma once

#include "dp_blocks.cuh"
#include "dp_internal.h"

namespace dp {

namespace {

// Status of one system: a plain store into status[system]; the host folds the
// systems of a subcarrier.
__device__ __forceinline__ void report(int *status, int sys, int st) { status[sys] = st; }

// ------------------------------------------------------------------ gram ---
template <int UP>
__global__ void __launch_bounds__(NT) k_gram(SysDesc d, const float2 *__restrict__ H,
                                             float2 *__restrict__ Gout, int chunk) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int RS = Geo<UP>::RS;
  const int tid = threadIdx.x;
  const int sys = blockIdx.x;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  int lo, hi;
  sys_rows(d, g, lo, hi);
  const int nrows = hi - lo;
  if (sys_is_small(d, nrows)) return;
  float *Hs = reinterpret_cast<float *>(smem_raw);
  float2 *G = reinterpret_cast<float2 *>(Hs + (size_t)chunk * RS);
  uint64_t *bar = reinterpret_cast<uint64_t *>(G + UP * UP);
  const bool tma = d.tma_ok != 0;

  zero_row_pads<UP>(Hs, chunk, d.U, tid);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  fence_proxy_async_smem();
  __syncthreads();

  GramAcc<UP> ga;
  ga.init(tid);
  const float2 *Hn = H + (size_t)n * d.B * d.U;
  bool timeout = false;
  int it = 0;
  for (int c0 = 0; c0 < nrows; c0 += chunk, ++it) {
    const int m = min(chunk, nrows - c0);
    if (c0 > 0) {
      __syncthreads();
      fence_proxy_async_smem();
    }
    fetch_rows<UP>(Hs, Hn, lo + c0, m, d.U, tma, bar, tid);
    if (tma) {
      if (!mbar_wait_cta(bar, it & 1)) timeout = true;
    } else {
      __syncthreads();
    }
    if (timeout) {
      if (tid == 0) mbar_wait(bar, it & 1);  // let copies in flight land before exiting
      __syncthreads();
      break;
    }
    ga.accumulate(Hs, m);
  }
  __syncthreads();
  ga.finish(G, tid);
  __syncthreads();
  float2 *out = Gout + ((size_t)g * d.n_sc + n) * d.U * d.U;
  const float nanv = __int_as_float(0x7fc00000);
  for (int e = tid; e < d.U * d.U; e += NT) {
    const int i = e / d.U, j = e - i * d.U;
    out[e] = timeout ? make_float2(nanv, nanv) : G[i * UP + j];
  }
}

template <int UP>
__global__ void __launch_bounds__(NT) k_solve_warp(SysDesc d, const float2 *__restrict__ Gin,
                                                   const float2 *__restrict__ S,
                                                   float2 *__restrict__ Z,
                                                   float *__restrict__ scale,
                                                   int *__restrict__ status) {
  static_assert(UP <= 32, "one row per lane");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sys = blockIdx.x * (NT / 32) + w;
  const int nsys_total = d.n_sc * d.nsys;
  if (sys >= nsys_total) return;  // warp-uniform; no CTA barriers below
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  const int U = d.U, K = d.K;
  {
    int lo, hi;
    sys_rows(d, g, lo, hi);
    if (sys_is_small(d, hi - lo)) return;
  }
  float2 *Gw = reinterpret_cast<float2 *>(smem_raw) + (size_t)w * (UP * UP + K * UP);
  float2 *Sw = Gw + UP * UP;

  const float2 *gsrc = Gin + ((size_t)g * d.n_sc + n) * U * U;
  bool fin = true;
  for (int e = lane; e < UP * UP; e += 32) {
    const int i = e / UP, j = e - i * UP;
    float2 v = make_float2(0.f, 0.f);
    if (i < U && j < U) {
      v = __ldg(gsrc + i * U + j);
      fin = fin && cfinite(v);
    }
    Gw[e] = v;
  }
  const float2 *ssrc = S + (size_t)n * K * U;
  for (int e = lane; e < K * UP; e += 32) {
    const int k = e / UP, u = e - k * UP;
    float2 v = make_float2(0.f, 0.f);
    if (u < U) {
      v = __ldg(ssrc + (size_t)k * U + u);
      fin = fin && cfinite(v);
    }
    Sw[e] = v;
  }
  fin = __all_sync(FULL, fin);
  __syncwarp();

  float sc = 0.f;
  const int st = warp_solve<UP>(Gw, Sw, Z + (size_t)sys * K * U, U, sys_kappa(d, sys), sys_rho2(d, sys), d.Es, U,
                                K, lane, fin, sc, d.mrt != 0);
  if (lane == 0) {
    scale[sys] = sc;
    report(status, sys, st);
  }
}

// ------------------------------------------------------- CTA-per-system solve ---
template <int UP>
__global__ void __launch_bounds__(NT) k_solve_cta(SysDesc d, const float2 *__restrict__ Gin,
                                                  const float2 *__restrict__ S,
                                                  float2 *__restrict__ Z,
                                                  float *__restrict__ scale,
                                                  int *__restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int sys = blockIdx.x;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  const int U = d.U, K = d.K;
  {
    int lo, hi;
    sys_rows(d, g, lo, hi);
    if (sys_is_small(d, hi - lo)) return;
  }
  float2 *G = reinterpret_cast<float2 *>(smem_raw);
  float2 *A = G + UP * UP;
  float2 *Ss = A + UP * UP;
  float2 *Zs = Ss + K * UP;
  float *red = reinterpret_cast<float *>(Zs + K * UP);

  const float2 *gsrc = Gin + ((size_t)g * d.n_sc + n) * U * U;
  bool fin = true;
  for (int e = tid; e < UP * UP; e += NT) {
    const int i = e / UP, j = e - i * UP;
    float2 v = make_float2(0.f, 0.f);
    if (i < U && j < U) {
      v = __ldg(gsrc + i * U + j);
      fin = fin && cfinite(v);
    }
    G[e] = v;
    if (i == j) v.x += sys_kappa(d, sys);
    A[e] = v;
  }
  fin = __syncthreads_and(fin) != 0;
  fin = load_symbols<UP>(S + (size_t)n * K * U, Ss, U, K, tid) && fin;
  int st = fin ? ST_OK : ST_NONFINITE;
  float sc = 0.f;
  if (st == ST_OK && d.mrt) {  // MRT: t = tr(G), z = s
    const float t = cta_mrt<UP>(G, Ss, Zs, U, K, red, tid);
    if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
    else sc = sqrtf(sys_rho2(d, sys) / (d.Es * t));
  } else {
    if (st == ST_OK) st = cta_gj_inverse<UP>(A, U, tid);
    if (st == ST_OK) {
      const float t = cta_trace_tgt<UP>(A, G, sys_kappa(d, sys), U, red, tid);
      if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
      else sc = sqrtf(sys_rho2(d, sys) / (d.Es * t));
    }
  }
  if (st == ST_OK && !d.mrt) cta_whiten<UP>(A, Ss, Zs, U, K, tid);
  __syncthreads();
  float2 *zdst = Z + (size_t)sys * K * U;
  for (int e = tid; e < K * U; e += NT) {
    const int k = e / U, i = e - k * U;
    zdst[e] = (st == ST_OK) ? Zs[k * UP + i] : make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    scale[sys] = sc;
    report(status, sys, st);
  }
}

// ----------------------------------------------------------------- apply ---
template <int UP>
__global__ void __launch_bounds__(NT) k_apply(SysDesc d, const float2 *__restrict__ H,
                                              const float2 *__restrict__ Z,
                                              const float *__restrict__ scale,
                                              float2 *__restrict__ X, int chunk) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int RS = Geo<UP>::RS;
  const int tid = threadIdx.x;
  const int sys = blockIdx.x;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  int lo, hi;
  sys_rows(d, g, lo, hi);
  const int nrows = hi - lo;
  if (sys_is_small(d, nrows)) return;
  const int U = d.U, K = d.K;
  float *Hs = reinterpret_cast<float *>(smem_raw);
  float2 *Zs = reinterpret_cast<float2 *>(Hs + (size_t)chunk * RS);
  uint64_t *bar = reinterpret_cast<uint64_t *>(Zs + K * UP);
  float2 *Xn = X + (size_t)n * K * d.B;

  const float sc = __ldg(scale + sys);
  if (!(sc > 0.f) || !isfinite(sc)) {  // failed system: zero output
    zero_rows<UP>(nrows, K, Xn, d.B, lo, tid);
    return;
  }
  const float2 *zsrc = Z + (size_t)sys * K * U;
  for (int e = tid; e < K * UP; e += NT) {
    const int k = e / UP, u = e - k * UP;
    Zs[e] = (u < U) ? __ldg(zsrc + (size_t)k * U + u) : make_float2(0.f, 0.f);
  }
  zero_row_pads<UP>(Hs, chunk, U, tid);
  const bool tma = d.tma_ok != 0;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  fence_proxy_async_smem();
  __syncthreads();
  const float2 *Hn = H + (size_t)n * d.B * U;
  bool timeout = false;
  int it = 0;
  for (int c0 = 0; c0 < nrows; c0 += chunk, ++it) {
    const int m = min(chunk, nrows - c0);
    if (c0 > 0) {
      __syncthreads();
      fence_proxy_async_smem();
    }
    fetch_rows<UP>(Hs, Hn, lo + c0, m, U, tma, bar, tid);
    if (tma) {
      if (!mbar_wait_cta(bar, it & 1)) timeout = true;
    } else {
      __syncthreads();
    }
    if (timeout) {
      if (tid == 0) mbar_wait(bar, it & 1);
      __syncthreads();
      zero_rows<UP>(nrows, K, Xn, d.B, lo, tid);
      return;
    }
    apply_rows<UP, 7>(Hs, m, Zs, K, sc, Xn, d.B, lo + c0, tid);
  }
}

template <int UP>
__host__ __device__ constexpr size_t fused_bar_offset(int maxrows, int K) {
  return (size_t)maxrows * Geo<UP>::RS * 4 + 2 * (size_t)UP * UP * 8 + 2 * (size_t)K * UP * 8 +
         16 * 4;
}

// ----------------------------------------------------------------- fused ---
// One system with its antenna block resident in shared memory.  tma_waits
// counts the phases of bar consumed by this CTA so far (persistent CTAs run
// many systems).  Returns false if the bounded wait for the rows gave up.
template <int UP>
__device__ bool fused_system(const InstDesc &in, int sys, unsigned char *smem_raw, int maxrows,
                             int Kmax, uint64_t *bar, uint32_t &tma_waits) {
  constexpr int RS = Geo<UP>::RS;
  const SysDesc &d = in.d;
  const int tid = threadIdx.x;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  int lo, hi;
  sys_rows(d, g, lo, hi);
  const int nrows = hi - lo;
  if (sys_is_small(d, nrows)) return true;  // the B_c x B_c kernel's system
  const int U = d.U, K = d.K;
  float *Hs = reinterpret_cast<float *>(smem_raw);
  float2 *G = reinterpret_cast<float2 *>(Hs + (size_t)maxrows * RS);
  float2 *A = G + UP * UP;
  float2 *Ss = A + UP * UP;
  float2 *Zs = Ss + Kmax * UP;
  float *red = reinterpret_cast<float *>(Zs + Kmax * UP);
  float2 *Xn = in.X + (size_t)n * K * d.B;
  const bool tma = d.tma_ok != 0;

  // a1 prologue: fetch this system's antenna block and the symbols
  __syncthreads();  // the previous system is done with the buffers
  zero_row_pads<UP>(Hs, nrows, U, tid);
  fence_proxy_async_smem();
  __syncthreads();
  fetch_rows<UP>(Hs, in.H + (size_t)n * d.B * U, lo, nrows, U, tma, bar, tid);
  const bool sfin = load_symbols<UP>(in.S + (size_t)n * K * U, Ss, U, K, tid);
  if (tma) {
    const bool ok = mbar_wait_cta(bar, tma_waits & 1);
    ++tma_waits;
    if (!ok) {
      if (tid == 0) mbar_wait(bar, (tma_waits - 1) & 1);
      __syncthreads();
      zero_rows<UP>(nrows, K, Xn, d.B, lo, tid);
      if (tid == 0) {
        report(in.status, sys, ST_TIMEOUT);
        if (in.scale_out) in.scale_out[sys] = 0.f;
      }
      return false;
    }
  }

  // a1 + a2: Gram over all antennas of the system (the cluster sum is the
  // accumulation over the concatenated cluster blocks)
  {
    GramAcc<UP> ga;
    ga.init(tid);
    ga.accumulate(Hs, nrows);
    ga.finish(G, tid);
  }
  __syncthreads();
  bool gfin = true;
  for (int e = tid; e < UP * UP; e += NT) {
    float2 v = G[e];
    gfin = gfin && cfinite(v);
    if (e / UP == e % UP) v.x += sys_kappa(d, sys);  // a3: A = G + kappa I
    A[e] = v;
  }
  gfin = __syncthreads_and(gfin) != 0;
  int st = (sfin && gfin) ? ST_OK : ST_NONFINITE;

  // a3 + a4: inverse and precoding factor
  float sc = 0.f;
  if (st == ST_OK && d.mrt) {  // MRT: t = tr(G), z = s
    const float t = cta_mrt<UP>(G, Ss, Zs, U, K, red, tid);
    if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
    else sc = sqrtf(sys_rho2(d, sys) / (d.Es * t));
  } else {
    if (st == ST_OK) st = cta_gj_inverse<UP>(A, U, tid);
    if (st == ST_OK) {
      const float t = cta_trace_tgt<UP>(A, G, sys_kappa(d, sys), U, red, tid);
      if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
      else sc = sqrtf(sys_rho2(d, sys) / (d.Es * t));
    }
  }
  // a5 + a6: whiten, then x = scale H^H z over the resident antenna block
  if (st == ST_OK) {
    if (!d.mrt) cta_whiten<UP>(A, Ss, Zs, U, K, tid);
    __syncthreads();
    apply_rows<UP, 7>(Hs, nrows, Zs, K, sc, Xn, d.B, lo, tid);
  } else {
    zero_rows<UP>(nrows, K, Xn, d.B, lo, tid);
  }
  if (tid == 0) {
    report(in.status, sys, st);
    if (in.scale_out) in.scale_out[sys] = sc;
  }
  return true;
}

template <int UP>
__global__ void __launch_bounds__(NT) k_fused(InstDesc in, int maxrows) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + fused_bar_offset<UP>(maxrows, in.d.K));
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  uint32_t waits = 0;
  fused_system<UP>(in, blockIdx.x, smem_raw, maxrows, in.d.K, bar, waits);
}

// Persistent form over a work-item queue (one system per item).
template <int UP>
__global__ void __launch_bounds__(NT) k_batch_fused(const InstDesc *__restrict__ insts,
                                                    const WorkItem *__restrict__ items,
                                                    int n_items, int *__restrict__ queue,
                                                    int maxrows, int Kmax) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int next;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + fused_bar_offset<UP>(maxrows, Kmax));
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  uint32_t waits = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next = atomicAdd(queue, 1);
    __syncthreads();
    const int it = next;
    if (it >= n_items) break;
    const WorkItem w = items[it];
    if (!fused_system<UP>(insts[w.inst], w.sys0, smem_raw, maxrows, Kmax, bar, waits)) break;
  }
}

// Allow `bytes` of dynamic shared memory and ask for the largest shared
// carve-out, so that the SM is configured for as many CTAs as fit.
template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess || bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

constexpr size_t kSmemCap = 220 * 1024;

template <int UP>
size_t fused_bytes_t(int maxrows, int K) {
  return fused_bar_offset<UP>(maxrows, K) + 16;
}

template <int UP>
cudaError_t launch_gram_t(const SysDesc &d, const float2 *H, float2 *Gout, cudaStream_t s) {
  const int chunk = stream_chunk_rows(UP);
  const size_t bytes = (size_t)chunk * Geo<UP>::RS * 4 + (size_t)UP * UP * 8 + 16;
  cudaError_t e = set_smem(k_gram<UP>, bytes);
  if (e != cudaSuccess) return e;
  k_gram<UP><<<d.n_sc * d.nsys, NT, bytes, s>>>(d, H, Gout, chunk);
  return cudaGetLastError();
}

template <int UP>
cudaError_t launch_solve_t(const SysDesc &d, const float2 *Gin, const float2 *S, float2 *Z,
                           float *scale, int *status, cudaStream_t s) {
  const int total = d.n_sc * d.nsys;
  if constexpr (UP <= 32) {
    const size_t bytes = (size_t)(NT / 32) * ((size_t)UP * UP + (size_t)d.K * UP) * 8;
    cudaError_t e = set_smem(k_solve_warp<UP>, bytes);
    if (e != cudaSuccess) return e;
    k_solve_warp<UP><<<(total + NT / 32 - 1) / (NT / 32), NT, bytes, s>>>(d, Gin, S, Z, scale,
                                                                          status);
  } else {
    const size_t bytes = 2 * (size_t)UP * UP * 8 + 2 * (size_t)d.K * UP * 8 + 16 * 4;
    cudaError_t e = set_smem(k_solve_cta<UP>, bytes);
    if (e != cudaSuccess) return e;
    k_solve_cta<UP><<<total, NT, bytes, s>>>(d, Gin, S, Z, scale, status);
  }
  return cudaGetLastError();
}

template <int UP>
cudaError_t launch_apply_t(const SysDesc &d, const float2 *H, const float2 *Z, const float *scale,
                           float2 *X, cudaStream_t s) {
  const int chunk = stream_chunk_rows(UP);
  const size_t bytes = (size_t)chunk * Geo<UP>::RS * 4 + (size_t)d.K * UP * 8 + 16;
  cudaError_t e = set_smem(k_apply<UP>, bytes);
  if (e != cudaSuccess) return e;
  k_apply<UP><<<d.n_sc * d.nsys, NT, bytes, s>>>(d, H, Z, scale, X, chunk);
  return cudaGetLastError();
}

template <int UP>
cudaError_t launch_fused_t(const SysDesc &d, int maxrows, const float2 *H, const float2 *S,
                           float2 *X, int *status, float *scale_out, cudaStream_t s) {
  const size_t bytes = fused_bytes_t<UP>(maxrows, d.K);
  cudaError_t e = set_smem(k_fused<UP>, bytes);
  if (e != cudaSuccess) return e;
  InstDesc in{d, H, S, X, status, scale_out};
  k_fused<UP><<<d.n_sc * d.nsys, NT, bytes, s>>>(in, maxrows);
  return cudaGetLastError();
}

template <int UP>
cudaError_t launch_batch_fused_t(const InstDesc *insts, const WorkItem *items, int n_items,
                                 int *queue, int maxrows, int Kmax, int grid, cudaStream_t s) {
  const size_t bytes = fused_bytes_t<UP>(maxrows, Kmax);
  cudaError_t e = set_smem(k_batch_fused<UP>, bytes);
  if (e != cudaSuccess) return e;
  k_batch_fused<UP><<<grid, NT, bytes, s>>>(insts, items, n_items, queue, maxrows, Kmax);
  return cudaGetLastError();
}

template <int UP>
int fused_blocks_t(int maxrows, int Kmax) {
  const size_t bytes = fused_bytes_t<UP>(maxrows, Kmax);
  if (set_smem(k_batch_fused<UP>, bytes) != cudaSuccess) return 0;
  return resident_blocks((const void *)k_batch_fused<UP>, NT, bytes, 0);
}

}  // namespace

template <int UP>
cudaError_t Fp32Ops<UP>::gram(const SysDesc &d, const float2 *H, float2 *Gout, cudaStream_t s) {
  return launch_gram_t<UP>(d, H, Gout, s);
}
template <int UP>
cudaError_t Fp32Ops<UP>::solve(const SysDesc &d, const float2 *Gin, const float2 *S, float2 *Z,
                               float *scale, int *status, cudaStream_t s) {
  return launch_solve_t<UP>(d, Gin, S, Z, scale, status, s);
}
template <int UP>
cudaError_t Fp32Ops<UP>::apply(const SysDesc &d, const float2 *H, const float2 *Z,
                               const float *scale, float2 *X, cudaStream_t s) {
  return launch_apply_t<UP>(d, H, Z, scale, X, s);
}
template <int UP>
cudaError_t Fp32Ops<UP>::fused(const SysDesc &d, int maxrows, const float2 *H, const float2 *S,
                               float2 *X, int *status, float *scale_out, cudaStream_t s) {
  return launch_fused_t<UP>(d, maxrows, H, S, X, status, scale_out, s);
}
template <int UP>
cudaError_t Fp32Ops<UP>::batch_fused(const InstDesc *insts, const WorkItem *items, int n_items,
                                     int *queue, int maxrows, int Kmax, int grid,
                                     cudaStream_t s) {
  return launch_batch_fused_t<UP>(insts, items, n_items, queue, maxrows, Kmax, grid, s);
}
template <int UP>
int Fp32Ops<UP>::blocks(int maxrows, int Kmax) {
  return fused_blocks_t<UP>(maxrows, Kmax);
}
template <int UP>
size_t Fp32Ops<UP>::fused_bytes(int maxrows, int K) {
  return fused_bytes_t<UP>(maxrows, K);
}

}  // namespace dp
