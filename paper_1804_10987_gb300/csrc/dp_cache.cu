// dp_cache.cu -- the served path's per-channel solve cache.  Between channel
// updates (the serving pattern refreshes a cell's channel every few slots)
// everything that depends on H alone is computed once: the Gram, its
// inverse T = (G + kappa I)^{-1} (Thm. 1; per cluster for FD-WF, Sec. III-D)
// and the precoding factor (Lemma 1).  A request then only whitens its own
// symbols, z = T s, and applies x_c = scale H_c^H z.
//
// k_cache_invert  one CTA per system: G (from the FP32 Gram kernel) -> A ->
//                 T (register-blocked Gauss-Jordan), t, scale, status;
//                 MRT stores T = I and t = tr(G).
// k_cache_whiten  one CTA per system: T and s into shared memory, z = T s,
//                 the request's status and scale (0 for a failed system, so
//                 that the apply zeroes its rows).
// FD-WF clusters with B_c < U keep their per-request B_c x B_c kernel.
#include "dp_blocks.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

template <int UP>
__global__ void __launch_bounds__(NT) k_cache_invert(SysDesc d, const float2 *__restrict__ Gin,
                                                     float2 *__restrict__ Tout,
                                                     float *__restrict__ scale,
                                                     int *__restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, sys = blockIdx.x;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  int lo, hi;
  sys_rows(d, g, lo, hi);
  if (sys_is_small(d, hi - lo)) return;
  const int U = d.U;
  const float kappa = sys_kappa(d, sys), rho2 = sys_rho2(d, sys);
  float2 *G = reinterpret_cast<float2 *>(smem_raw);
  float2 *A = G + UP * UP;
  float2 *rc = A + UP * UP;  // [2][2][UP] row / column exchange
  float *red = reinterpret_cast<float *>(rc + 4 * UP);
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
    if (i == j) v.x += kappa;
    A[e] = v;
  }
  fin = __syncthreads_and(fin) != 0;
  int st = fin ? ST_OK : ST_NONFINITE;
  float sc = 0.f;
  if (st == ST_OK && d.mrt) {  // MRT: T = I, t = tr(G)
    float v = 0.f;
    for (int i = tid; i < U; i += NT) v += G[i * UP + i].x;
    const float t = cta_sum(v, red, tid);
    if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
    else sc = sqrtf(rho2 / (d.Es * t));
    for (int e = tid; e < UP * UP; e += NT)
      A[e] = (e / UP == e % UP) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    __syncthreads();
  } else if (st == ST_OK) {
    st = cta_gj_inverse_reg<UP>(A, U, tid, rc);
    if (st == ST_OK) {
      const float t = cta_trace_tgt<UP>(A, G, kappa, U, red, tid);
      if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
      else sc = sqrtf(rho2 / (d.Es * t));
    }
  }
  float2 *tdst = Tout + (size_t)sys * U * U;
  for (int e = tid; e < U * U; e += NT) {
    const int i = e / U, j = e - i * U;
    tdst[e] = (st == ST_OK) ? A[i * UP + j] : make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    scale[sys] = (st == ST_OK) ? sc : 0.f;
    status[sys] = st;
  }
}

template <int UP>
__global__ void __launch_bounds__(NT) k_cache_whiten(SysDesc d, const float2 *__restrict__ T,
                                                     const float *__restrict__ cscale,
                                                     const int *__restrict__ cstatus,
                                                     const float2 *__restrict__ S,
                                                     float2 *__restrict__ Z,
                                                     float *__restrict__ rscale,
                                                     int *__restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, sys = blockIdx.x;
  const int n = sys / d.nsys, g = sys - n * d.nsys;
  int lo, hi;
  sys_rows(d, g, lo, hi);
  if (sys_is_small(d, hi - lo)) return;
  const int U = d.U, K = d.K;
  float2 *Ts = reinterpret_cast<float2 *>(smem_raw);
  float2 *Ss = Ts + UP * UP;
  float2 *Zs = Ss + K * UP;
  int st = __ldg(cstatus + sys);
  const float2 *tsrc = T + (size_t)sys * U * U;
  for (int e = tid; e < UP * UP; e += NT) {
    const int i = e / UP, j = e - i * UP;
    Ts[e] = (i < U && j < U) ? __ldg(tsrc + i * U + j) : make_float2(0.f, 0.f);
  }
  const bool sfin = load_symbols<UP>(S + (size_t)n * K * U, Ss, U, K, tid);
  if (st == ST_OK && !sfin) st = ST_NONFINITE;
  if (st == ST_OK) cta_whiten<UP>(Ts, Ss, Zs, U, K, tid);
  __syncthreads();
  float2 *zdst = Z + (size_t)sys * K * U;
  for (int e = tid; e < K * U; e += NT) {
    const int k = e / U, i = e - k * U;
    zdst[e] = (st == ST_OK) ? Zs[k * UP + i] : make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    rscale[sys] = (st == ST_OK) ? __ldg(cscale + sys) : 0.f;
    status[sys] = st;
  }
}

template <typename KernelT>
cudaError_t smem_attr(KernelT k, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess || bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int UP>
cudaError_t launch_invert_t(const SysDesc &d, const float2 *G, float2 *T, float *scale,
                            int *status, cudaStream_t s) {
  const size_t bytes = 2 * (size_t)UP * UP * 8 + 4 * (size_t)UP * 8 + (NT / 32) * 4;
  cudaError_t e = smem_attr(k_cache_invert<UP>, bytes);
  if (e != cudaSuccess) return e;
  k_cache_invert<UP><<<d.n_sc * d.nsys, NT, bytes, s>>>(d, G, T, scale, status);
  return cudaGetLastError();
}

template <int UP>
cudaError_t launch_whiten_t(const SysDesc &d, const float2 *T, const float *cscale,
                            const int *cstatus, const float2 *S, float2 *Z, float *rscale,
                            int *status, cudaStream_t s) {
  const size_t bytes = (size_t)UP * UP * 8 + 2 * (size_t)d.K * UP * 8;
  cudaError_t e = smem_attr(k_cache_whiten<UP>, bytes);
  if (e != cudaSuccess) return e;
  k_cache_whiten<UP><<<d.n_sc * d.nsys, NT, bytes, s>>>(d, T, cscale, cstatus, S, Z, rscale,
                                                        status);
  return cudaGetLastError();
}

#define DP_CACHE_DISPATCH(UPV, CALL)                  \
  switch (UPV) {                                      \
    case 8: { constexpr int UPC = 8; return CALL; }   \
    case 16: { constexpr int UPC = 16; return CALL; } \
    case 24: { constexpr int UPC = 24; return CALL; } \
    case 32: { constexpr int UPC = 32; return CALL; } \
    case 40: { constexpr int UPC = 40; return CALL; } \
    case 48: { constexpr int UPC = 48; return CALL; } \
    case 56: { constexpr int UPC = 56; return CALL; } \
    case 64: { constexpr int UPC = 64; return CALL; } \
    default: return cudaErrorInvalidValue;            \
  }

}  // namespace

cudaError_t launch_cache_invert(const SysDesc &d, int UP, const float2 *G, float2 *T, float *scale,
                                int *status, cudaStream_t s) {
  if (d.n_sc * d.nsys == 0) return cudaSuccess;
  DP_CACHE_DISPATCH(UP, (launch_invert_t<UPC>(d, G, T, scale, status, s)));
}

cudaError_t launch_cache_whiten(const SysDesc &d, int UP, const float2 *T, const float *cscale,
                                const int *cstatus, const float2 *S, float2 *Z, float *rscale,
                                int *status, cudaStream_t s) {
  if (d.n_sc * d.nsys == 0) return cudaSuccess;
  DP_CACHE_DISPATCH(UP,
                    (launch_whiten_t<UPC>(d, T, cscale, cstatus, S, Z, rscale, status, s)));
}

}  // namespace dp
