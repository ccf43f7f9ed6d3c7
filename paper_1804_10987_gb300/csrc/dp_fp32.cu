// dp_fp32.cu -- dispatch of the FP32 path's launchers on the padded user
// count (the kernels themselves: dp_fp32_impl.cuh, instantiated per user
// count in dp_fp32_u*.cu so that they compile in parallel), and the cluster
// sum k_reduce (step a2, Fig. 1(a) adder tree).
#include "dp_internal.h"

namespace dp {

extern template struct Fp32Ops<8>;
extern template struct Fp32Ops<16>;
extern template struct Fp32Ops<24>;
extern template struct Fp32Ops<32>;
extern template struct Fp32Ops<40>;
extern template struct Fp32Ops<48>;
extern template struct Fp32Ops<56>;
extern template struct Fp32Ops<64>;

namespace {

// a2: G = sum_c G_c in cluster order
__global__ void k_reduce(const float2 *__restrict__ Gloc, float2 *__restrict__ G, int C,
                         size_t per) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < per;
       e += (size_t)gridDim.x * blockDim.x) {
    float2 acc = __ldg(Gloc + e);
    for (int c = 1; c < C; ++c) acc = cadd(acc, __ldg(Gloc + (size_t)c * per + e));
    G[e] = acc;
  }
}

constexpr size_t kSmemCap = 220 * 1024;

#define DP_DISPATCH_UP(UPV, CALL, FAIL)                 \
  switch (UPV) {                                        \
    case 8: { using O = Fp32Ops<8>; return CALL; }      \
    case 16: { using O = Fp32Ops<16>; return CALL; }    \
    case 24: { using O = Fp32Ops<24>; return CALL; }    \
    case 32: { using O = Fp32Ops<32>; return CALL; }    \
    case 40: { using O = Fp32Ops<40>; return CALL; }    \
    case 48: { using O = Fp32Ops<48>; return CALL; }    \
    case 56: { using O = Fp32Ops<56>; return CALL; }    \
    case 64: { using O = Fp32Ops<64>; return CALL; }    \
    default: return FAIL;                               \
  }

size_t fused_bytes_any(int UP, int maxrows, int K) {
  DP_DISPATCH_UP(UP, O::fused_bytes(maxrows, K), size_t(0));
}

}  // namespace

int stream_chunk_rows(int UP) { return UP <= 32 ? 128 : 64; }

size_t fused_smem_bytes(int UP, int maxrows, int K) {
  const size_t b = fused_bytes_any(UP, maxrows, K);
  return b <= kSmemCap ? b : 0;
}

cudaError_t launch_gram(const SysDesc &d, int UP, const float2 *H, float2 *Gout, cudaStream_t s) {
  DP_DISPATCH_UP(UP, O::gram(d, H, Gout, s), cudaErrorInvalidValue);
}

cudaError_t launch_reduce(const float2 *Gloc, float2 *G, int C, size_t per, cudaStream_t s) {
  if (per == 0) return cudaSuccess;
  const int threads = 256;
  size_t blocks = (per + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_reduce<<<(unsigned)blocks, threads, 0, s>>>(Gloc, G, C, per);
  return cudaGetLastError();
}

cudaError_t launch_solve(const SysDesc &d, int UP, const float2 *Gin, const float2 *S, float2 *Z,
                         float *scale, int *status, cudaStream_t s) {
  DP_DISPATCH_UP(UP, O::solve(d, Gin, S, Z, scale, status, s), cudaErrorInvalidValue);
}

cudaError_t launch_apply(const SysDesc &d, int UP, const float2 *H, const float2 *Z,
                         const float *scale, float2 *X, cudaStream_t s) {
  DP_DISPATCH_UP(UP, O::apply(d, H, Z, scale, X, s), cudaErrorInvalidValue);
}

cudaError_t launch_fused(const SysDesc &d, int UP, int maxrows, const float2 *H, const float2 *S,
                         float2 *X, int *status, float *scale_out, cudaStream_t s) {
  DP_DISPATCH_UP(UP, O::fused(d, maxrows, H, S, X, status, scale_out, s), cudaErrorInvalidValue);
}

cudaError_t launch_batch_fused(int UP, const InstDesc *insts, const WorkItem *items, int n_items,
                               int *queue, int maxrows, int Kmax, int grid, cudaStream_t s) {
  DP_DISPATCH_UP(UP, O::batch_fused(insts, items, n_items, queue, maxrows, Kmax, grid, s),
                 cudaErrorInvalidValue);
}

int fused_max_blocks_per_sm(int UP, int maxrows, int Kmax) {
  DP_DISPATCH_UP(UP, O::blocks(maxrows, Kmax), 0);
}

}  // namespace dp
