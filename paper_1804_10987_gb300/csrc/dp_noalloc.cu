// dp_noalloc.cu -- dp_precode_noalloc: the streaming precoder (Gram, solve,
// apply) for callers that must not allocate device memory.
//
// Its workspace (cluster offsets, per-system status, Gram matrices, whitened
// vectors and scales) lives in one file-scope device array of fixed size
// instead of a plan's cudaMalloc'd buffers.  Every GPU that loads this library
// reserves the array until the process exits.  All calls on a device share
// it: a call overwrites everything it reads before reading it, so nothing has
// to start at zero, but two calls whose work overlaps on the GPU (different
// streams, or different host threads without ordering) race on it.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/dprecode.h"
#include "dp_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(DP_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of g_scratch on device dev (the current device).  In host
// code the symbol names a host-side stand-in, so the address is looked up
// once per device with that device current and cached for the life of the
// process (keyed on the device ordinal only: a cudaDeviceReset, which gives
// the device a new context, leaves the cached address stale).
dp_status scratch_on(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return DP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return DP_ERR_CUDA;
    }
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return DP_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Cluster offsets passed by value (kernel parameters): the device copy is
// written by a kernel, so no host buffer (pageable or pinned) is involved.
constexpr int kOffChunk = 512;
struct OffChunk {
  int first, n;
  int v[kOffChunk];
};
__global__ void k_fill_offsets(OffChunk c, int *dst) {
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) dst[c.first + i] = c.v[i];
}
bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" dp_status dp_precode_noalloc(const dp_plan_desc *desc, dp_stream_t stream,
                                        const void *H, const void *S, void *X,
                                        int *host_status) {
  if (!desc) return DP_ERR_INVALID_ARG;
  const dp_plan_desc &d = *desc;
  if (d.U < 1 || d.U > 64 || d.B < 1 || d.B > 4096 || d.C < 1 || d.C > d.B || d.n_sc < 0 ||
      d.K < 0 || d.K > 64)
    return DP_ERR_INVALID_ARG;
  if (d.mode != DP_ZF && d.mode != DP_WF && d.mode != DP_FDWF && d.mode != DP_MRT) return DP_ERR_INVALID_ARG;
  if (d.prec != DP_FP32 && d.prec != DP_BF16 && d.prec != DP_FP16) return DP_ERR_INVALID_ARG;
  if (!(d.rho2 > 0.f) || !std::isfinite(d.rho2) || !(d.Es > 0.f) || !std::isfinite(d.Es) ||
      !(d.N0 >= 0.f) || !std::isfinite(d.N0) || !(d.tau >= 0.f) || !std::isfinite(d.tau) ||
      (d.refine != 0 && d.refine != 1))
    return DP_ERR_INVALID_ARG;
  if (d.prec != DP_FP32 || d.refine != 0) return DP_ERR_UNSUPPORTED;
  {
    std::vector<float2> ckr;
    if (!dp::cluster_power_table(d.mode == DP_FDWF, d.cluster_power, d.C, d.rho2, d.tau, d.U,
                                 d.N0, ckr))
      return DP_ERR_INVALID_ARG;
    if (!ckr.empty()) return DP_ERR_UNSUPPORTED;  // per-cluster power: use a plan
  }

  std::vector<int> off(d.C + 1, 0);
  for (int c = 0; c < d.C; ++c) {
    int bc;
    if (d.cluster_sizes) {
      bc = d.cluster_sizes[c];
    } else {
      if (d.B % d.C != 0) return DP_ERR_PARTITION;
      bc = d.B / d.C;
    }
    if (bc < 1) return DP_ERR_PARTITION;
    off[c + 1] = off[c] + bc;
  }
  if (off[d.C] != d.B) return DP_ERR_PARTITION;
  int minbc = d.B;
  for (int c = 0; c < d.C; ++c) minbc = std::min(minbc, off[c + 1] - off[c]);
  const bool fd = d.mode == DP_FDWF;
  const double kappa_fd = (double)d.tau * d.U * d.N0 * d.C / d.rho2;
  if ((d.mode == DP_ZF || (d.mode == DP_WF && d.N0 == 0.f)) && d.B < d.U)
    return DP_ERR_UNSUPPORTED;
  if (fd && kappa_fd == 0.0 && minbc < d.U) return DP_ERR_UNSUPPORTED;

  // Workspace carved from the static array; sizes beyond it are refused
  // before anything is enqueued.
  const int nsys = fd ? d.C : 1;
  const size_t ns = (size_t)d.n_sc * nsys;
  const size_t b_off = up256(sizeof(int) * (d.C + 1));
  const size_t b_st = up256(sizeof(int) * (ns > 0 ? ns : 1));
  const size_t b_G = up256(sizeof(float2) * ns * d.U * d.U);
  const size_t b_Z = up256(sizeof(float2) * ns * (size_t)d.K * d.U);
  const size_t b_sc = up256(sizeof(float) * (ns > 0 ? ns : 1));
  if (b_off + b_st + b_G + b_Z + b_sc > kScratchBytes) return DP_ERR_UNSUPPORTED;

  if (d.n_sc == 0) return DP_OK;
  const bool k0 = d.K == 0;
  if (!H || !a16(H) || (!k0 && (!S || !a16(S) || !X || !a16(X)))) return DP_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  unsigned char *base = nullptr;
  if (dp_status s = scratch_on(dev, &base)) return s;
  int *w_off = reinterpret_cast<int *>(base);
  int *w_st = reinterpret_cast<int *>(base + b_off);
  float2 *w_G = reinterpret_cast<float2 *>(base + b_off + b_st);
  float2 *w_Z = reinterpret_cast<float2 *>(base + b_off + b_st + b_G);
  float *w_sc = reinterpret_cast<float *>(base + b_off + b_st + b_G + b_Z);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  cudaError_t e = cudaSuccess;
  for (int first = 0; first <= d.C && e == cudaSuccess; first += kOffChunk) {
    OffChunk c{};
    c.first = first;
    c.n = std::min(kOffChunk, d.C + 1 - first);
    for (int i = 0; i < c.n; ++i) c.v[i] = off[first + i];
    k_fill_offsets<<<1, 128, 0, st>>>(c, w_off);
    e = cudaGetLastError();
  }

  dp::SysDesc sd{};
  sd.U = d.U;
  sd.B = d.B;
  sd.K = d.K;
  sd.n_sc = d.n_sc;
  sd.nsys = nsys;
  sd.off = w_off;
  sd.Es = d.Es;
  const double U = d.U, N0 = d.N0, rho2 = d.rho2, C = d.C;
  if (d.mode == DP_ZF || d.mode == DP_MRT) {
    sd.kappa = 0.f;
    sd.rho2_sys = d.rho2;
  } else if (d.mode == DP_WF) {
    sd.kappa = (float)(U * N0 / rho2);
    sd.rho2_sys = d.rho2;
  } else {
    sd.kappa = (float)(d.tau * U * N0 / (rho2 / C));
    sd.rho2_sys = (float)(rho2 / C);
  }
  sd.tma_ok = (d.U % 2 == 0) && a16(H);
  sd.mrt = d.mode == DP_MRT;
  const int UP = dp::padded_users(d.U);
  const float2 *h = static_cast<const float2 *>(H);
  // FD-WF clusters with fewer antennas than users (at most 32) take the
  // paper's B_c x B_c form, as in dp_precode; it needs no workspace
  int maxsmall = 0, nsmall = 0;
  if (fd)
    for (int c = 0; c < d.C; ++c) {
      const int bc = off[c + 1] - off[c];
      if (bc < d.U && bc <= 32) {
        ++nsmall;
        maxsmall = std::max(maxsmall, bc);
      }
    }
  if (nsmall > 0) {
    sd.skip_small = 1;
    if (e == cudaSuccess)
      e = dp::launch_fd_small(dp::InstDesc{sd, h, static_cast<const float2 *>(S),
                                           static_cast<float2 *>(X), w_st, nullptr},
                              dp::fd_small_bcp(maxsmall), st);
  }
  if (nsmall < (fd ? d.C : 1)) {
    if (e == cudaSuccess) e = dp::launch_gram(sd, UP, h, w_G, st);
    if (e == cudaSuccess)
      e = dp::launch_solve(sd, UP, w_G, static_cast<const float2 *>(S), w_Z, w_sc, w_st, st);
    if (e == cudaSuccess && !k0)
      e = dp::launch_apply(sd, UP, h, w_Z, w_sc, static_cast<float2 *>(X), st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  if (!host_status) return DP_OK;

  std::vector<int> sys(ns);
  if (cudaMemcpyAsync(sys.data(), w_st, sizeof(int) * ns, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  dp_status first = DP_OK;
  for (int n = 0; n < d.n_sc; ++n) {
    int worst = 0;
    for (int g = 0; g < nsys; ++g) worst = std::max(worst, sys[(size_t)n * nsys + g]);
    host_status[n] = worst;
    if (first == DP_OK && worst != 0) first = static_cast<dp_status>(worst);
  }
  return first;
}
