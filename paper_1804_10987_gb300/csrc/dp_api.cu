// dp_api.cu -- the C ABI declared in include/dprecode.h: plan validation and
// workspace, argument checks, and the enqueueing of the kernels on the plan's
// stream.  No arithmetic of the method happens on the host.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/dprecode.h"
#include "dp_internal.h"

struct dp_plan {
  dp_plan_desc d{};
  std::vector<int> sizes, off;
  int device = 0;
  cudaStream_t stream = nullptr;
  int UP = 8;
  int maxrows_sys = 0;     // antenna rows of the largest system (B, or max B_c in FD)
  bool fused_fits = false;
  int *d_off = nullptr;     // [C + 1]
  int *d_status = nullptr;  // [n_sc * nsys]: status of every system of the last call
  int nsys = 1;
  // FD-WF clusters with B_c < U (<= 32) run the B_c x B_c form
  bool has_small = false, all_small = false;
  int bcp = 0;
  // workspace of the streaming (unfused) form of dp_precode
  float2 *w_G = nullptr;
  float2 *w_Z = nullptr;
  float *w_scale = nullptr;
};

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
// A device array argument: non-NULL and 16-byte aligned, or an empty array
// (then any value, NULL included, is accepted and never dereferenced).
bool arg_ok(const void *p, bool empty) { return empty || (p != nullptr && aligned16(p)); }

dp::SysDesc make_sys(const dp_plan *p, bool per_cluster, const void *H) {
  dp::SysDesc s{};
  s.U = p->d.U;
  s.B = p->d.B;
  s.K = p->d.K;
  s.n_sc = p->d.n_sc;
  s.nsys = per_cluster ? p->d.C : 1;
  s.off = p->d_off;
  s.Es = p->d.Es;
  const double U = p->d.U, N0 = p->d.N0, rho2 = p->d.rho2, C = p->d.C;
  switch (p->d.mode) {
    case DP_ZF:
      s.kappa = 0.f;
      s.rho2_sys = p->d.rho2;
      break;
    case DP_WF:
      s.kappa = (float)(U * N0 / rho2);  // Thm. 1
      s.rho2_sys = p->d.rho2;
      break;
    case DP_FDWF:
      s.kappa = (float)(p->d.tau * U * N0 / (rho2 / C));  // Eq. (16), rho_c^2 = rho^2 / C
      s.rho2_sys = (float)(rho2 / C);
      break;
  }
  s.tma_ok = (p->d.U % 2 == 0) && (H == nullptr || aligned16(H));
  return s;
}

dp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DP_OK : DP_ERR_CUDA; }

dp_status ensure_workspace(dp_plan *p) {
  if (p->w_G) return DP_OK;
  const int nsys = (p->d.mode == DP_FDWF) ? p->d.C : 1;
  const size_t ns = (size_t)p->d.n_sc * nsys;
  if (ns == 0) return DP_OK;
  if (cudaMalloc(&p->w_G, ns * p->d.U * p->d.U * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&p->w_Z, ns * (p->d.K ? p->d.K : 1) * p->d.U * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&p->w_scale, ns * sizeof(float)) != cudaSuccess) {
    cudaFree(p->w_G);
    cudaFree(p->w_Z);
    cudaFree(p->w_scale);
    p->w_G = p->w_Z = nullptr;
    p->w_scale = nullptr;
    cudaGetLastError();
    return DP_ERR_OOM;
  }
  return DP_OK;
}

size_t status_len(const dp_plan_desc &d) {
  const size_t nsys = (d.mode == DP_FDWF) ? d.C : 1;
  const size_t n = (size_t)d.n_sc * nsys;
  return n > 0 ? n : 1;
}

dp_status set_device(const dp_plan *p) {
  return cuda_status(cudaSetDevice(p->device));
}

}  // namespace

extern "C" {

const char *dp_version(void) { return "dprecode 0.1 (sm_103a)"; }

const char *dp_status_string(dp_status s) {
  switch (s) {
    case DP_OK: return "ok";
    case DP_ERR_INVALID_ARG: return "invalid argument";
    case DP_ERR_PARTITION: return "invalid cluster partition";
    case DP_ERR_UNSUPPORTED: return "unsupported configuration";
    case DP_ERR_OOM: return "device out of memory";
    case DP_ERR_CUDA: return "CUDA error";
    case DP_ERR_NOT_PD: return "matrix not positive definite";
    case DP_ERR_NONFINITE: return "non-finite input";
    case DP_ERR_TIMEOUT: return "on-device wait timed out";
  }
  return "unknown status";
}

dp_status dp_plan_create(const dp_plan_desc *desc, dp_stream_t stream, dp_plan_t *out) {
  if (!out) return DP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return DP_ERR_INVALID_ARG;
  const dp_plan_desc &d = *desc;
  if (d.U < 1 || d.U > 64 || d.B < 1 || d.B > 4096 || d.C < 1 || d.C > d.B || d.n_sc < 0 ||
      d.K < 0 || d.K > 64)
    return DP_ERR_INVALID_ARG;
  if (d.mode != DP_ZF && d.mode != DP_WF && d.mode != DP_FDWF) return DP_ERR_INVALID_ARG;
  if (d.prec != DP_FP32 && d.prec != DP_BF16 && d.prec != DP_FP16) return DP_ERR_INVALID_ARG;
  if (!(d.rho2 > 0.f) || !std::isfinite(d.rho2) || !(d.Es > 0.f) || !std::isfinite(d.Es) ||
      !(d.N0 >= 0.f) || !std::isfinite(d.N0) || !(d.tau >= 0.f) || !std::isfinite(d.tau))
    return DP_ERR_INVALID_ARG;
  if (d.refine != 0 && d.refine != 1) return DP_ERR_INVALID_ARG;
  // The tensor-core path covers up to 64 users; refinement is not built.
  if (d.prec != DP_FP32 && !dp::tc_supported(dp::padded_users(d.U))) return DP_ERR_UNSUPPORTED;
  if (d.refine != 0) return DP_ERR_UNSUPPORTED;

  std::vector<int> sizes(d.C);
  if (d.cluster_sizes) {
    long long sum = 0;
    for (int c = 0; c < d.C; ++c) {
      if (d.cluster_sizes[c] < 1) return DP_ERR_PARTITION;
      sizes[c] = d.cluster_sizes[c];
      sum += sizes[c];
    }
    if (sum != d.B) return DP_ERR_PARTITION;
  } else {
    if (d.B % d.C != 0) return DP_ERR_PARTITION;
    for (int c = 0; c < d.C; ++c) sizes[c] = d.B / d.C;
  }
  const double kappa_fd = (double)d.tau * d.U * d.N0 * d.C / d.rho2;
  int maxbc = 0;
  for (int c = 0; c < d.C; ++c) maxbc = sizes[c] > maxbc ? sizes[c] : maxbc;
  int minbc = d.B;
  for (int c = 0; c < d.C; ++c) minbc = sizes[c] < minbc ? sizes[c] : minbc;
  // Systems with kappa = 0 are singular when they have fewer antennas than users.
  if ((d.mode == DP_ZF || (d.mode == DP_WF && d.N0 == 0.f)) && d.B < d.U)
    return DP_ERR_UNSUPPORTED;
  if (d.mode == DP_FDWF && kappa_fd == 0.0 && minbc < d.U) return DP_ERR_UNSUPPORTED;

  dp_plan *p = new (std::nothrow) dp_plan;
  if (!p) return DP_ERR_OOM;
  p->d = d;
  p->sizes = sizes;
  p->d.cluster_sizes = nullptr;  // the copy lives in p->sizes
  p->off.resize(d.C + 1);
  p->off[0] = 0;
  for (int c = 0; c < d.C; ++c) p->off[c + 1] = p->off[c] + sizes[c];
  p->stream = reinterpret_cast<cudaStream_t>(stream);
  p->UP = dp::padded_users(d.U);
  p->maxrows_sys = (d.mode == DP_FDWF) ? maxbc : d.B;
  p->nsys = (d.mode == DP_FDWF) ? d.C : 1;
  if (d.mode == DP_FDWF) {
    int maxsmall = 0, nsmall = 0;
    for (int c = 0; c < d.C; ++c)
      if (sizes[c] < d.U && sizes[c] <= 32) {
        ++nsmall;
        maxsmall = sizes[c] > maxsmall ? sizes[c] : maxsmall;
      }
    p->has_small = nsmall > 0;
    p->all_small = nsmall == d.C;
    p->bcp = dp::fd_small_bcp(maxsmall);
  }
  p->fused_fits = dp::fused_smem_bytes(p->UP, p->maxrows_sys, d.K) != 0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return DP_ERR_CUDA;
  }
  if (cudaMalloc(&p->d_off, sizeof(int) * (d.C + 1)) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(int) * status_len(d)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->d_off);
    delete p;
    return DP_ERR_OOM;
  }
  if (cudaMemcpy(p->d_off, p->off.data(), sizeof(int) * (d.C + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(p->d_status, 0, sizeof(int) * status_len(d)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->d_off);
    cudaFree(p->d_status);
    delete p;
    return DP_ERR_CUDA;
  }
  *out = p;
  return DP_OK;
}

dp_status dp_plan_destroy(dp_plan_t p) {
  if (!p) return DP_ERR_INVALID_ARG;
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  cudaFree(p->d_off);
  cudaFree(p->d_status);
  cudaFree(p->w_G);
  cudaFree(p->w_Z);
  cudaFree(p->w_scale);
  cudaGetLastError();
  delete p;
  return DP_OK;
}

dp_status dp_plan_set_stream(dp_plan_t p, dp_stream_t stream) {
  if (!p) return DP_ERR_INVALID_ARG;
  p->stream = reinterpret_cast<cudaStream_t>(stream);
  return DP_OK;
}

dp_status dp_gram_local(dp_plan_t p, const void *H, void *Gloc) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (p->d.n_sc == 0) return DP_OK;
  if (!arg_ok(H, false) || !arg_ok(Gloc, false)) return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  dp::SysDesc sd = make_sys(p, true, H);
  return cuda_status(dp::launch_gram(sd, p->UP, static_cast<const float2 *>(H),
                                     static_cast<float2 *>(Gloc), p->stream));
}

dp_status dp_gram_reduce(dp_plan_t p, const void *Gloc, void *G) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (p->d.n_sc == 0) return DP_OK;
  if (!arg_ok(Gloc, false) || !arg_ok(G, false)) return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  const size_t per = (size_t)p->d.n_sc * p->d.U * p->d.U;
  return cuda_status(dp::launch_reduce(static_cast<const float2 *>(Gloc),
                                       static_cast<float2 *>(G), p->d.C, per, p->stream));
}

dp_status dp_solve(dp_plan_t p, const void *G_or_Gloc, const void *S, void *Z, float *scale) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (p->d.n_sc == 0) return DP_OK;
  const bool k0 = p->d.K == 0;
  if (!arg_ok(G_or_Gloc, false) || !arg_ok(S, k0) || !arg_ok(Z, k0) || !arg_ok(scale, false))
    return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  dp::SysDesc sd = make_sys(p, p->d.mode == DP_FDWF, nullptr);
  cudaError_t e = dp::launch_solve(sd, p->UP, static_cast<const float2 *>(G_or_Gloc),
                         static_cast<const float2 *>(S), static_cast<float2 *>(Z), scale,
                         p->d_status, p->stream);
  return cuda_status(e);
}

dp_status dp_precode_apply(dp_plan_t p, const void *H, const void *Z, const float *scale,
                           void *X) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (p->d.n_sc == 0 || p->d.K == 0) return DP_OK;
  if (!arg_ok(H, false) || !arg_ok(Z, false) || !arg_ok(scale, false) || !arg_ok(X, false))
    return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  dp::SysDesc sd = make_sys(p, p->d.mode == DP_FDWF, H);
  return cuda_status(dp::launch_apply(sd, p->UP, static_cast<const float2 *>(H),
                                      static_cast<const float2 *>(Z), scale,
                                      static_cast<float2 *>(X), p->stream));
}

dp_status dp_precode(dp_plan_t p, const void *H, const void *S, void *X) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (p->d.n_sc == 0) return DP_OK;
  const bool k0 = p->d.K == 0;
  if (!arg_ok(H, false) || !arg_ok(S, k0) || !arg_ok(X, k0)) return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  const bool fd = p->d.mode == DP_FDWF;
  dp::SysDesc sd = make_sys(p, fd, H);
  const float2 *h = static_cast<const float2 *>(H);
  const float2 *sy = static_cast<const float2 *>(S);
  float2 *x = static_cast<float2 *>(X);
  cudaError_t e = cudaSuccess;
  if (p->has_small) {  // FD-WF clusters with B_c < U: the paper's B_c x B_c form
    sd.skip_small = 1;
    e = dp::launch_fd_small(dp::InstDesc{sd, h, sy, x, p->d_status, nullptr}, p->bcp, p->stream);
    if (e != cudaSuccess || p->all_small) return cuda_status(e);
  }
  if (p->d.prec != DP_FP32 && dp::pipe_tc_supported(sd, p->UP))
    return cuda_status(dp::launch_pipe_tc(sd, p->UP, p->d.prec == DP_BF16, h, sy, x, p->d_status,
                                          nullptr, p->stream));
  if (p->d.prec != DP_FP32)
    return cuda_status(dp::launch_fused_tc(sd, p->UP, p->d.prec == DP_BF16, h, sy, x, p->d_status,
                                           nullptr, p->stream));
  if (p->fused_fits)
    return cuda_status(
        dp::launch_fused(sd, p->UP, p->maxrows_sys, h, sy, x, p->d_status, nullptr, p->stream));
  // Streaming form: Gram (cluster sum fused for WF/ZF), solve, apply.
  if (dp_status s = ensure_workspace(p)) return s;
  e = dp::launch_gram(sd, p->UP, h, p->w_G, p->stream);
  if (e == cudaSuccess)
    e = dp::launch_solve(sd, p->UP, p->w_G, sy, p->w_Z, p->w_scale, p->d_status, p->stream);
  if (e == cudaSuccess) e = dp::launch_apply(sd, p->UP, h, p->w_Z, p->w_scale, x, p->stream);
  return cuda_status(e);
}

dp_status dp_status_get(dp_plan_t p, int *host_status) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return DP_ERR_CUDA;
  if (p->d.n_sc == 0) return DP_OK;
  std::vector<int> sys((size_t)p->d.n_sc * p->nsys);
  if (cudaMemcpy(sys.data(), p->d_status, sizeof(int) * sys.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return DP_ERR_CUDA;
  dp_status first = DP_OK;
  for (int n = 0; n < p->d.n_sc; ++n) {
    int worst = 0;  // fold the systems (clusters) of the subcarrier
    for (int g = 0; g < p->nsys; ++g) {
      const int v = sys[(size_t)n * p->nsys + g];
      worst = v > worst ? v : worst;
    }
    if (host_status) host_status[n] = worst;
    if (first == DP_OK && worst != 0) first = static_cast<dp_status>(worst);
  }
  return first;
}

}  // extern "C"
