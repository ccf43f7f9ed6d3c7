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
  int *d_fix = nullptr;     // reduced precision: groups to redo (list, then its count)
  int n_fix = 0;            // entries of the list
  int n_sm = 0;             // SMs of the plan's device
  float2 *d_ckr = nullptr;  // FD-WF with per-cluster power: (kappa_c, rho_c^2) [C]
  int nsys = 1;
  int dbg_stall_us = 0;  // failure injection for tests (dp_debug_stall)
  // FD-WF clusters with B_c < U (<= 32) run the B_c x B_c form
  bool has_small = false, all_small = false;
  int bcp = 0;
  // workspace of the streaming (unfused) form of dp_precode
  float2 *w_G = nullptr;
  float2 *w_Z = nullptr;
  float *w_scale = nullptr;
  // dp_precode_host: 3-deep ring of device staging chunks, copy streams and
  // the events that order them (allocated on first use)
  static constexpr int NSTAGE = 3;
  int hp_chunk = 0;
  float2 *hp_H = nullptr, *hp_S = nullptr, *hp_X = nullptr;
  cudaStream_t hp_up = nullptr, hp_down = nullptr;
  cudaEvent_t hp_start = nullptr;
  cudaEvent_t hp_up_done[NSTAGE] = {}, hp_calc_done[NSTAGE] = {}, hp_down_done[NSTAGE] = {};
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
    case DP_MRT:
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
  s.refine = dp::refine_mode(p->d.refine, p->d.prec == DP_FP32, p->d.mode == DP_MRT);
  s.mrt = p->d.mode == DP_MRT;
  s.dbg_stall_us = p->dbg_stall_us;
  s.ckr = (p->d.mode == DP_FDWF && per_cluster) ? p->d_ckr : nullptr;
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

void free_host_pipeline(dp_plan *p) {
  if (p->hp_up) cudaStreamSynchronize(p->hp_up);
  if (p->hp_down) cudaStreamSynchronize(p->hp_down);
  cudaFree(p->hp_H);
  cudaFree(p->hp_S);
  cudaFree(p->hp_X);
  p->hp_H = p->hp_S = p->hp_X = nullptr;
  for (int b = 0; b < dp_plan::NSTAGE; ++b) {
    if (p->hp_up_done[b]) cudaEventDestroy(p->hp_up_done[b]);
    if (p->hp_calc_done[b]) cudaEventDestroy(p->hp_calc_done[b]);
    if (p->hp_down_done[b]) cudaEventDestroy(p->hp_down_done[b]);
    p->hp_up_done[b] = p->hp_calc_done[b] = p->hp_down_done[b] = nullptr;
  }
  if (p->hp_start) cudaEventDestroy(p->hp_start);
  if (p->hp_up) cudaStreamDestroy(p->hp_up);
  if (p->hp_down) cudaStreamDestroy(p->hp_down);
  p->hp_start = nullptr;
  p->hp_up = p->hp_down = nullptr;
  p->hp_chunk = 0;
  cudaGetLastError();
}

// Staging ring for chunks of `chunk` subcarriers (kept if already as large).
dp_status ensure_host_pipeline(dp_plan *p, int chunk) {
  if (p->hp_chunk >= chunk) return DP_OK;
  if (p->hp_chunk) {  // earlier calls' copies and kernels finish first
    cudaStreamSynchronize(p->stream);
    free_host_pipeline(p);
  }
  const size_t n = (size_t)dp_plan::NSTAGE * chunk;
  const size_t hb = (size_t)p->d.B * p->d.U, sb = (size_t)p->d.K * p->d.U,
               xb = (size_t)p->d.K * p->d.B;
  bool ok = cudaMalloc(&p->hp_H, n * hb * sizeof(float2)) == cudaSuccess &&
            (sb == 0 || cudaMalloc(&p->hp_S, n * sb * sizeof(float2)) == cudaSuccess) &&
            (xb == 0 || cudaMalloc(&p->hp_X, n * xb * sizeof(float2)) == cudaSuccess);
  ok = ok && cudaStreamCreateWithFlags(&p->hp_up, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&p->hp_down, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&p->hp_start, cudaEventDisableTiming) == cudaSuccess;
  for (int b = 0; ok && b < dp_plan::NSTAGE; ++b)
    ok = cudaEventCreateWithFlags(&p->hp_up_done[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->hp_calc_done[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->hp_down_done[b], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    free_host_pipeline(p);
    return DP_ERR_OOM;
  }
  p->hp_chunk = chunk;
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
  if (d.mode != DP_ZF && d.mode != DP_WF && d.mode != DP_FDWF && d.mode != DP_MRT)
    return DP_ERR_INVALID_ARG;
  if (d.prec != DP_FP32 && d.prec != DP_BF16 && d.prec != DP_FP16) return DP_ERR_INVALID_ARG;
  if (!(d.rho2 > 0.f) || !std::isfinite(d.rho2) || !(d.Es > 0.f) || !std::isfinite(d.Es) ||
      !(d.N0 >= 0.f) || !std::isfinite(d.N0) || !(d.tau >= 0.f) || !std::isfinite(d.tau))
    return DP_ERR_INVALID_ARG;
  if (!dp::refine_valid(d.refine)) return DP_ERR_INVALID_ARG;
  std::vector<float2> ckr;  // per-cluster power (FD-WF)
  if (!dp::cluster_power_table(d.mode == DP_FDWF, d.cluster_power, d.C, d.rho2, d.tau, d.U,
                               d.N0, ckr))
    return DP_ERR_INVALID_ARG;
  // The tensor-core path covers up to 64 users.
  if (d.prec != DP_FP32 && !dp::tc_supported(dp::padded_users(d.U))) return DP_ERR_UNSUPPORTED;

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
  p->d.cluster_power = nullptr;  // the table goes to p->d_ckr
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
  if (d.prec != DP_FP32) {
    const int ng = dp::tc_systems_per_group(p->UP);
    p->n_fix = (int)((status_len(d) + ng - 1) / ng);
  }
  if (cudaMalloc(&p->d_off, sizeof(int) * (d.C + 1)) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(int) * status_len(d)) != cudaSuccess ||
      (p->n_fix && cudaMalloc(&p->d_fix, sizeof(int) * (p->n_fix + 2)) != cudaSuccess) ||
      (!ckr.empty() && cudaMalloc(&p->d_ckr, sizeof(float2) * ckr.size()) != cudaSuccess)) {
    cudaGetLastError();
    cudaFree(p->d_off);
    cudaFree(p->d_status);
    cudaFree(p->d_fix);
    cudaFree(p->d_ckr);
    delete p;
    return DP_ERR_OOM;
  }
  int dev = 0;
  if (cudaMemcpy(p->d_off, p->off.data(), sizeof(int) * (d.C + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(p->d_status, 0, sizeof(int) * status_len(d)) != cudaSuccess ||
      (p->d_fix && cudaMemset(p->d_fix + p->n_fix, 0, 2 * sizeof(int)) != cudaSuccess) ||
      (p->d_ckr && cudaMemcpy(p->d_ckr, ckr.data(), sizeof(float2) * ckr.size(),
                              cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->d_off);
    cudaFree(p->d_status);
    cudaFree(p->d_fix);
    cudaFree(p->d_ckr);
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
  free_host_pipeline(p);
  cudaFree(p->d_off);
  cudaFree(p->d_status);
  cudaFree(p->d_fix);
  cudaFree(p->d_ckr);
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

namespace {

// Steps a1-a6 for subcarriers [0, n_sc) of the given arrays (a chunk of the
// plan's subcarriers when n_sc < the plan's), status to `status`
// [n_sc * nsys], enqueued on the plan's stream.
cudaError_t precode_range(dp_plan *p, const float2 *h, const float2 *sy, float2 *x, int n_sc,
                          int *status) {
  const bool fd = p->d.mode == DP_FDWF;
  dp::SysDesc sd = make_sys(p, fd, h);
  sd.n_sc = n_sc;
  cudaError_t e = cudaSuccess;
  if (p->has_small) {  // FD-WF clusters with B_c < U: the paper's B_c x B_c form
    sd.skip_small = 1;
    e = dp::launch_fd_small(dp::InstDesc{sd, h, sy, x, status, nullptr}, p->bcp, p->stream);
    if (e != cudaSuccess || p->all_small) return e;
  }
  if (p->d.prec != DP_FP32 && dp::pipe_tc_supported(sd, p->UP)) {
    const bool fix = sd.refine == 2 && p->d_fix;
    int *list = fix ? p->d_fix : nullptr, *count = fix ? p->d_fix + p->n_fix : nullptr;
    e = dp::launch_pipe_tc(sd, p->UP, p->d.prec == DP_BF16, h, sy, x, status, nullptr,
                           p->stream, list, count);
    if (e != cudaSuccess || !fix) return e;
    // automatic precision escalation: the group kernel redoes the groups the
    // warp-specialized kernel listed (with an empty list its CTAs leave at
    // once), and empties the list for the next call
    return dp::launch_fixup_tc(sd, p->UP, p->d.prec == DP_BF16, h, sy, x, status, list, count,
                               p->n_sm, p->stream);
  }
  if (p->d.prec != DP_FP32)
    return dp::launch_fused_tc(sd, p->UP, p->d.prec == DP_BF16, h, sy, x, status, nullptr,
                               p->stream);
  if (p->fused_fits)
    return dp::launch_fused(sd, p->UP, p->maxrows_sys, h, sy, x, status, nullptr, p->stream);
  // Streaming form: Gram (cluster sum fused for WF/ZF), solve, apply.
  if (ensure_workspace(p) != DP_OK) return cudaErrorMemoryAllocation;
  e = dp::launch_gram(sd, p->UP, h, p->w_G, p->stream);
  if (e == cudaSuccess)
    e = dp::launch_solve(sd, p->UP, p->w_G, sy, p->w_Z, p->w_scale, status, p->stream);
  if (e == cudaSuccess) e = dp::launch_apply(sd, p->UP, h, p->w_Z, p->w_scale, x, p->stream);
  return e;
}

}  // namespace

dp_status dp_precode(dp_plan_t p, const void *H, const void *S, void *X) {
  if (!p) return DP_ERR_INVALID_ARG;
  if (p->d.n_sc == 0) return DP_OK;
  const bool k0 = p->d.K == 0;
  if (!arg_ok(H, false) || !arg_ok(S, k0) || !arg_ok(X, k0)) return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  const cudaError_t e = precode_range(p, static_cast<const float2 *>(H),
                                      static_cast<const float2 *>(S), static_cast<float2 *>(X),
                                      p->d.n_sc, p->d_status);
  return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : cuda_status(e);
}

dp_status dp_precode_host(dp_plan_t p, const void *H, const void *S, void *X, int chunk_sc) {
  if (!p) return DP_ERR_INVALID_ARG;
  const int n_sc = p->d.n_sc;
  if (n_sc == 0) return DP_OK;
  const bool k0 = p->d.K == 0;
  if (!H || (!k0 && (!S || !X))) return DP_ERR_INVALID_ARG;
  if (dp_status s = set_device(p)) return s;
  int chunk = chunk_sc > 0 ? chunk_sc : (n_sc + 7) / 8;
  if (chunk > n_sc) chunk = n_sc;
  if (dp_status s = ensure_host_pipeline(p, chunk)) return s;
  const size_t hb = (size_t)p->d.B * p->d.U * sizeof(float2),
               sb = (size_t)p->d.K * p->d.U * sizeof(float2),
               xb = (size_t)p->d.K * p->d.B * sizeof(float2);
  const char *Hh = static_cast<const char *>(H);
  const char *Sh = static_cast<const char *>(S);
  char *Xh = static_cast<char *>(X);
  const size_t stage = (size_t)p->hp_chunk;
  // uploads start after the work already on the plan's stream (earlier
  // calls' downloads included: the plan's stream waited for them)
  cudaError_t e = cudaEventRecord(p->hp_start, p->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hp_up, p->hp_start, 0);
  const int nchunks = (n_sc + chunk - 1) / chunk;
  for (int i = 0; i < nchunks && e == cudaSuccess; ++i) {
    const int b = i % dp_plan::NSTAGE;
    const int n0 = i * chunk, nc = n_sc - n0 < chunk ? n_sc - n0 : chunk;
    float2 *dH = p->hp_H + stage * b * (hb / sizeof(float2));
    float2 *dS = sb ? p->hp_S + stage * b * (sb / sizeof(float2)) : nullptr;
    float2 *dX = xb ? p->hp_X + stage * b * (xb / sizeof(float2)) : nullptr;
    // stage b's H and S are free once chunk i - 3 was precoded
    if (i >= dp_plan::NSTAGE) e = cudaStreamWaitEvent(p->hp_up, p->hp_calc_done[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dH, Hh + hb * n0, hb * nc, cudaMemcpyHostToDevice, p->hp_up);
    if (e == cudaSuccess && sb)
      e = cudaMemcpyAsync(dS, Sh + sb * n0, sb * nc, cudaMemcpyHostToDevice, p->hp_up);
    if (e == cudaSuccess) e = cudaEventRecord(p->hp_up_done[b], p->hp_up);
    // the kernels: after the upload, and once stage b's X went home
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->hp_up_done[b], 0);
    if (e == cudaSuccess && i >= dp_plan::NSTAGE)
      e = cudaStreamWaitEvent(p->stream, p->hp_down_done[b], 0);
    if (e == cudaSuccess)
      e = precode_range(p, dH, dS, dX, nc, p->d_status + (size_t)n0 * p->nsys);
    if (e == cudaSuccess) e = cudaEventRecord(p->hp_calc_done[b], p->stream);
    // the download
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hp_down, p->hp_calc_done[b], 0);
    if (e == cudaSuccess && xb)
      e = cudaMemcpyAsync(Xh + xb * n0, dX, xb * nc, cudaMemcpyDeviceToHost, p->hp_down);
    if (e == cudaSuccess) e = cudaEventRecord(p->hp_down_done[b], p->hp_down);
  }
  // the call completes on the plan's stream
  for (int i = nchunks - dp_plan::NSTAGE; i < nchunks && e == cudaSuccess; ++i)
    if (i >= 0) e = cudaStreamWaitEvent(p->stream, p->hp_down_done[i % dp_plan::NSTAGE], 0);
  return e == cudaErrorMemoryAllocation ? DP_ERR_OOM : cuda_status(e);
}

dp_status dp_debug_stall(dp_plan_t p, int microseconds) {
  if (!p || microseconds < 0 || microseconds > 1000000) return DP_ERR_INVALID_ARG;
  p->dbg_stall_us = microseconds;
  return DP_OK;
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
