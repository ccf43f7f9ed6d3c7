// dp_batch.cu -- batched precoding of many instances of uneven size (users,
// antennas, clusters, subcarriers, mode, precision) in persistent launches.
//
// The instances are sorted into buckets by kernel family and padded user
// count: the tensor-core family (BF16/FP16 Gram, <= 32 users), the FP32
// fused family (antenna block resident in shared memory) and a streaming
// remainder (instances whose blocks do not fit: Gram, solve and apply
// kernels per instance).  Every bucket is one persistent launch whose CTAs
// pull work items (a group of systems of one instance) from an atomic queue,
// largest items first.  The launch sequence is captured once into a CUDA
// graph and replayed; per call only the table of device pointers is
// uploaded.  dp_batch_tune times each bucket at every feasible CTAs-per-SM
// count and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dprecode.h"
#include "dp_internal.h"

namespace {

enum Family { FAM_TC = 0, FAM_FUSED = 1, FAM_STREAM = 2, FAM_FDSMALL = 3, FAM_PIPE = 4 };

struct Bucket {
  int family;
  int UP;
  bool bf16;
  int Kmax = 0;
  int maxrows = 0;
  std::vector<dp::WorkItem> items;
  dp::WorkItem *d_items = nullptr;
  int max_blocks = 1;   // occupancy limit per SM
  int blocks = 1;       // chosen CTAs per SM
  float tuned_ms = -1.f;
  long long systems = 0;    // systems of the bucket's items
  double alg_bytes = 0.0;   // algorithmic bytes: H rows, their X rows and the
                            // system's symbols, once each
  // warp-specialized family with automatic refinement: the list of groups
  // holding marked systems (items ints, then the count) and the CTAs per SM
  // of its fix-up launch
  bool fix = false;
  int *d_fix = nullptr;
  int fix_blocks = 1;
  // tensor-core family with many users: Gram, solve and apply as three
  // launches through a workspace (none of its instances refines every system)
  bool split = false, forced_refine = false;
  dp::SplitWs ws{};
};

struct Inst {
  dp_plan_desc d;
  std::vector<int> off;
  int UP, nsys, maxrows, family;
  bool bf16;
  bool has_small = false, all_small = false;  // FD-WF clusters with B_c < U
  int bcp = 0;
  size_t status_off;  // offset of this instance's status block in the batch array
  // workspace of the streaming family
  float2 *w_G = nullptr, *w_Z = nullptr;
  float *w_scale = nullptr;
  int *d_off = nullptr;
  // FD-WF with per-cluster power: (kappa_c, rho_c^2) per cluster
  std::vector<float2> ckr;
  float2 *d_ckr = nullptr;
};

bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

dp_status validate(const dp_plan_desc &d, std::vector<int> &off) {
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
  off.assign(d.C + 1, 0);
  for (int c = 0; c < d.C; ++c) {
    int bc;
    if (d.cluster_sizes) {
      bc = d.cluster_sizes[c];
    } else {
      if (d.B % d.C) return DP_ERR_PARTITION;
      bc = d.B / d.C;
    }
    if (bc < 1) return DP_ERR_PARTITION;
    off[c + 1] = off[c] + bc;
  }
  if (off[d.C] != d.B) return DP_ERR_PARTITION;
  int minbc = d.B;
  for (int c = 0; c < d.C; ++c) minbc = std::min(minbc, off[c + 1] - off[c]);
  if ((d.mode == DP_ZF || (d.mode == DP_WF && d.N0 == 0.f)) && d.B < d.U)
    return DP_ERR_UNSUPPORTED;
  if (d.mode == DP_FDWF && (double)d.tau * d.U * d.N0 * d.C / d.rho2 == 0.0 && minbc < d.U)
    return DP_ERR_UNSUPPORTED;
  return DP_OK;
}

dp::SysDesc sys_of(const Inst &in, const void *H) {
  dp::SysDesc s{};
  const dp_plan_desc &d = in.d;
  s.U = d.U;
  s.B = d.B;
  s.K = d.K;
  s.n_sc = d.n_sc;
  s.nsys = in.nsys;
  s.off = in.d_off;
  s.Es = d.Es;
  const double U = d.U, N0 = d.N0, rho2 = d.rho2, C = d.C;
  if (d.mode == DP_ZF || d.mode == DP_MRT) {
    s.kappa = 0.f;
    s.rho2_sys = d.rho2;
  } else if (d.mode == DP_WF) {
    s.kappa = (float)(U * N0 / rho2);
    s.rho2_sys = d.rho2;
  } else {
    s.kappa = (float)(d.tau * U * N0 / (rho2 / C));
    s.rho2_sys = (float)(rho2 / C);
  }
  s.tma_ok = (d.U % 2 == 0) && (H == nullptr || a16(H));
  s.skip_small = in.has_small ? 1 : 0;
  s.refine = dp::refine_mode(d.refine, d.prec == DP_FP32, d.mode == DP_MRT);
  s.mrt = d.mode == DP_MRT;
  s.ckr = in.d_ckr;
  return s;
}

}  // namespace

struct dp_batch {
  int device = 0, n_sm = 0;
  cudaStream_t stream = nullptr;
  std::vector<Inst> insts;
  std::vector<Bucket> buckets;
  std::vector<int> streaming;            // instances of the streaming family
  dp::InstDesc *d_insts = nullptr;        // device table, rewritten every call
  std::vector<dp::InstDesc> h_insts;
  int *d_queues = nullptr;                // three counters per bucket
  int *d_status = nullptr;
  size_t status_len = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string info;
  // per-bucket timing (dp_batch_set_timing): event k before bucket k, the
  // last after every bucket; 1 = recorded from the graph, 2 = eager launches
  int timing = 0;
  std::vector<cudaEvent_t> ev;
};

namespace {

void free_batch(dp_batch *b) {
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto &bk : b->buckets) {
    cudaFree(bk.d_items);
    cudaFree(bk.d_fix);
    cudaFree(bk.ws.G);
    cudaFree(bk.ws.Z);
    cudaFree(bk.ws.sc);
    cudaFree(bk.ws.st);
  }
  for (auto &in : b->insts) {
    cudaFree(in.w_G);
    cudaFree(in.w_Z);
    cudaFree(in.w_scale);
    cudaFree(in.d_off);
    cudaFree(in.d_ckr);
  }
  cudaFree(b->d_insts);
  cudaFree(b->d_queues);
  cudaFree(b->d_status);
  cudaGetLastError();
  delete b;
}

// Enqueue bucket k (queue reset + persistent launch).
cudaError_t enqueue_bucket(dp_batch *b, int k, cudaStream_t s) {
  Bucket &bk = b->buckets[k];
  if (bk.items.empty()) return cudaSuccess;
  int *q = b->d_queues + 3 * k;  // three counters per bucket
  cudaError_t e = cudaMemsetAsync(q, 0, 3 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int n = (int)bk.items.size();
  const int grid = std::max(1, std::min<int>(bk.blocks * b->n_sm, n));
  if (bk.family == FAM_PIPE) {
    // the list's count is the bucket's third counter (zeroed above)
    e = dp::launch_batch_pipe_tc(bk.UP, bk.bf16, b->d_insts, bk.d_items, n,
                                 bk.fix ? bk.d_fix : nullptr, bk.fix ? q + 2 : nullptr,
                                 std::min(b->n_sm, n), s);
    if (e != cudaSuccess || !bk.fix) return e;
    // automatic refinement: the group kernel redoes the listed groups
    return dp::launch_batch_tc(bk.UP, bk.bf16, b->d_insts, bk.d_items, n, q, bk.Kmax,
                               std::max(1, bk.fix_blocks * b->n_sm), s, bk.d_fix, q + 2);
  }
  if (bk.family == FAM_TC && bk.split) {
    for (int ph = 1; ph <= 3 && e == cudaSuccess; ++ph)
      e = (ph == 2 && dp::row_solve_supported(bk.UP))
              ? dp::launch_solve_rows(bk.UP, bk.bf16, b->d_insts, bk.d_items, n, q + 1, bk.ws,
                                      b->n_sm, s)
              : dp::launch_batch_tc(bk.UP, bk.bf16, b->d_insts, bk.d_items, n, q + ph - 1,
                                    bk.Kmax, grid, s, nullptr, nullptr, ph, bk.ws);
    return e;
  }
  if (bk.family == FAM_TC)
    return dp::launch_batch_tc(bk.UP, bk.bf16, b->d_insts, bk.d_items, n, q, bk.Kmax, grid, s);
  if (bk.family == FAM_FDSMALL)
    return dp::launch_batch_fd_small(bk.UP, b->d_insts, bk.d_items, n, q, bk.Kmax, grid, s);
  return dp::launch_batch_fused(bk.UP, b->d_insts, bk.d_items, n, q, bk.maxrows, bk.Kmax, grid,
                                s);
}

cudaError_t enqueue_streaming(dp_batch *b, int i, cudaStream_t s) {
  Inst &in = b->insts[i];
  const dp::InstDesc &t = b->h_insts[i];
  if (in.d.n_sc == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (in.has_small) {
    e = dp::launch_fd_small(t, in.bcp, s);
    if (e != cudaSuccess || in.all_small) return e;
  }
  e = dp::launch_gram(t.d, in.UP, t.H, in.w_G, s);
  if (e == cudaSuccess) e = dp::launch_solve(t.d, in.UP, in.w_G, t.S, in.w_Z, in.w_scale, t.status, s);
  if (e == cudaSuccess && in.d.K > 0) e = dp::launch_apply(t.d, in.UP, t.H, in.w_Z, in.w_scale, t.X, s);
  return e;
}

// The persistent bucket launches (the part a graph captures: they read every
// pointer from the device table, so the graph is independent of the call).
cudaError_t enqueue_buckets(dp_batch *b, cudaStream_t s, bool capturing = false) {
  cudaError_t e = cudaSuccess;
  const bool ev = b->timing != 0 && b->ev.size() == b->buckets.size() + 1;
  // inside a capture the records become event-record nodes of the graph
  const unsigned fl = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  for (size_t k = 0; k < b->buckets.size() && e == cudaSuccess; ++k) {
    if (ev) e = cudaEventRecordWithFlags(b->ev[k], s, fl);
    if (e == cudaSuccess) e = enqueue_bucket(b, (int)k, s);
  }
  if (ev && e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev[b->buckets.size()], s, fl);
  return e;
}

// Streaming instances take their pointers as kernel arguments: enqueued
// eagerly on every call.
cudaError_t enqueue_streams(dp_batch *b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (size_t j = 0; j < b->streaming.size() && e == cudaSuccess; ++j)
    e = enqueue_streaming(b, b->streaming[j], s);
  return e;
}

// Write the pointer table for this call (host copy + upload on the stream).
dp_status upload_table(dp_batch *b, const void *const *H, const void *const *S, void *const *X) {
  for (size_t i = 0; i < b->insts.size(); ++i) {
    const Inst &in = b->insts[i];
    const bool empty = in.d.n_sc == 0, k0 = in.d.K == 0;
    if (!empty && (!H[i] || !a16(H[i]))) return DP_ERR_INVALID_ARG;
    if (!empty && !k0 && (!S[i] || !a16(S[i]) || !X[i] || !a16(X[i]))) return DP_ERR_INVALID_ARG;
    dp::InstDesc &t = b->h_insts[i];
    t.d = sys_of(in, H[i]);
    t.H = static_cast<const float2 *>(H[i]);
    t.S = static_cast<const float2 *>(S[i]);
    t.X = static_cast<float2 *>(X[i]);
    t.status = b->d_status + in.status_off;
    t.scale_out = nullptr;
  }
  if (cudaMemcpyAsync(b->d_insts, b->h_insts.data(), sizeof(dp::InstDesc) * b->h_insts.size(),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return DP_ERR_CUDA;
  return DP_OK;
}

dp_status build_graph(dp_batch *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  // the legacy stream cannot be captured, and timing mode 2 asks for eager
  // launches: run eagerly
  if (b->stream == nullptr || b->timing == 2) return DP_OK;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return DP_OK;
  }
  cudaError_t e = enqueue_buckets(b, b->stream, true);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    b->exec = nullptr;
    return DP_ERR_CUDA;
  }
  b->graph = g;
  return DP_OK;
}

void describe(dp_batch *b) {
  std::string s = "{\"buckets\": [";
  for (size_t k = 0; k < b->buckets.size(); ++k) {
    const Bucket &bk = b->buckets[k];
    char buf[256];
    std::snprintf(buf, sizeof buf,
                  "%s{\"family\": \"%s\", \"users_padded\": %d, \"items\": %zu, "
                  "\"systems\": %lld, \"alg_bytes\": %.0f, "
                  "\"ctas_per_sm\": %d, \"max_ctas_per_sm\": %d, \"tuned_ms\": %.4f, "
                  "\"launches\": %d}",
                  k ? ", " : "",
                  bk.family == FAM_TC ? (bk.split ? (bk.bf16 ? "tc_split_bf16" : "tc_split_fp16")
                                               : (bk.bf16 ? "tc_bf16" : "tc_fp16"))
                  : bk.family == FAM_PIPE ? (bk.bf16 ? "tc_pipe_bf16" : "tc_pipe_fp16")
                  : bk.family == FAM_FDSMALL ? "fd_small_clusters" : "fp32_fused", bk.UP,
                  bk.items.size(), bk.systems, bk.alg_bytes, bk.blocks, bk.max_blocks,
                  bk.tuned_ms,
                  bk.items.empty() ? 0
                  : bk.family == FAM_PIPE ? (bk.fix ? 2 : 1)
                  : (bk.family == FAM_TC && bk.split) ? 3 : 1);
    s += buf;
  }
  char tail[64];
  std::snprintf(tail, sizeof tail, "], \"streaming_instances\": %zu}", b->streaming.size());
  s += tail;
  b->info = s;
}

}  // namespace

namespace dp {
int resident_blocks(const void *kernel, int threads, size_t dyn_bytes, int tmem_cols) {
  cudaFuncAttributes a{};
  int dev = 0, regs_sm = 0, thr_sm = 0, smem_sm = 0, resv = 0, blk_sm = 0;
  if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ||
      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev)) {
    cudaGetLastError();
    return 0;
  }
  const int warps = (threads + 31) / 32;
  int n = std::min(blk_sm, thr_sm / (32 * warps));
  const int regs_warp = ((a.numRegs * 32 + 255) / 256) * 256;
  if (regs_warp > 0) n = std::min(n, (regs_sm / regs_warp) / warps);
  const size_t smem = dyn_bytes + a.sharedSizeBytes + (size_t)resv;
  n = std::min<size_t>(n, (size_t)smem_sm / smem);
  if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
  return std::max(n, 0);
}
}  // namespace dp

extern "C" {

dp_status dp_batch_create(const dp_plan_desc *descs, int n, dp_stream_t stream, dp_batch_t *out) {
  if (!out) return DP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || n < 1) return DP_ERR_INVALID_ARG;
  dp_batch *b = new (std::nothrow) dp_batch;
  if (!b) return DP_ERR_OOM;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->insts.resize(n);
  std::map<std::tuple<int, int, int>, int> bucket_of;
  size_t status_len = 0;
  for (int i = 0; i < n; ++i) {
    Inst &in = b->insts[i];
    in.d = descs[i];
    dp_status st = validate(in.d, in.off);
    if (st == DP_OK &&
        !dp::cluster_power_table(in.d.mode == DP_FDWF, in.d.cluster_power, in.d.C, in.d.rho2,
                                 in.d.tau, in.d.U, in.d.N0, in.ckr))
      st = DP_ERR_INVALID_ARG;
    if (st != DP_OK) {
      delete b;
      return st;
    }
    in.d.cluster_sizes = nullptr;
    in.d.cluster_power = nullptr;  // the table is in.ckr
    in.UP = dp::padded_users(in.d.U);
    in.nsys = in.d.mode == DP_FDWF ? in.d.C : 1;
    int maxbc = 0;
    for (int c = 0; c < in.d.C; ++c) maxbc = std::max(maxbc, in.off[c + 1] - in.off[c]);
    in.maxrows = in.d.mode == DP_FDWF ? maxbc : in.d.B;
    in.bf16 = in.d.prec == DP_BF16;
    if (in.d.mode == DP_FDWF) {
      int maxsmall = 0, nsmall = 0;
      for (int c = 0; c < in.d.C; ++c) {
        const int bc = in.off[c + 1] - in.off[c];
        if (bc < in.d.U && bc <= 32) {
          ++nsmall;
          maxsmall = std::max(maxsmall, bc);
        }
      }
      in.has_small = nsmall > 0;
      in.all_small = nsmall == in.d.C;
      in.bcp = dp::fd_small_bcp(maxsmall);
    }
    if (in.d.prec != DP_FP32 && dp::tc_supported(in.UP))
      in.family = dp::pipe_tc_supported(sys_of(in, nullptr), in.UP) ? FAM_PIPE : FAM_TC;
    else if (dp::fused_smem_bytes(in.UP, in.maxrows, in.d.K) != 0) in.family = FAM_FUSED;
    else in.family = FAM_STREAM;
    in.status_off = status_len;
    status_len += (size_t)in.d.n_sc * in.nsys;
  }
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return DP_ERR_CUDA;
  }
  b->status_len = status_len;
  bool oom = cudaMalloc(&b->d_status, sizeof(int) * std::max<size_t>(1, status_len)) != cudaSuccess ||
             cudaMalloc(&b->d_insts, sizeof(dp::InstDesc) * n) != cudaSuccess;
  if (!oom) cudaMemset(b->d_status, 0, sizeof(int) * std::max<size_t>(1, status_len));
  // cluster offsets and work items
  for (int i = 0; i < n && !oom; ++i) {
    Inst &in = b->insts[i];
    oom = cudaMalloc(&in.d_off, sizeof(int) * in.off.size()) != cudaSuccess ||
          (!in.ckr.empty() &&
           cudaMalloc(&in.d_ckr, sizeof(float2) * in.ckr.size()) != cudaSuccess);
    if (oom) break;
    cudaMemcpy(in.d_off, in.off.data(), sizeof(int) * in.off.size(), cudaMemcpyHostToDevice);
    if (in.d_ckr)
      cudaMemcpy(in.d_ckr, in.ckr.data(), sizeof(float2) * in.ckr.size(), cudaMemcpyHostToDevice);
    const int nsys_total = in.d.n_sc * in.nsys;
    if (nsys_total == 0) continue;
    if (in.has_small && in.family != FAM_STREAM) {
      // small clusters: one item per system in the B_c x B_c bucket
      auto key = std::make_tuple((int)FAM_FDSMALL, in.bcp, 0);
      auto it = bucket_of.find(key);
      int k;
      if (it == bucket_of.end()) {
        k = (int)b->buckets.size();
        bucket_of[key] = k;
        Bucket bk;
        bk.family = FAM_FDSMALL;
        bk.UP = in.bcp;
        bk.bf16 = false;
        b->buckets.push_back(bk);
      } else {
        k = it->second;
      }
      Bucket &bk = b->buckets[k];
      bk.Kmax = std::max(bk.Kmax, in.d.K);
      for (int n = 0; n < in.d.n_sc; ++n)
        for (int c = 0; c < in.d.C; ++c) {
          const int bc = in.off[c + 1] - in.off[c];
          if (bc < in.d.U && bc <= 32) bk.items.push_back(dp::WorkItem{i, n * in.nsys + c, 1});
        }
      if (in.all_small) continue;
    }
    if (in.family == FAM_STREAM) {
      b->streaming.push_back(i);
      oom = cudaMalloc(&in.w_G, sizeof(float2) * nsys_total * in.d.U * in.d.U) != cudaSuccess ||
            cudaMalloc(&in.w_Z, sizeof(float2) * nsys_total * std::max(1, in.d.K) * in.d.U) !=
                cudaSuccess ||
            cudaMalloc(&in.w_scale, sizeof(float) * nsys_total) != cudaSuccess;
      continue;
    }
    const bool tcfam = in.family == FAM_TC || in.family == FAM_PIPE;
    auto key = std::make_tuple(in.family, in.UP, tcfam ? (int)in.bf16 : 0);
    auto it = bucket_of.find(key);
    int k;
    if (it == bucket_of.end()) {
      k = (int)b->buckets.size();
      bucket_of[key] = k;
      Bucket bk;
      bk.family = in.family;
      bk.UP = in.UP;
      bk.bf16 = tcfam && in.bf16;
      b->buckets.push_back(bk);
    } else {
      k = it->second;
    }
    Bucket &bk = b->buckets[k];
    bk.Kmax = std::max(bk.Kmax, in.d.K);
    bk.maxrows = std::max(bk.maxrows, in.maxrows);
    if (in.family == FAM_PIPE && sys_of(in, nullptr).refine == 2) bk.fix = true;
    if (sys_of(in, nullptr).refine == 1) bk.forced_refine = true;
    const int per = in.family == FAM_TC   ? dp::tc_systems_per_group(in.UP)
                    : in.family == FAM_PIPE ? dp::pipe_systems_per_group(in.UP)
                                            : 1;
    for (int s0 = 0; s0 < nsys_total; s0 += per)
      bk.items.push_back(dp::WorkItem{i, s0, std::min(per, nsys_total - s0)});
  }
  if (oom) {
    free_batch(b);
    return DP_ERR_OOM;
  }
  // algorithmic bytes per bucket: every system's H rows and X rows, and the
  // symbols it reads (per cluster in FD-WF, which hands s to every cluster)
  for (auto &bk : b->buckets) {
    for (const dp::WorkItem &w : bk.items) {
      const Inst &in = b->insts[w.inst];
      for (int j = 0; j < w.nact; ++j) {
        const int sys = w.sys0 + j;
        const int c = sys % in.nsys;
        const int rows = in.nsys == 1 ? in.d.B : in.off[c + 1] - in.off[c];
        bk.alg_bytes += 8.0 * ((double)in.d.U * rows + (double)in.d.K * rows +
                               (double)in.d.K * in.d.U);
        ++bk.systems;
      }
    }
  }
  // largest items first (antenna rows of the item's systems), so that the
  // queue's tail is made of small items
  for (auto &bk : b->buckets) {
    auto cost = [&](const dp::WorkItem &w) {
      const Inst &in = b->insts[w.inst];
      return (long long)in.maxrows * in.UP * in.UP * w.nact;
    };
    std::stable_sort(bk.items.begin(), bk.items.end(),
                     [&](const dp::WorkItem &a, const dp::WorkItem &c) { return cost(a) > cost(c); });
    if (cudaMalloc(&bk.d_items, sizeof(dp::WorkItem) * bk.items.size()) != cudaSuccess) {
      free_batch(b);
      return DP_ERR_OOM;
    }
    cudaMemcpy(bk.d_items, bk.items.data(), sizeof(dp::WorkItem) * bk.items.size(),
               cudaMemcpyHostToDevice);
    bk.max_blocks = bk.family == FAM_TC
                        ? dp::tc_max_blocks_per_sm(bk.UP, bk.bf16, bk.Kmax)
                        : bk.family == FAM_PIPE ? 1  // one warp-specialized CTA per SM
                        : bk.family == FAM_FDSMALL
                              ? dp::fd_small_max_blocks_per_sm(bk.UP, bk.Kmax)
                              : dp::fused_max_blocks_per_sm(bk.UP, bk.maxrows, bk.Kmax);
    if (bk.family == FAM_TC && bk.UP > 16 && !bk.forced_refine) {
      const size_t ni = bk.items.size(), ng = (size_t)dp::tc_systems_per_group(bk.UP);
      bk.split = true;
      bk.ws.kmax = bk.Kmax;
      if (cudaMalloc(&bk.ws.G, sizeof(float2) * ni * ng * bk.UP * bk.UP) != cudaSuccess ||
          cudaMalloc(&bk.ws.Z, sizeof(float2) * ni * ng * std::max(1, bk.Kmax) * bk.UP) !=
              cudaSuccess ||
          cudaMalloc(&bk.ws.sc, sizeof(float) * ni * ng) != cudaSuccess ||
          cudaMalloc(&bk.ws.st, sizeof(int) * ni * ng) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return DP_ERR_OOM;
      }
    }
    if (bk.fix) {
      bk.fix_blocks = dp::tc_max_blocks_per_sm(bk.UP, bk.bf16, bk.Kmax);
      if (bk.fix_blocks < 1 ||
          cudaMalloc(&bk.d_fix, sizeof(int) * bk.items.size()) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return bk.fix_blocks < 1 ? DP_ERR_UNSUPPORTED : DP_ERR_OOM;
      }
    }
    if (bk.max_blocks < 1) {
      free_batch(b);
      return DP_ERR_UNSUPPORTED;
    }
    bk.blocks = bk.max_blocks;
  }
  if (cudaMalloc(&b->d_queues, 3 * sizeof(int) * std::max<size_t>(1, b->buckets.size())) !=
      cudaSuccess) {
    free_batch(b);
    return DP_ERR_OOM;
  }
  b->h_insts.resize(n);
  for (int i = 0; i < n; ++i) b->h_insts[i] = dp::InstDesc{sys_of(b->insts[i], nullptr), nullptr,
                                                           nullptr, nullptr,
                                                           b->d_status + b->insts[i].status_off,
                                                           nullptr};
  describe(b);
  *out = b;
  return DP_OK;
}

dp_status dp_batch_destroy(dp_batch_t b) {
  if (!b) return DP_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  return DP_OK;
}

dp_status dp_batch_precode(dp_batch_t b, const void *const *H, const void *const *S,
                           void *const *X) {
  if (!b || !H || !S || !X) return DP_ERR_INVALID_ARG;
  if (cudaSetDevice(b->device) != cudaSuccess) return DP_ERR_CUDA;
  if (dp_status st = upload_table(b, H, S, X)) return st;
  if (!b->exec && b->stream != nullptr) {
    if (dp_status st = build_graph(b)) return st;
  }
  cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, b->stream) : enqueue_buckets(b, b->stream);
  if (e == cudaSuccess) e = enqueue_streams(b, b->stream);
  return e == cudaSuccess ? DP_OK : DP_ERR_CUDA;
}

dp_status dp_batch_tune(dp_batch_t b, const void *const *H, const void *const *S, void *const *X,
                        int trials) {
  if (!b || !H || !S || !X || trials < 1) return DP_ERR_INVALID_ARG;
  if (cudaSetDevice(b->device) != cudaSuccess) return DP_ERR_CUDA;
  if (dp_status st = upload_table(b, H, S, X)) return st;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return DP_ERR_CUDA;
  // every trial starts with a cold L2, as a bucket does in the replayed pass
  // (the bucket before it streamed other instances' data): a buffer twice the
  // L2 size is written before each timed run (none if it cannot be had)
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device);
  void *flush = nullptr;
  const size_t flush_bytes = 2 * (size_t)std::max(l2, 0);
  if (flush_bytes && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  dp_status rc = DP_OK;
  for (size_t k = 0; k < b->buckets.size() && rc == DP_OK; ++k) {
    Bucket &bk = b->buckets[k];
    if (bk.items.empty()) continue;
    float best = 1e30f;
    int best_blocks = bk.max_blocks;
    for (int c = 1; c <= bk.max_blocks && rc == DP_OK; ++c) {
      bk.blocks = c;
      float sum = 0.f;
      for (int t = 0; t <= trials && rc == DP_OK; ++t) {  // first run warms up
        if (flush && cudaMemsetAsync(flush, t & 0xff, flush_bytes, b->stream) != cudaSuccess)
          rc = DP_ERR_CUDA;
        cudaEventRecord(e0, b->stream);
        if (enqueue_bucket(b, (int)k, b->stream) != cudaSuccess) rc = DP_ERR_CUDA;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = DP_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (t > 0) sum += ms;
      }
      // the largest count within 2 % of the fastest: alone, more resident
      // CTAs can look no faster, while in the replayed pass (cold L2, the
      // previous bucket's tail) they hide more latency
      const float ms = sum / trials;
      if (ms < best) {
        if (ms < best * 0.98f || c > best_blocks) best_blocks = c;
        best = ms;
      } else if (ms <= best * 1.02f) {
        best_blocks = c;
      }
    }
    bk.blocks = best_blocks;
    bk.tuned_ms = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(flush);
  if (rc != DP_OK) return rc;
  describe(b);
  return build_graph(b);
}

dp_status dp_batch_set_timing(dp_batch_t b, int mode) {
  if (!b || mode < 0 || mode > 2) return DP_ERR_INVALID_ARG;
  if (cudaSetDevice(b->device) != cudaSuccess) return DP_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DP_ERR_CUDA;
  if (mode != 0 && b->ev.empty()) {
    b->ev.assign(b->buckets.size() + 1, nullptr);
    for (auto &e : b->ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return DP_ERR_CUDA;
      }
  }
  b->timing = mode;
  return build_graph(b);
}

dp_status dp_batch_bucket_ms(dp_batch_t b, float *ms, int n) {
  if (!b || !ms || n < 0) return DP_ERR_INVALID_ARG;
  if (b->timing == 0 || b->ev.size() != b->buckets.size() + 1) return DP_ERR_UNSUPPORTED;
  if (cudaSetDevice(b->device) != cudaSuccess) return DP_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DP_ERR_CUDA;
  for (int k = 0; k < n && k < (int)b->buckets.size(); ++k) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, b->ev[k], b->ev[k + 1]) != cudaSuccess) {
      cudaGetLastError();
      return DP_ERR_CUDA;
    }
    ms[k] = t;
  }
  return DP_OK;
}

const char *dp_batch_describe(dp_batch_t b) { return b ? b->info.c_str() : ""; }

dp_status dp_batch_status_get(dp_batch_t b, int *host_status) {
  if (!b) return DP_ERR_INVALID_ARG;
  if (cudaSetDevice(b->device) != cudaSuccess) return DP_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return DP_ERR_CUDA;
  std::vector<int> sys(std::max<size_t>(1, b->status_len));
  if (b->status_len &&
      cudaMemcpy(sys.data(), b->d_status, sizeof(int) * b->status_len, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return DP_ERR_CUDA;
  dp_status first = DP_OK;
  size_t o = 0;
  for (const Inst &in : b->insts) {
    for (int n = 0; n < in.d.n_sc; ++n) {
      int worst = 0;
      for (int g = 0; g < in.nsys; ++g) worst = std::max(worst, sys[in.status_off + (size_t)n * in.nsys + g]);
      if (host_status) host_status[o] = worst;
      ++o;
      if (first == DP_OK && worst) first = static_cast<dp_status>(worst);
    }
  }
  return first;
}

}  // extern "C"
