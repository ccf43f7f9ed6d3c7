// dp_server.cu -- continuous-batching precoding server.
//
// A cell is one channel (its plan description and a device-resident H that
// the caller can swap, e.g. after each uplink channel estimate).  A request
// precodes one slot of a cell: symbols S (device) -> precoded X written into
// a buffer the server takes from its device arena.  A dispatcher thread
// admits pending requests in arrival order whenever an in-flight slot and
// enough arena memory are free (admission by free device memory), launches
// them round-robin over the server's CUDA streams (so requests overlap on the
// GPU, those of one cell included; only cells in the streaming FP32 form,
// whose workspace is per cell, keep their slots in order on the cell's
// stream), and retires completed ones: status copied out, latency recorded
// (arrival -> completion observed on the host), output buffer kept until the
// caller releases it (or released at once in auto-release mode).
//
// Solve cache: a cell's T = (G + kappa I)^{-1} and scale are recomputed on
// the cell's own cache stream when a request arrives with a channel other
// than the cached one; the recomputation first waits for every in-flight
// request of the cell (they still read the old T), and every request waits for
// the newest recomputation before it whitens.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dprecode.h"
#include "dp_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device allocation (256-byte granules).
class Arena {
 public:
  bool init(size_t bytes) {
    bytes_ = (bytes + 255) & ~size_t(255);
    if (cudaMalloc(&base_, bytes_) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    free_[0] = bytes_;
    return true;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  // offset of a block of >= bytes, or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        high_ = std::max(high_, used_);
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  unsigned char *ptr(size_t off) const { return static_cast<unsigned char *>(base_) + off; }
  size_t bytes() const { return bytes_; }
  size_t high_water() const { return high_; }

 private:
  void *base_ = nullptr;
  size_t bytes_ = 0, used_ = 0, high_ = 0;
  std::map<size_t, size_t> free_;
};

struct Cell {
  dp_plan_desc d;
  std::vector<int> off;
  int *d_off = nullptr;
  // FD-WF with per-cluster power: (kappa_c, rho_c^2) per cluster, in the same
  // allocation as d_off (after it)
  float2 *d_ckr = nullptr;
  int UP = 8, nsys = 1, maxrows = 0;
  bool tc = false, fused = false;
  bool has_small = false, all_small = false;  // FD-WF clusters with B_c < U
  int bcp = 0;
  const void *H = nullptr;
  int stream = 0;
  bool overlap = false;  // requests of this cell may run concurrently
  size_t x_bytes = 0, st_bytes = 0;
  size_t w_bytes = 0;  // per-request workspace: z [sys][K][U], then scale [sys]
  // streaming-form workspace (cells whose antenna block exceeds shared memory,
  // and cells with a solve cache)
  float2 *w_G = nullptr, *w_Z = nullptr;
  float *w_scale = nullptr;
  // solve cache: T, scale and status per system for the channel c_H, written
  // on c_stream; c_ready marks the newest recomputation
  bool cached = false;
  const void *c_H = nullptr;
  float2 *c_T = nullptr;
  float *c_scale = nullptr;
  int *c_st = nullptr;
  cudaStream_t c_stream = nullptr;
  cudaEvent_t c_ready = nullptr;
};

struct Request {
  uint64_t id;
  int cell;
  const void *S;
  const void *H;  // channel at submission
  Clock::time_point t_arrival, t_done;
  size_t x_off = SIZE_MAX, st_off = SIZE_MAX, w_off = SIZE_MAX;
  cudaEvent_t ev = nullptr;
  int status = 0;
  bool done = false, released = false;
};

bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

struct dp_server {
  dp_server_config cfg{};
  int n_sm = 0;
  Arena arena;
  std::vector<cudaStream_t> streams;
  std::vector<Cell> cells;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> pending;
  std::vector<Request *> inflight;
  std::unordered_map<uint64_t, Request *> all;  // not yet released
  std::vector<double> lat_ms;
  uint64_t next_id = 1;
  uint64_t next_stream = 0;  // round-robin stream choice
  long long subcarriers_done = 0;
  int inflight_peak = 0;
  int failures = 0;
  bool stop = false;
  bool error = false;
  std::thread worker;
  Clock::time_point t_first, t_last;
  bool have_first = false;
};

namespace {

dp::SysDesc sys_of(const Cell &c, const void *H) {
  dp::SysDesc s{};
  const dp_plan_desc &d = c.d;
  s.U = d.U;
  s.B = d.B;
  s.K = d.K;
  s.n_sc = d.n_sc;
  s.nsys = c.nsys;
  s.off = c.d_off;
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
  s.tma_ok = (d.U % 2 == 0) && a16(H);
  s.skip_small = c.has_small ? 1 : 0;
  s.refine = dp::refine_mode(d.refine, d.prec == DP_FP32, d.mode == DP_MRT);
  s.mrt = d.mode == DP_MRT;
  s.ckr = c.d_ckr;
  return s;
}

cudaError_t launch_request(dp_server *sv, Request *r) {
  Cell &c = sv->cells[r->cell];
  cudaStream_t st = c.overlap ? sv->streams[sv->next_stream++ % sv->streams.size()]
                              : sv->streams[c.stream];
  const dp::SysDesc d = sys_of(c, r->H);
  const float2 *H = static_cast<const float2 *>(r->H);
  const float2 *S = static_cast<const float2 *>(r->S);
  float2 *X = reinterpret_cast<float2 *>(sv->arena.ptr(r->x_off));
  int *status = reinterpret_cast<int *>(sv->arena.ptr(r->st_off));
  cudaError_t e = cudaSuccess;
  if (c.cached) {
    // the channel's Gram, inverse and scale once per channel; then z = T s
    // and the apply for every request
    const size_t ns = (size_t)c.d.n_sc * c.nsys;
    float2 *Z = reinterpret_cast<float2 *>(sv->arena.ptr(r->w_off));
    float *zscale = reinterpret_cast<float *>(Z + ns * c.d.K * c.d.U);
    if (r->H != c.c_H) {
      // the cell's in-flight requests still read the old T
      for (const Request *q : sv->inflight)
        if (q->cell == r->cell && e == cudaSuccess) e = cudaStreamWaitEvent(c.c_stream, q->ev, 0);
      if (e == cudaSuccess) e = dp::launch_gram(d, c.UP, H, c.w_G, c.c_stream);
      if (e == cudaSuccess)
        e = dp::launch_cache_invert(d, c.UP, c.w_G, c.c_T, c.c_scale, c.c_st, c.c_stream);
      if (e == cudaSuccess) e = cudaEventRecord(c.c_ready, c.c_stream);
      if (e == cudaSuccess) c.c_H = r->H;
    }
    if (e == cudaSuccess && c.has_small)
      e = dp::launch_fd_small(dp::InstDesc{d, H, S, X, status, nullptr}, c.bcp, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c.c_ready, 0);
    if (e == cudaSuccess)
      e = dp::launch_cache_whiten(d, c.UP, c.c_T, c.c_scale, c.c_st, S, Z, zscale, status, st);
    if (e == cudaSuccess) e = dp::launch_apply(d, c.UP, H, Z, zscale, X, st);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, st);
    return e;
  }
  if (c.has_small) e = dp::launch_fd_small(dp::InstDesc{d, H, S, X, status, nullptr}, c.bcp, st);
  if (e != cudaSuccess || c.all_small) {
  } else if (c.tc)
    e = dp::launch_fused_tc(d, c.UP, c.d.prec == DP_BF16, H, S, X, status, nullptr, st);
  else if (c.fused)
    e = dp::launch_fused(d, c.UP, c.maxrows, H, S, X, status, nullptr, st);
  else {
    e = dp::launch_gram(d, c.UP, H, c.w_G, st);
    if (e == cudaSuccess) e = dp::launch_solve(d, c.UP, c.w_G, S, c.w_Z, c.w_scale, status, st);
    if (e == cudaSuccess && c.d.K > 0) e = dp::launch_apply(d, c.UP, H, c.w_Z, c.w_scale, X, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(r->ev, st);
  return e;
}

// Retire completed requests (lock held).
void retire(dp_server *sv) {
  for (size_t i = 0; i < sv->inflight.size();) {
    Request *r = sv->inflight[i];
    const cudaError_t q = cudaEventQuery(r->ev);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    r->t_done = Clock::now();
    if (q != cudaSuccess) {
      cudaGetLastError();
      sv->error = true;
    }
    Cell &c = sv->cells[r->cell];
    const size_t ns = (size_t)c.d.n_sc * c.nsys;
    if (ns) {
      std::vector<int> st(ns);
      cudaMemcpy(st.data(), sv->arena.ptr(r->st_off), sizeof(int) * ns, cudaMemcpyDeviceToHost);
      for (int v : st) r->status = std::max(r->status, v);
    }
    if (r->status) ++sv->failures;
    sv->arena.release(r->st_off, c.st_bytes);
    if (r->w_off != SIZE_MAX) sv->arena.release(r->w_off, c.w_bytes);
    r->w_off = SIZE_MAX;
    r->done = true;
    sv->lat_ms.push_back(
        std::chrono::duration<double, std::milli>(r->t_done - r->t_arrival).count());
    sv->subcarriers_done += c.d.n_sc;
    sv->t_last = r->t_done;
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
    if (sv->cfg.auto_release) {
      sv->arena.release(r->x_off, c.x_bytes);
      sv->all.erase(r->id);
      delete r;
    }
    sv->inflight[i] = sv->inflight.back();
    sv->inflight.pop_back();
  }
}

// Admit pending requests in order while slots and memory allow (lock held).
void admit(dp_server *sv) {
  while (!sv->pending.empty() && (int)sv->inflight.size() < sv->cfg.max_inflight) {
    Request *r = sv->pending.front();
    Cell &c = sv->cells[r->cell];
    const size_t xo = sv->arena.alloc(c.x_bytes);
    if (xo == SIZE_MAX) break;
    const size_t so = sv->arena.alloc(c.st_bytes);
    if (so == SIZE_MAX) {
      sv->arena.release(xo, c.x_bytes);
      break;
    }
    const size_t wo = c.w_bytes ? sv->arena.alloc(c.w_bytes) : SIZE_MAX;
    if (c.w_bytes && wo == SIZE_MAX) {
      sv->arena.release(xo, c.x_bytes);
      sv->arena.release(so, c.st_bytes);
      break;
    }
    r->x_off = xo;
    r->st_off = so;
    r->w_off = wo;
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess ||
        launch_request(sv, r) != cudaSuccess) {
      cudaGetLastError();
      sv->error = true;
      sv->arena.release(xo, c.x_bytes);
      sv->arena.release(so, c.st_bytes);
      if (wo != SIZE_MAX) sv->arena.release(wo, c.w_bytes);
      r->w_off = SIZE_MAX;
      if (r->ev) cudaEventDestroy(r->ev);
      r->ev = nullptr;
      r->done = true;
      r->status = DP_ERR_CUDA;
      sv->pending.pop_front();
      continue;
    }
    sv->pending.pop_front();
    sv->inflight.push_back(r);
    sv->inflight_peak = std::max(sv->inflight_peak, (int)sv->inflight.size());
  }
}

void worker_loop(dp_server *sv) {
  cudaSetDevice(sv->cfg.device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    retire(sv);
    admit(sv);
    if (sv->stop && sv->pending.empty() && sv->inflight.empty()) break;
    if (sv->inflight.empty() && sv->pending.empty()) {
      sv->cv.notify_all();
      sv->cv.wait(lk);
      continue;
    }
    sv->cv.notify_all();
    // requests in flight: poll finely so completion times are accurate
    lk.unlock();
    std::this_thread::sleep_for(std::chrono::microseconds(2));
    lk.lock();
  }
  sv->cv.notify_all();
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

dp_status dp_server_create(const dp_server_config *cfg, dp_server_t *out) {
  if (!out) return DP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->max_inflight < 1 || cfg->max_inflight > 1024 || cfg->streams < 1 ||
      cfg->streams > 64 || cfg->arena_bytes < 4096 ||
      (cfg->auto_release != 0 && cfg->auto_release != 1) ||
      (cfg->cache_solve != 0 && cfg->cache_solve != 1))
    return DP_ERR_INVALID_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  dp_server *sv = new (std::nothrow) dp_server;
  if (!sv) return DP_ERR_OOM;
  sv->cfg = *cfg;
  cudaDeviceGetAttribute(&sv->n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
  if (!sv->arena.init(cfg->arena_bytes)) {
    delete sv;
    return DP_ERR_OOM;
  }
  for (int i = 0; i < cfg->streams; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : sv->streams) cudaStreamDestroy(x);
      delete sv;
      return DP_ERR_CUDA;
    }
    sv->streams.push_back(s);
  }
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return DP_OK;
}

dp_status dp_server_add_cell(dp_server_t sv, const dp_plan_desc *desc, const void *H,
                             int *cell_id) {
  if (!sv || !desc || !cell_id || !H || !a16(H)) return DP_ERR_INVALID_ARG;
  const dp_plan_desc &d = *desc;
  if (d.U < 1 || d.U > 64 || d.B < 1 || d.B > 4096 || d.C < 1 || d.C > d.B || d.n_sc < 1 ||
      d.K < 1 || d.K > 64 || (d.mode != DP_ZF && d.mode != DP_WF && d.mode != DP_FDWF && d.mode != DP_MRT) ||
      (d.prec != DP_FP32 && d.prec != DP_BF16 && d.prec != DP_FP16) || !dp::refine_valid(d.refine) ||
      !(d.rho2 > 0.f) || !(d.Es > 0.f) || !(d.N0 >= 0.f) || !(d.tau >= 0.f))
    return DP_ERR_INVALID_ARG;
  std::vector<float2> ckr;
  if (!dp::cluster_power_table(d.mode == DP_FDWF, d.cluster_power, d.C, d.rho2, d.tau, d.U,
                               d.N0, ckr))
    return DP_ERR_INVALID_ARG;
  Cell c;
  c.d = d;
  c.d.cluster_power = nullptr;  // the table goes to c.d_ckr
  c.off.assign(d.C + 1, 0);
  for (int k = 0; k < d.C; ++k) {
    const int bc = d.cluster_sizes ? d.cluster_sizes[k] : (d.B % d.C ? -1 : d.B / d.C);
    if (bc < 1) return DP_ERR_PARTITION;
    c.off[k + 1] = c.off[k] + bc;
  }
  if (c.off[d.C] != d.B) return DP_ERR_PARTITION;
  int minbc = d.B, maxbc = 0;
  for (int k = 0; k < d.C; ++k) {
    minbc = std::min(minbc, c.off[k + 1] - c.off[k]);
    maxbc = std::max(maxbc, c.off[k + 1] - c.off[k]);
  }
  if ((d.mode == DP_ZF || (d.mode == DP_WF && d.N0 == 0.f)) && d.B < d.U) return DP_ERR_UNSUPPORTED;
  if (d.mode == DP_FDWF && (double)d.tau * d.U * d.N0 * d.C / d.rho2 == 0.0 && minbc < d.U)
    return DP_ERR_UNSUPPORTED;
  c.d.cluster_sizes = nullptr;
  c.UP = dp::padded_users(d.U);
  c.nsys = d.mode == DP_FDWF ? d.C : 1;
  c.maxrows = d.mode == DP_FDWF ? maxbc : d.B;
  if (d.mode == DP_FDWF) {
    int maxsmall = 0, nsmall = 0;
    for (int k = 0; k < d.C; ++k) {
      const int bc = c.off[k + 1] - c.off[k];
      if (bc < d.U && bc <= 32) {
        ++nsmall;
        maxsmall = std::max(maxsmall, bc);
      }
    }
    c.has_small = nsmall > 0;
    c.all_small = nsmall == d.C;
    c.bcp = dp::fd_small_bcp(maxsmall);
  }
  c.tc = d.prec != DP_FP32 && dp::tc_supported(c.UP);
  c.fused = !c.tc && dp::fused_smem_bytes(c.UP, c.maxrows, d.K) != 0;
  c.H = H;
  c.x_bytes = sizeof(float2) * (size_t)d.n_sc * d.K * d.B;
  c.st_bytes = sizeof(int) * (size_t)d.n_sc * c.nsys;
  if (c.x_bytes + c.st_bytes + 512 > sv->arena.bytes()) return DP_ERR_OOM;
  std::lock_guard<std::mutex> lk(sv->mu);
  const size_t off_bytes = (sizeof(int) * c.off.size() + 15) / 16 * 16;
  if (cudaSetDevice(sv->cfg.device) != cudaSuccess ||
      cudaMalloc(&c.d_off, off_bytes + sizeof(float2) * ckr.size()) != cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_OOM;
  }
  cudaMemcpy(c.d_off, c.off.data(), sizeof(int) * c.off.size(), cudaMemcpyHostToDevice);
  if (!ckr.empty()) {
    c.d_ckr = reinterpret_cast<float2 *>(reinterpret_cast<char *>(c.d_off) + off_bytes);
    cudaMemcpy(c.d_ckr, ckr.data(), sizeof(float2) * ckr.size(), cudaMemcpyHostToDevice);
  }
  c.cached = sv->cfg.cache_solve != 0 && !c.all_small;
  // the streaming FP32 form keeps G and z per cell, so its requests stay in
  // order on the cell's stream; every other form may overlap
  c.overlap = c.cached || c.tc || c.fused;
  const size_t ns = (size_t)d.n_sc * c.nsys;
  if (c.cached) {
    c.w_bytes = sizeof(float2) * ns * d.K * d.U + sizeof(float) * ns;
    if (c.x_bytes + c.st_bytes + c.w_bytes + 768 > sv->arena.bytes()) {
      cudaFree(c.d_off);
      return DP_ERR_OOM;
    }
  }
  if (c.cached || !c.overlap) {
    bool ok = cudaMalloc(&c.w_G, sizeof(float2) * ns * d.U * d.U) == cudaSuccess;
    if (ok && !c.cached)
      ok = cudaMalloc(&c.w_Z, sizeof(float2) * ns * d.K * d.U) == cudaSuccess &&
           cudaMalloc(&c.w_scale, sizeof(float) * ns) == cudaSuccess;
    if (ok && c.cached)
      ok = cudaMalloc(&c.c_T, sizeof(float2) * ns * d.U * d.U) == cudaSuccess &&
           cudaMalloc(&c.c_scale, sizeof(float) * ns) == cudaSuccess &&
           cudaMalloc(&c.c_st, sizeof(int) * ns) == cudaSuccess &&
           cudaStreamCreateWithFlags(&c.c_stream, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&c.c_ready, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaFree(c.d_off);
      cudaFree(c.w_G);
      cudaFree(c.w_Z);
      cudaFree(c.w_scale);
      cudaFree(c.c_T);
      cudaFree(c.c_scale);
      cudaFree(c.c_st);
      if (c.c_stream) cudaStreamDestroy(c.c_stream);
      return DP_ERR_OOM;
    }
  }
  c.stream = (int)(sv->cells.size() % sv->streams.size());
  *cell_id = (int)sv->cells.size();
  sv->cells.push_back(c);
  return DP_OK;
}

dp_status dp_server_set_channel(dp_server_t sv, int cell, const void *H) {
  if (!sv || !H || !a16(H)) return DP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (cell < 0 || cell >= (int)sv->cells.size()) return DP_ERR_INVALID_ARG;
  sv->cells[cell].H = H;
  sv->cells[cell].c_H = nullptr;  // the cached solve belongs to the old channel
  return DP_OK;
}

dp_status dp_server_submit(dp_server_t sv, int cell, const void *S, unsigned long long *req_id) {
  if (!sv || !S || !a16(S)) return DP_ERR_INVALID_ARG;
  Request *r = new (std::nothrow) Request;
  if (!r) return DP_ERR_OOM;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (cell < 0 || cell >= (int)sv->cells.size()) {
      delete r;
      return DP_ERR_INVALID_ARG;
    }
    r->id = sv->next_id++;
    r->cell = cell;
    r->S = S;
    r->H = sv->cells[cell].H;
    r->t_arrival = Clock::now();
    if (!sv->have_first) {
      sv->t_first = r->t_arrival;
      sv->have_first = true;
    }
    sv->all[r->id] = r;
    sv->pending.push_back(r);
    if (req_id) *req_id = r->id;
  }
  sv->cv.notify_all();
  return DP_OK;
}

dp_status dp_server_drain(dp_server_t sv) {
  if (!sv) return DP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv.notify_all();
  sv->cv.wait(lk, [&] { return sv->pending.empty() && sv->inflight.empty(); });
  return sv->error ? DP_ERR_CUDA : DP_OK;
}

dp_status dp_server_result(dp_server_t sv, unsigned long long req_id, void **X, int *status) {
  if (!sv) return DP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(req_id);
  if (it == sv->all.end() || !it->second->done) return DP_ERR_INVALID_ARG;
  Request *r = it->second;
  if (X) *X = r->x_off == SIZE_MAX ? nullptr : sv->arena.ptr(r->x_off);
  if (status) *status = r->status;
  return DP_OK;
}

dp_status dp_server_copy_result(dp_server_t sv, unsigned long long req_id, void *dst, int to_host) {
  if (!sv || !dst) return DP_ERR_INVALID_ARG;
  void *x = nullptr;
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(req_id);
    if (it == sv->all.end() || !it->second->done || it->second->x_off == SIZE_MAX)
      return DP_ERR_INVALID_ARG;
    x = sv->arena.ptr(it->second->x_off);
    bytes = sv->cells[it->second->cell].x_bytes;
  }
  if (cudaSetDevice(sv->cfg.device) != cudaSuccess ||
      cudaMemcpy(dst, x, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice) !=
          cudaSuccess) {
    cudaGetLastError();
    return DP_ERR_CUDA;
  }
  return DP_OK;
}

dp_status dp_server_release(dp_server_t sv, unsigned long long req_id) {
  if (!sv) return DP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(req_id);
    if (it == sv->all.end() || !it->second->done) return DP_ERR_INVALID_ARG;
    Request *r = it->second;
    if (r->x_off != SIZE_MAX) sv->arena.release(r->x_off, sv->cells[r->cell].x_bytes);
    sv->all.erase(it);
    delete r;
  }
  sv->cv.notify_all();
  return DP_OK;
}

dp_status dp_server_replay(dp_server_t sv, int n, const int *cells, const void *const *S,
                           const double *arrival_s, const void *const *H_switch) {
  if (!sv || n < 0 || (n && (!cells || !S || !arrival_s))) return DP_ERR_INVALID_ARG;
  const Clock::time_point t0 = Clock::now();
  for (int i = 0; i < n; ++i) {
    const Clock::time_point due =
        t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
    while (Clock::now() < due) {
    }
    if (H_switch && H_switch[i]) {
      if (dp_status s = dp_server_set_channel(sv, cells[i], H_switch[i])) return s;
    }
    if (dp_status s = dp_server_submit(sv, cells[i], S[i], nullptr)) return s;
  }
  return dp_server_drain(sv);
}

dp_status dp_server_stats(dp_server_t sv, dp_server_stats_t *out) {
  if (!sv || !out) return DP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  dp_server_stats_t s{};
  s.completed = (long long)sv->lat_ms.size();
  s.failed = sv->failures;
  s.subcarriers = sv->subcarriers_done;
  s.p50_ms = percentile(sv->lat_ms, 0.50);
  s.p99_ms = percentile(sv->lat_ms, 0.99);
  s.max_ms = sv->lat_ms.empty() ? 0.0 : *std::max_element(sv->lat_ms.begin(), sv->lat_ms.end());
  double sum = 0;
  for (double v : sv->lat_ms) sum += v;
  s.mean_ms = sv->lat_ms.empty() ? 0.0 : sum / sv->lat_ms.size();
  s.wall_s = sv->have_first ? std::chrono::duration<double>(sv->t_last - sv->t_first).count() : 0.0;
  s.inflight_peak = sv->inflight_peak;
  s.arena_high_water = (long long)sv->arena.high_water();
  *out = s;
  return DP_OK;
}

dp_status dp_server_reset_stats(dp_server_t sv) {
  if (!sv) return DP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->lat_ms.clear();
  sv->subcarriers_done = 0;
  sv->inflight_peak = 0;
  sv->failures = 0;
  sv->have_first = false;
  return DP_OK;
}

dp_status dp_server_destroy(dp_server_t sv) {
  if (!sv) return DP_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->cfg.device);
  for (auto &kv : sv->all) delete kv.second;
  for (auto &c : sv->cells) {
    cudaFree(c.d_off);
    cudaFree(c.w_G);
    cudaFree(c.w_Z);
    cudaFree(c.w_scale);
    cudaFree(c.c_T);
    cudaFree(c.c_scale);
    cudaFree(c.c_st);
    if (c.c_ready) cudaEventDestroy(c.c_ready);
    if (c.c_stream) cudaStreamDestroy(c.c_stream);
  }
  for (auto s : sv->streams) cudaStreamDestroy(s);
  cudaGetLastError();
  delete sv;
  return DP_OK;
}

}  // extern "C"
