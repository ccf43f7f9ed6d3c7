// dp_internal.h -- host-side declarations shared by the C ABI and the kernel
// translation units (not part of the public interface).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "dp_common.cuh"

namespace dp {

// Users padded to the kernels' granularity (a multiple of 8, at most 64).
inline int padded_users(int U) { return ((U + 7) / 8) * 8; }

// SysDesc::refine from a description's refine field (-1 none, 0 automatic,
// 1 every system) and its precision / mode: refinement concerns the 16-bit
// Gram of the tensor-core path, and MRT has nothing to refine.
inline int refine_mode(int refine, bool fp32, bool mrt) {
  if (fp32 || mrt) return 0;
  return refine == 1 ? 1 : (refine == 0 ? 2 : 0);
}
inline bool refine_valid(int refine) { return refine >= -1 && refine <= 1; }

// FD-WF with per-cluster power (Sec. III-D): from the weights w[0..C) the
// table of (kappa_c, rho_c^2) per cluster, rho_c^2 = rho2 w_c / sum w and
// kappa_c = tau U N0 / rho_c^2 (Eq. (16)).  Equal weights give the uniform
// split rho2 / C bit for bit.  An empty table when w is NULL; false when w is
// given for another mode or a weight is not a positive finite number.
inline bool cluster_power_table(bool fdwf, const float *w, int C, double rho2, double tau,
                                double U, double N0, std::vector<float2> &t) {
  t.clear();
  if (!w) return true;
  if (!fdwf || C < 1) return false;
  double sum = 0.0;
  for (int c = 0; c < C; ++c) {
    if (!(w[c] > 0.f) || !std::isfinite(w[c])) return false;
    sum += w[c];
  }
  if (!std::isfinite(sum)) return false;
  for (int c = 0; c < C; ++c) {
    const double rho2c = rho2 * (double)w[c] / sum;
    t.push_back(make_float2((float)(tau * U * N0 / rho2c), (float)rho2c));
  }
  return true;
}

// CTAs of `kernel` (launched with `threads` threads and `dyn_bytes` of dynamic
// shared memory, each holding `tmem_cols` TMEM columns) that one SM holds at
// once, from the limits themselves: threads, registers (allocated per warp in
// units of 256), shared memory with the per-block reserve, resident blocks,
// and the 512 TMEM columns.  0 if an attribute query fails.
int resident_blocks(const void *kernel, int threads, size_t dyn_bytes, int tmem_cols);

// Antenna rows per shared-memory chunk of the streaming Gram / apply kernels.
int stream_chunk_rows(int UP);

// Dynamic shared memory of the fused kernel for systems of up to maxrows
// antennas; 0 if it cannot fit in one CTA.
size_t fused_smem_bytes(int UP, int maxrows, int K);

// The FP32 path's launchers for one padded user count (defined in
// dp_fp32_impl.cuh, instantiated in dp_fp32_u*.cu).
template <int UP>
struct Fp32Ops {
  static cudaError_t gram(const SysDesc &d, const float2 *H, float2 *Gout, cudaStream_t s);
  static cudaError_t solve(const SysDesc &d, const float2 *Gin, const float2 *S, float2 *Z,
                           float *scale, int *status, cudaStream_t s);
  static cudaError_t apply(const SysDesc &d, const float2 *H, const float2 *Z, const float *scale,
                           float2 *X, cudaStream_t s);
  static cudaError_t fused(const SysDesc &d, int maxrows, const float2 *H, const float2 *S,
                           float2 *X, int *status, float *scale_out, cudaStream_t s);
  static cudaError_t batch_fused(const InstDesc *insts, const WorkItem *items, int n_items,
                                 int *queue, int maxrows, int Kmax, int grid, cudaStream_t s);
  static int blocks(int maxrows, int Kmax);
  static size_t fused_bytes(int maxrows, int K);
};

// The tensor-core group kernel's launchers for one padded user count
// (defined in dp_tc_impl.cuh, instantiated in dp_tc_u*.cu).
template <int UP>
struct TcOps {
  static cudaError_t fused(const SysDesc &d, bool bf16, const float2 *H, const float2 *S,
                           float2 *X, int *status, float *scale_out, cudaStream_t s);
  static cudaError_t batch(bool bf16, const InstDesc *insts, const WorkItem *items, int n_items,
                           int *queue, int Kmax, int grid, cudaStream_t s, const int *fix_list,
                           const int *fix_count, int phase, const SplitWs &ws);
  static int blocks(bool bf16, int Kmax);
  static cudaError_t fixup(const SysDesc &d, bool bf16, const float2 *H, const float2 *S,
                           float2 *X, int *status, const int *fix_list, int *fix_count,
                           int grid, cudaStream_t s);
};

cudaError_t launch_gram(const SysDesc &d, int UP, const float2 *H, float2 *Gout,
                        cudaStream_t s);
cudaError_t launch_reduce(const float2 *Gloc, float2 *G, int C, size_t per, cudaStream_t s);
cudaError_t launch_solve(const SysDesc &d, int UP, const float2 *Gin, const float2 *S, float2 *Z,
                         float *scale, int *status, cudaStream_t s);
cudaError_t launch_apply(const SysDesc &d, int UP, const float2 *H, const float2 *Z,
                         const float *scale, float2 *X, cudaStream_t s);
cudaError_t launch_fused(const SysDesc &d, int UP, int maxrows, const float2 *H, const float2 *S,
                         float2 *X, int *status, float *scale_out, cudaStream_t s);
// Persistent FP32 fused kernel over a work-item queue (one system per item;
// queue must be 0); maxrows / Kmax bound the bucket's systems.
cudaError_t launch_batch_fused(int UP, const InstDesc *insts, const WorkItem *items, int n_items,
                               int *queue, int maxrows, int Kmax, int grid, cudaStream_t s);
int fused_max_blocks_per_sm(int UP, int maxrows, int Kmax);

// Reduced-precision fused path (tensor-core Gram and apply): users padded to <= 64.
bool tc_supported(int UP);
cudaError_t launch_fused_tc(const SysDesc &d, int UP, bool bf16, const float2 *H, const float2 *S,
                            float2 *X, int *status, float *scale_out, cudaStream_t s);
// Systems per work item of the tensor-core path (the CTA's group).
int tc_systems_per_group(int UP);
// Persistent tensor-core kernel over a work-item queue (queue must be 0).
// With fix_count non-NULL it takes only items[fix_list[i]], i < *fix_count
// (the fix-up after the warp-specialized kernel; its CTAs exit at once when
// the count is 0).
// phase: 0 every step in one launch; 1 Gram, 2 solve, 3 apply of the split
// form, through the workspace ws (sized for n_items work items).
cudaError_t launch_batch_tc(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                            int n_items, int *queue, int Kmax, int grid, cudaStream_t s,
                            const int *fix_list = nullptr, const int *fix_count = nullptr,
                            int phase = 0, const SplitWs &ws = SplitWs{});
int tc_max_blocks_per_sm(int UP, bool bf16, int Kmax);
// Warp-specialized persistent form of the same arithmetic (bit-identical),
// for users padded to 8 or 16, 1 <= K <= 16 and bulk-copyable rows.
bool pipe_tc_supported(const SysDesc &d, int UP);
// fix_list / fix_count (may be NULL): with automatic refinement the groups
// (of tc_systems_per_group(UP) systems) holding flagged systems are appended
// there, for launch_fixup_tc: fix_count[0] the entries, fix_count[1] that
// kernel's reader count; both zero before the first launch, and that kernel
// leaves them zero again.
cudaError_t launch_pipe_tc(const SysDesc &d, int UP, bool bf16, const float2 *H, const float2 *S,
                           float2 *X, int *status, float *scale_out, cudaStream_t s,
                           int *fix_list = nullptr, int *fix_count = nullptr);
// The group kernel over those listed groups (grid CTAs; nothing when the
// list is empty), which then empties the list.
cudaError_t launch_fixup_tc(const SysDesc &d, int UP, bool bf16, const float2 *H, const float2 *S,
                            float2 *X, int *status, const int *fix_list, int *fix_count,
                            int grid, cudaStream_t s);
// The same kernel over a batch bucket's work items (groups of up to
// pipe_systems_per_group(UP) systems of one instance), one CTA per SM (grid);
// with automatic refinement the groups holding marked systems are appended
// to fix_list (counter fix_count, zeroed before the launch).
int pipe_systems_per_group(int UP);
cudaError_t launch_batch_pipe_tc(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                                 int n_items, int *fix_list, int *fix_count, int grid,
                                 cudaStream_t s);

// The split form's solve phase for 24..64 padded users with one row of A per
// thread (the blocked Gauss-Jordan of dp_rowsolve.cu; n_sm: SMs of the
// device); same workspace and queue conventions as launch_batch_tc's phase 2,
// the queue counting systems.
bool row_solve_supported(int UP);
cudaError_t launch_solve_rows(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                              int n_items, int *queue, const SplitWs &ws, int n_sm,
                              cudaStream_t s);

// FD-WF clusters with B_c < U (and B_c <= 32) in the B_c x B_c form:
// padded cluster width (8, 16, 32; 0 if none fits) and the launchers.
int fd_small_bcp(int maxbc);
cudaError_t launch_fd_small(const InstDesc &in, int bcp, cudaStream_t s);
cudaError_t launch_batch_fd_small(int bcp, const InstDesc *insts, const WorkItem *items,
                                  int n_items, int *queue, int Kmax, int grid, cudaStream_t s);
int fd_small_max_blocks_per_sm(int bcp, int Kmax);

// Served path's solve cache: T = (G + kappa I)^{-1}, scale and status per
// system from an FP32 Gram (layout of launch_gram), and the per-request
// whitening z = T s with the request's status and scale (0 when failed).
cudaError_t launch_cache_invert(const SysDesc &d, int UP, const float2 *G, float2 *T, float *scale,
                                int *status, cudaStream_t s);
cudaError_t launch_cache_whiten(const SysDesc &d, int UP, const float2 *T, const float *cscale,
                                const int *cstatus, const float2 *S, float2 *Z, float *rscale,
                                int *status, cudaStream_t s);

}  // namespace dp
