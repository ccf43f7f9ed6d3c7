// dp_common.cuh -- device helpers shared by the precoding kernels: complex
// float2 arithmetic, mbarrier / bulk-copy (TMA) wrappers with bounded waits,
// and the parameter blocks the host passes to the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dp {

// Device-side status codes; the values equal the public dp_status ones.
enum : int {
  ST_OK = 0,
  ST_NOT_PD = 6,
  ST_NONFINITE = 7,
  ST_TIMEOUT = 8,
  // internal, never returned: the warp-specialized kernel's mark of a system
  // that the automatic refinement wants; its fix-up launch replaces it
  ST_REFINE = 100,
};

// Automatic precision escalation (reduced-precision path): a system is
// flagged when eps * sens >= kRefineTrigger, with eps the unit roundoff of the
// Gram's 16-bit type (2^-8 BF16, 2^-11 FP16) and sens = ||G||_F ||T||_F / U
// the sensitivity of z to a relative perturbation of G.  The worst relative
// error of the unflagged outputs measured about 0.25 eps sens, so the trigger
// keeps them near 5e-4, half the reduced-precision bar; a flagged system's
// Gram is recomputed in FP32.
constexpr float kRefineTrigger = 2e-3f;

constexpr unsigned FULL = 0xffffffffu;
// Iteration bound of every spin on an mbarrier.  After a few immediate
// retries each iteration also sleeps ~64 ns, so a wait gives up after well
// under a second instead of hanging.
constexpr uint32_t kWaitIters = 1u << 22;
constexpr uint32_t kSpinBeforeSleep = 8;

// ---------------------------------------------------------------- complex ---
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cmac_cj(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
// acc -= a * b
__device__ __forceinline__ void cmsub(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ bool cfinite(float2 a) { return isfinite(a.x) && isfinite(a.y); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ------------------------------------------------------ mbarrier and TMA ---
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy / tensor core) accesses, and the reverse.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 1-D bulk copy global -> shared (the TMA unit's non-tensor form).  dst, src
// 16-byte aligned, bytes a multiple of 16; completion counted on bar.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitIters; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i >= kSpinBeforeSleep) __nanosleep(64);
  }
  return false;
}

// The same bounded wait, which also gives up as soon as *abort_f is set (a
// role of a warp-specialized kernel whose partner role gave up).  Waits that
// guard the kernel's exit -- its own copies and MMAs landing before the CTA
// leaves or frees TMEM -- use mbar_wait, never this form.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *bar, uint32_t parity,
                                             const volatile int *abort_f) {
  for (uint32_t i = 0; i < kWaitIters; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i >= kSpinBeforeSleep) {  // the flag is read once the wait is a long one
      if (*abort_f) return false;
      __nanosleep(64);
    }
  }
  return false;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// CTA-wide wait: one thread polls the barrier, the others park at the CTA
// barrier (no issue slots spent spinning).  Returns false on timeout, the
// same value in every thread.
__device__ __forceinline__ bool mbar_wait_cta(uint64_t *bar, uint32_t parity) {
  bool ok = true;
  if (threadIdx.x == 0) ok = mbar_wait(bar, parity);
  return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------- parameters ----
// One "system" is one regularized U x U problem: a subcarrier in WF/ZF mode
// (all B antennas), or one (subcarrier, cluster) pair in FD-WF mode and for
// the per-cluster Grams.  System s covers subcarrier s / nsys and antenna
// rows [lo, hi) of that subcarrier, where nsys == 1 means [0, B) and
// otherwise [off[g], off[g + 1]) with g = s % nsys.
struct SysDesc {
  int U, B, K, n_sc;
  int nsys;         // systems per subcarrier (1 or C)
  const int *off;   // device, C + 1 cluster offsets
  float kappa;      // regularizer of every system (0 for ZF)
  float rho2_sys;   // power of one system: rho^2, or rho^2 / C in FD-WF
  float Es;
  int tma_ok;       // rows may be fetched with 1-D bulk copies
  int skip_small;   // FD-WF: systems with fewer antennas than users (and at
                    // most 32) are left to the B_c x B_c kernel
  int refine;       // tensor-core path, one step of iterative refinement of z:
                    // 0 never, 1 every system, 2 systems the trigger flags
  int mrt;          // maximum ratio transmission: no inverse, z = s, t = tr(G)
  int dbg_stall_us; // failure injection (tests): the warp-specialized kernel's
                    // MMA issuer first waits this long on a flag that nothing
                    // sets, then gives up as a timed-out wait does; 0: off
  const float2 *ckr;  // FD-WF with per-cluster power (device, nsys entries):
                      // (kappa_c, rho_c^2) of cluster c; NULL: kappa and
                      // rho2_sys for every system
};

// Regularizer and power of system sys (a global system index; its cluster is
// sys % nsys).
__device__ __forceinline__ float sys_kappa(const SysDesc &d, int sys) {
  return d.ckr ? d.ckr[sys % d.nsys].x : d.kappa;
}
__device__ __forceinline__ float sys_rho2(const SysDesc &d, int sys) {
  return d.ckr ? d.ckr[sys % d.nsys].y : d.rho2_sys;
}

// One precoding instance: its systems and its device arrays (H [n_sc][B][U],
// S [n_sc][K][U], X [n_sc][K][B], status [n_sc * nsys], optional scale).
struct InstDesc {
  SysDesc d;
  const float2 *H;
  const float2 *S;
  float2 *X;
  int *status;
  float *scale_out;
};

// Workspace of the split tensor-core form (Gram, solve and apply as three
// launches over one bucket's work items), per work item and system:
// G [UP][UP], z [kmax][UP], scale, status.
struct SplitWs {
  float2 *G;
  float2 *Z;
  float *sc;
  int *st;
  int kmax;
};

// A unit of work of a persistent kernel: systems [sys0, sys0 + nact) of
// instance inst.
struct WorkItem {
  int inst;
  int sys0;
  int nact;
};

// True for a system the B_c x B_c small-cluster kernel handles instead.
__device__ __forceinline__ bool sys_is_small(const SysDesc &d, int nrows) {
  return d.skip_small && d.nsys > 1 && nrows < d.U && nrows <= 32;
}

__device__ __forceinline__ void sys_rows(const SysDesc &d, int g, int &lo, int &hi) {
  if (d.nsys == 1) {
    lo = 0;
    hi = d.B;
  } else {
    lo = __ldg(d.off + g);
    hi = __ldg(d.off + g + 1);
  }
}

}  // namespace dp
