// dp_tc_impl.cuh -- the reduced-precision fused precoder (instantiated per
// padded user count by dp_tc_u*.cu; dp_tc.cu dispatches): Gram contraction on the
// 5th-generation tensor cores (tcgen05, BF16 or FP16 inputs, FP32
// accumulation in TMEM), solve in FP32, apply as a split-FP16 tensor-core
// product.
//
// One CTA takes a group of NG = 128 / (2 UP) systems.  The complex Gram of a
// system is one real product: with P = R R^T for R = [Re H; Im H] (2U rows,
// antennas along K), Re G = P11 + P22 and Im G = P21 - P12 (Sec. III-B,
// G = H H^H).  The group's realified rows are stacked into the M = 128 rows
// of one K-major operand that serves as both A and B (D = R R^T, N = 128);
// the block-diagonal blocks of D are the systems' P.  Antennas stream in
// chunks of 64: coalesced 8-byte loads of H straight into registers,
// conversion to BF16/FP16 into a 128-byte-swizzled tile (two tiles alternate
// so that the conversion of chunk c+1 overlaps the MMAs of chunk c), four
// MMAs of K = 16 per chunk accumulating in TMEM.
// Then: TMEM -> shared P -> G, warp-per-system Gauss-Jordan solve in
// registers (Thm. 1, Lemma 1 through tr(T G T), z = A^{-1} s; a CTA solve for
// U > 32), and the apply x_c = scale H_c^H z (tc_apply): 128-antenna tiles of
// H split into FP16 hi / lo parts, z split likewise, three MMAs per K-step
// into TMEM, scaled on the way out.  The 32 KB tile region is reused for P
// and for the apply operands, which keeps three to four CTAs on an SM.
#pragma once

#include "dp_blocks.cuh"
#include "dp_internal.h"
#include "dp_quad.cuh"
#include "dp_tc.cuh"

namespace dp {
namespace {

constexpr int KC = 64;          // antennas per Gram chunk (one 128-byte K-block of 16-bit data)
constexpr int TILE_BYTES = 128 * 128;
constexpr int BOP = 32 * 128;  // bytes of one B operand of the apply (32 rows x 128 B)
constexpr int TMEM_COLS = 128;

template <int UP>
struct TcGeo {
  static constexpr int NG = (128 / (2 * UP)) > 0 ? 128 / (2 * UP) : 1;  // systems per CTA
  static constexpr int RS = Geo<UP>::RS;
  static constexpr int M2 = 2 * UP;
  // one region holds the two Gram tiles, then P, then the apply operands:
  // A hi / lo tiles (128 antennas x 64 16-bit entries) and three B operands
  // (32 symbol rows x 64 entries)
  static constexpr int BOP_BYTES = 32 * 128;
  static constexpr int REGION = 2 * TILE_BYTES + 3 * BOP_BYTES;
  // P blocks padded by one float, or XOR-swizzled when that does not fit
  // small U: the diagonal P blocks, padded by one float or XOR-swizzled;
  // U > 32 (one system per CTA): only rows U..2U of P, padded
  static constexpr bool LARGE = UP > 32;
  static constexpr bool P_PAD = LARGE || (size_t)NG * M2 * (M2 + 1) * 4 <= REGION;
  static constexpr int PS = P_PAD ? M2 + 1 : M2;
  static_assert(P_PAD || (M2 % 32 == 0), "swizzled P needs 32-float rows");
  static_assert(LARGE || (size_t)NG * M2 * PS * 4 <= REGION, "P fits the region");
  static_assert(!LARGE || ((size_t)UP * PS * 4 <= REGION && (size_t)UP * (UP + 4) * 8 <= REGION),
                "half of P, the inverse and its row / column buffers fit the region");
  // realified users per apply K-block (one 128-byte row of 16-bit entries)
  static constexpr int KBLK = (2 * UP + 63) / 64;
  // refinement keeps dz [NG][K][UP] (K <= 64) in the region
  static_assert((size_t)NG * 64 * UP * 8 <= REGION, "dz fits the region");
  static constexpr int MIN_BLOCKS = UP <= 16 ? 3 : 2;  // U > 32: one system, CTA solve
  __device__ static __forceinline__ int p_index(int s, int r, int c) {
    return (s * M2 + r) * PS + (P_PAD ? c : (c ^ (r & 31)));
  }
};

struct TcSmem {
  size_t region, G, S, Z, scale, status, info, bars, tmem, total;
};

template <int UP>
__host__ __device__ TcSmem tc_smem_layout(int K) {
  using T = TcGeo<UP>;
  TcSmem L{};
  size_t o = 0;
  auto take = [&](size_t bytes, size_t align) {
    o = (o + align - 1) / align * align;
    size_t at = o;
    o += bytes;
    return at;
  };
  L.region = take(T::REGION, 1024);
  L.G = take((size_t)T::NG * UP * UP * 8, 16);
  L.S = take((size_t)T::NG * K * UP * 8 + 16, 16);
  L.Z = take((size_t)T::NG * K * UP * 8 + 16, 16);
  L.scale = take((size_t)(T::NG + NT / 32) * 4, 16);
  L.status = take((size_t)T::NG * 4, 16);
  L.info = take((size_t)T::NG * 9 * 4, 16);
  L.bars = take(3 * 8, 8);
  L.tmem = take(4, 4);
  L.total = o + 1024;  // slack to align the dynamic base to 1024 bytes
  return L;
}

// Per-CTA state of the tensor-core path, kept across the groups a persistent
// CTA processes: shared-memory carve-up, TMEM base, and the number of phases
// of each mbarrier consumed so far (every arrival is matched by one wait).
struct TcCtx {
  unsigned char *base;
  TcSmem L;
  uint32_t taddr;
  uint32_t tma_waits;
  uint32_t mma_commits[2];
  uint32_t mma_waits[2];
};

template <int UP>
__device__ __forceinline__ void tc_setup(TcCtx &cx, unsigned char *smem_raw, int Kmax) {
  cx.base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  cx.L = tc_smem_layout<UP>(Kmax);
  cx.tma_waits = 0;
  cx.mma_commits[0] = cx.mma_commits[1] = 0;
  cx.mma_waits[0] = cx.mma_waits[1] = 0;
  uint64_t *bar_tma = reinterpret_cast<uint64_t *>(cx.base + cx.L.bars);
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(cx.base + cx.L.tmem);
  if (threadIdx.x == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_tma + 1, 1);
    mbar_init(bar_tma + 2, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tmem_holder, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  cx.taddr = *tmem_holder;
}

__device__ __forceinline__ void tc_teardown(TcCtx &cx) {
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(cx.taddr, TMEM_COLS);
  }
}

// Wait for the oldest outstanding commit of tile buffer buf (CTA-wide).
__device__ __forceinline__ bool tc_wait_mma(TcCtx &cx, int buf) {
  uint64_t *bar_mma = reinterpret_cast<uint64_t *>(cx.base + cx.L.bars) + 1;
  const bool ok = mbar_wait_cta(bar_mma + buf, cx.mma_waits[buf] & 1);
  ++cx.mma_waits[buf];
  return ok;
}

// ---- apply on the tensor cores ----------------------------------------------
// For the group's systems [0, nact) described in shared memory (first antenna,
// antennas, subcarrier, skip flag, status, scale, z [NG][K][UP]): systems with
// a failed status get zeroed rows, the others x = scale H^H z.
// Per 128-antenna M-tile: D[b][n] = sum_j A[b][j] Bm[n][j] with A[b][2u + r]
// = (Re, Im) H[b][u] and, for symbol q of a chunk of 16, Bm[2q] = (Re z_u,
// Im z_u)_u and Bm[2q + 1] = (Im z_u, -Re z_u)_u, so that D[b][2q] + i
// D[b][2q + 1] = sum_u conj(H[b][u]) z_q[u].  The realified users j run in
// K-blocks of 64 (one 128-byte swizzled row), accumulated in TMEM.  Split
// FP16 keeps ~22 bits: A = A_hi + 2^-11 A_lo, z = z_hi + z_lo, D = A_hi z_hi
// + A_hi z_lo + A_lo (2^-11 z_hi); z is first normalized by a power of two.
template <int UP, bool PF = false>
__device__ bool tc_apply(TcCtx &cx, const SysDesc &d, const float2 *__restrict__ H,
                         float2 *__restrict__ X, int nact, bool ok, const int *only = nullptr) {
  // PF: the next step's A entries are loaded while the current MMAs run (the
  // split form's apply launch, which has the registers for it)
  using T = TcGeo<UP>;
  constexpr int NG = T::NG;
  const TcSmem &L = cx.L;
  unsigned char *base = cx.base;
  const float2 *Zs = reinterpret_cast<const float2 *>(base + L.Z);
  float *sc_s = reinterpret_cast<float *>(base + L.scale);
  const int *st_s = reinterpret_cast<const int *>(base + L.status);
  const int *lo_s = reinterpret_cast<const int *>(base + L.info);
  const int *nr_s = lo_s + NG, *n_s = nr_s + NG, *sk_s = n_s + NG;
  uint64_t *bar_mma = reinterpret_cast<uint64_t *>(base + L.bars) + 1;
  const uint32_t taddr = cx.taddr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int U = d.U, K = d.K;
  unsigned char *a_hi = base + L.region;
  unsigned char *a_lo = a_hi + TILE_BYTES;
  unsigned char *b_op = a_hi + 2 * TILE_BYTES;  // hi, lo, hi * 2^-11
  const uint32_t a_hi_u = smem_u32(a_hi), a_lo_u = smem_u32(a_lo), b_u = smem_u32(b_op);
  const uint32_t idesc_ap = tc::idesc_f16(128, 32, false);
  for (int s = 0; s < nact && ok; ++s) {
    if (sk_s[s] || nr_s[s] == 0 || (only && !only[s])) continue;
    float2 *Xn = X + (size_t)n_s[s] * K * d.B + lo_s[s];
    if (st_s[s] != ST_OK) {
      zero_rows<UP>(nr_s[s], K, X + (size_t)n_s[s] * K * d.B, d.B, lo_s[s], tid);
      continue;
    }
    const float2 *zs = Zs + s * K * UP;
    // power-of-two normalization of z for the FP16 range
    float zmax = 0.f;
    for (int e = tid; e < K * UP; e += NT)
      if (e % UP < U) zmax = fmaxf(zmax, fmaxf(fabsf(zs[e].x), fabsf(zs[e].y)));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(FULL, zmax, o));
    __syncthreads();
    if (lane == 0) sc_s[NG + warp] = zmax;  // scratch slots after the scales
    __syncthreads();
    float zm = 0.f;
    for (int w = 0; w < NT / 32; ++w) zm = fmaxf(zm, sc_s[NG + w]);
    int zexp = 0;
    if (zm > 0.f) frexpf(zm, &zexp);        // zm = f 2^zexp, f in [0.5, 1)
    const float zn = ldexpf(1.f, -zexp);    // z * zn in (-1, 1)
    const float out_scale = ldexpf(sc_s[s], zexp);
    const float2 *hsys = H + ((size_t)n_s[s] * d.B + lo_s[s]) * U;
    // The thread's A-tile entries of one step (128-antenna tile m0, 64-entry
    // user block kb): items e = tid + NT i, row e / 8, users 4 (e % 8)..+3 of
    // the block.  The next step's are loaded while the current one's MMAs run.
    constexpr int AIT = 128 * 8 / NT;
    float2 pre[AIT][4];
    auto load_item = [&](int i, int m0, int kb) {
      const int mrows = min(128, nr_s[s] - m0), ent = min(64, 2 * UP - 64 * kb);
      const int e = tid + NT * i, r = e >> 3, c8 = e & 7;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int u = 32 * kb + 4 * c8 + j;
        pre[i][j] = (8 * c8 < ent && r < mrows && u < U)
                        ? __ldg(hsys + (size_t)(m0 + r) * U + u)
                        : make_float2(0.f, 0.f);
      }
    };
    auto load_a = [&](int m0, int kb) {
#pragma unroll
      for (int i = 0; i < AIT; ++i) load_item(i, m0, kb);
    };
    if constexpr (PF) load_a(0, 0);
    for (int q0 = 0; q0 < K && ok; q0 += 16) {
      const int nq = min(16, K - q0);
      for (int m0 = 0; m0 < nr_s[s] && ok; m0 += 128) {
        const int mrows = min(128, nr_s[s] - m0);
        for (int kb = 0; kb < T::KBLK && ok; ++kb) {
          const int ent = min(64, 2 * UP - 64 * kb);  // realified entries in this block
          const int ksteps = (ent + 15) / 16;
          __syncthreads();  // the previous MMAs and readout are done with A, B, TMEM
          // B operands: 32 rows x 8 chunks of 8 entries (4 users x Re/Im)
          for (int e = tid; e < 32 * 8; e += NT) {
            const int row = e >> 3, c8 = e & 7;
            const int q = row >> 1, im = row & 1;
            float v[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int u = 32 * kb + 4 * c8 + j;
              float2 z = make_float2(0.f, 0.f);
              if (q < nq && u < U && 8 * c8 < ent) z = zs[(q0 + q) * UP + u];
              z.x *= zn;
              z.y *= zn;
              v[2 * j] = im ? z.y : z.x;
              v[2 * j + 1] = im ? -z.x : z.y;
            }
            uint4 hi, lo, hs;
            uint32_t *ph = &hi.x, *pl = &lo.x, *ps = &hs.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const __half2 h2 = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
              const float2 hf = __half22float2(h2);
              const __half2 l2 = __floats2half2_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
              const __half2 s2 = __floats2half2_rn(hf.x * 0x1p-11f, hf.y * 0x1p-11f);
              ph[j] = *reinterpret_cast<const uint32_t *>(&h2);
              pl[j] = *reinterpret_cast<const uint32_t *>(&l2);
              ps[j] = *reinterpret_cast<const uint32_t *>(&s2);
            }
            const uint32_t off = tc::sw128_offset(row, c8);
            *reinterpret_cast<uint4 *>(b_op + off) = hi;
            *reinterpret_cast<uint4 *>(b_op + BOP + off) = lo;
            *reinterpret_cast<uint4 *>(b_op + 2 * BOP + off) = hs;
          }
          // A tiles: rows = antennas, 16-byte chunk c8 = users 4c8..4c8+3 of
          // the block; zero beyond the block's entries and the tile's rows
#pragma unroll
          for (int i = 0; i < AIT; ++i) {
            if constexpr (!PF) load_item(i, m0, kb);
            const int e = tid + NT * i, r = e >> 3, c8 = e & 7;
            uint4 hi = make_uint4(0, 0, 0, 0), lo = make_uint4(0, 0, 0, 0);
            if (8 * c8 < ent) {
              uint32_t *ph = &hi.x, *pl = &lo.x;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float2 h = pre[i][j];
                const __half2 h2 = __floats2half2_rn(h.x, h.y);
                const float2 hf = __half22float2(h2);
                const __half2 l2 = __floats2half2_rn((h.x - hf.x) * 0x1p11f,
                                                     (h.y - hf.y) * 0x1p11f);
                ph[j] = *reinterpret_cast<const uint32_t *>(&h2);
                pl[j] = *reinterpret_cast<const uint32_t *>(&l2);
              }
            }
            const uint32_t off = tc::sw128_offset(r, c8);
            *reinterpret_cast<uint4 *>(a_hi + off) = hi;
            *reinterpret_cast<uint4 *>(a_lo + off) = lo;
          }
          // the next step's A entries: next user block, else next tile, else
          // the first tile again for the next 16 symbols
          if constexpr (PF) {
            if (kb + 1 < T::KBLK) load_a(m0, kb + 1);
            else if (m0 + 128 < nr_s[s]) load_a(m0 + 128, 0);
            else if (q0 + 16 < K) load_a(0, 0);
          }
          fence_proxy_async_smem();
          __syncthreads();
          if (tid == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < ksteps; ++kk) {
              const uint32_t ko = kk * 32;
              tc::mma_f16(taddr, tc::desc_kmajor_sw128(a_hi_u + ko),
                          tc::desc_kmajor_sw128(b_u + ko), idesc_ap, kb > 0 || kk > 0);
              tc::mma_f16(taddr, tc::desc_kmajor_sw128(a_hi_u + ko),
                          tc::desc_kmajor_sw128(b_u + BOP + ko), idesc_ap, true);
              tc::mma_f16(taddr, tc::desc_kmajor_sw128(a_lo_u + ko),
                          tc::desc_kmajor_sw128(b_u + 2 * BOP + ko), idesc_ap, true);
            }
            tc::commit(bar_mma);
          }
          ++cx.mma_commits[0];
          ok = tc_wait_mma(cx, 0);
          tc::fence_after_sync();
        }
        if (!ok) break;
        if (warp < 4) {
          float v[32];
          tc::tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16), v);
          const int r = 32 * warp + lane;
          if (r < mrows) {
            float2 *xc = Xn + m0 + r;
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (q < nq) xc[(size_t)(q0 + q) * d.B] = make_float2(v[2 * q] * out_scale,
                                                                   v[2 * q + 1] * out_scale);
          }
        }
        tc::fence_before_sync();
      }
    }
  }
  __syncthreads();
  return ok;
}

// Systems [sys0, sys0 + nact) of one instance (nact <= NG): Gram on the tensor
// cores, solve, apply.  Returns false if a bounded wait gave up (the
// systems' outputs are then zeroed and their status set to ST_TIMEOUT).
// Phases of tc_group: PH_FUSED runs every step; the split form runs the
// Gram (PH_GRAM: G and its finiteness to the workspace), the solve (PH_SOLVE:
// G from the workspace; z, scale and status back to it) and the apply
// (PH_APPLY) as three launches over the same work items, so that the solve
// -- ALU-bound for many users -- does not hold the streaming phases.
enum : int { PH_FUSED = 0, PH_GRAM = 1, PH_SOLVE = 2, PH_APPLY = 3 };

template <int UP, bool BF16, int PH = PH_FUSED>
__device__ bool tc_group(TcCtx &cx, const InstDesc &in, int sys0, int nact,
                         const SplitWs *ws = nullptr, int it = 0) {
  using T = TcGeo<UP>;
  constexpr int NG = T::NG, M2 = T::M2;
  const SysDesc &d = in.d;
  const float2 *__restrict__ H = in.H;
  const float2 *__restrict__ S = in.S;
  float2 *__restrict__ X = in.X;
  int *__restrict__ status = in.status;
  float *__restrict__ scale_out = in.scale_out;
  const TcSmem &L = cx.L;
  unsigned char *base = cx.base;
  unsigned char *tiles = base + L.region;
  float *P = reinterpret_cast<float *>(base + L.region);
  float2 *Gs = reinterpret_cast<float2 *>(base + L.G);
  float2 *Ss = reinterpret_cast<float2 *>(base + L.S);
  float2 *Zs = reinterpret_cast<float2 *>(base + L.Z);
  float *sc_s = reinterpret_cast<float *>(base + L.scale);
  int *st_s = reinterpret_cast<int *>(base + L.status);
  int *lo_s = reinterpret_cast<int *>(base + L.info);  // first antenna of each system
  int *nr_s = lo_s + NG;                                // antennas of each system
  int *n_s = nr_s + NG;                                 // subcarrier of each system
  int *sk_s = n_s + NG;                                 // system left to another kernel
  int *rf_s = sk_s + NG;                                // refinement steps of the system
  float *sens_s = reinterpret_cast<float *>(rf_s + NG);  // its sensitivity estimate
  int *act_s = rf_s + 2 * NG;                            // refined in the current step
  int *es_s = rf_s + 3 * NG;                             // escalated to an FP32 Gram
  int *nes_s = rf_s + 4 * NG;                            // not escalated
  uint64_t *bar_tma = reinterpret_cast<uint64_t *>(base + L.bars);
  const uint32_t taddr = cx.taddr;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int U = d.U, K = d.K;

  // ---- systems of the group, symbols -----------------------------------------
  __syncthreads();  // the previous group is done with every shared buffer
  if (tid < NG) {
    int lo = 0, hi = 0, n = 0, skip = 1;
    if (tid < nact) {
      const int sys = sys0 + tid;
      n = sys / d.nsys;
      sys_rows(d, sys - n * d.nsys, lo, hi);
      skip = sys_is_small(d, hi - lo);  // the B_c x B_c kernel's system
      if (skip) hi = lo;
    }
    lo_s[tid] = lo;
    nr_s[tid] = hi - lo;
    n_s[tid] = n;
    sk_s[tid] = skip;
  }
  // rows of the tiles above the group's realified rows stay zero
  if constexpr (NG * M2 < 128) {
    constexpr int FREE = (128 - NG * M2) * 8;
    for (int e = tid; e < 2 * FREE; e += NT) {
      const int t = e / FREE, rem = e - t * FREE;
      const int m = NG * M2 + rem / 8, g8 = rem % 8;
      *reinterpret_cast<uint4 *>(tiles + t * TILE_BYTES + tc::sw128_offset(m, g8)) =
          make_uint4(0, 0, 0, 0);
    }
  }
  __syncthreads();
  int kmax = 0;
  for (int s = 0; s < NG; ++s) kmax = max(kmax, nr_s[s]);
  const int nchunks = (kmax + KC - 1) / KC;
  if constexpr (PH == PH_FUSED || PH == PH_SOLVE) {
    for (int e = tid; e < NG * K * UP; e += NT) {
      const int s = e / (K * UP), r = e - s * K * UP, k = r / UP, u = r - k * UP;
      float2 v = make_float2(0.f, 0.f);
      if (s < nact && u < U) v = __ldg(S + ((size_t)n_s[s] * K + k) * U + u);
      Ss[e] = v;
    }
  }
  if constexpr (PH == PH_APPLY) {
    // z, scale and status of the group's systems from the workspace
    for (int e = tid; e < NG * K * UP; e += NT) {
      const int s = e / (K * UP), r = e - s * K * UP;
      Zs[e] = ws->Z[((size_t)it * NG + s) * ws->kmax * UP + r];
    }
    if (tid < NG) {
      sc_s[tid] = ws->sc[it * NG + tid];
      st_s[tid] = ws->st[it * NG + tid];
    }
    fence_proxy_async_smem();
    __syncthreads();
    return tc_apply<UP, true>(cx, d, H, X, nact, true);
  }
  bool ok = true;
  if constexpr (PH == PH_FUSED || PH == PH_GRAM) {

  // ---- Gram mainloop --------------------------------------------------------
  const uint32_t idesc = tc::idesc_f16(128, 128, BF16);
  const uint32_t tiles_u32 = smem_u32(tiles);
  uint64_t *bar_mma = bar_tma + 1;
  // item = (antenna octet g8, system s, user u): eight coalesced 8-byte
  // loads, Re into tile row s*2UP + u, Im into row s*2UP + UP + u.  A
  // thread's items of chunk c + 1 are loaded into registers while chunk c is
  // converted and its MMAs issued.
  constexpr int ITEMS = 8 * NG * UP, IPT = (ITEMS + NT - 1) / NT;
  float2 pre[IPT][8];
  auto load_chunk = [&](int c) {
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int item = tid + q * NT;
      const int u = item % UP, s = (item / UP) % NG, g8 = item / (UP * NG);
      const bool live = item < ITEMS && s < nact && u < U;
      const int left = nr_s[s] - (c * KC + 8 * g8);
      const float2 *src =
          H + ((size_t)n_s[s] * d.B + lo_s[s] + c * KC + 8 * (live ? g8 : 0)) * U + u;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        pre[q][j] = (live && j < left) ? __ldg(src + (size_t)j * U) : make_float2(0.f, 0.f);
    }
  };
  if (nchunks > 0) load_chunk(0);
  for (int c = 0; c < nchunks && ok; ++c) {
    const int buf = c & 1;
    // the MMAs of chunk c - 2 read this tile
    if (c >= 2) ok = tc_wait_mma(cx, buf);
    if (!ok) break;
    unsigned char *tile = tiles + buf * TILE_BYTES;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int item = tid + q * NT;
      if (item >= ITEMS) continue;
      const int u = item % UP, s = (item / UP) % NG, g8 = item / (UP * NG);
      const float2 *v = pre[q];
      uint4 re, im;
      re.x = tc::pack2<BF16>(v[0].x, v[1].x);
      re.y = tc::pack2<BF16>(v[2].x, v[3].x);
      re.z = tc::pack2<BF16>(v[4].x, v[5].x);
      re.w = tc::pack2<BF16>(v[6].x, v[7].x);
      im.x = tc::pack2<BF16>(v[0].y, v[1].y);
      im.y = tc::pack2<BF16>(v[2].y, v[3].y);
      im.z = tc::pack2<BF16>(v[4].y, v[5].y);
      im.w = tc::pack2<BF16>(v[6].y, v[7].y);
      *reinterpret_cast<uint4 *>(tile + tc::sw128_offset(s * M2 + u, g8)) = re;
      *reinterpret_cast<uint4 *>(tile + tc::sw128_offset(s * M2 + UP + u, g8)) = im;
    }
    if (c + 1 < nchunks) load_chunk(c + 1);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < KC / 16; ++kk) {
        const uint64_t desc = tc::desc_kmajor_sw128(tiles_u32 + buf * TILE_BYTES + kk * 32);
        tc::mma_f16(taddr, desc, desc, idesc, c > 0 || kk > 0);
      }
      tc::commit(bar_mma + buf);
    }
    ++cx.mma_commits[buf];
  }
  // drain: wait for every outstanding commit (the last one covers all MMAs)
  for (int b = 0; b < 2 && ok; ++b)
    while (ok && cx.mma_waits[b] < cx.mma_commits[b]) ok = tc_wait_mma(cx, b);
  tc::fence_after_sync();

  if (!ok) {  // report; the caller stops and frees TMEM
    for (int s = 0; s < nact; ++s) {
      if (sk_s[s]) continue;
      zero_rows<UP>(nr_s[s], K, X + (size_t)n_s[s] * K * d.B, d.B, lo_s[s], tid);
      if (tid == 0) {
        status[sys0 + s] = ST_TIMEOUT;
        if (scale_out) scale_out[sys0 + s] = 0.f;
        if constexpr (PH == PH_GRAM) ws->st[it * NG + s] = ST_TIMEOUT;  // the later phases keep it
      }
    }
    return false;
  }

  if constexpr (T::LARGE) {
    // ---- TMEM -> G for one system with U > 32 ------------------------------
    // Re G_mn = P[m][n] + P[U'+m][U'+n], Im G_mn = P[U'+m][n] - P[m][U'+n]
    // (U' = UP): the rows U'..2U' go to shared memory, then lane m combines
    // its own TMEM row m with them.  It stores G_mn as conj into Gs[n][m]
    // (G is Hermitian), so that the lanes of a store write consecutive
    // entries; the solve reads it back the same way.
    float *Pim = P;  // [UP][PS]
    if (warp < 4) {
      const int m = 32 * warp + lane;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        float v[32];
        tc::tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + 32 * cc, v);
        if (m >= UP && m < M2) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = 32 * cc + j;
            if (n < M2) Pim[(m - UP) * T::PS + n] = v[j];
          }
        }
      }
    }
    for (int e = tid; e < UP * UP; e += NT) Gs[e] = make_float2(0.f, 0.f);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp < 4) {
      const int m = 32 * warp + lane;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        float v[32];
        tc::tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + 32 * cc, v);
        if (m < U && nact > 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = 32 * cc + j;
            if (n < U) {  // conj: (Re, -Im) with Im's first term P[U'+m][n]
              Gs[n * UP + m].x = v[j] + Pim[m * T::PS + UP + n];
              Gs[n * UP + m].y -= Pim[m * T::PS + n];
            } else if (n >= UP && n < UP + U) {  // Im's second term -P[m][U'+n]
              Gs[(n - UP) * UP + m].y += v[j];
            }
          }
          if (cc == 3) Gs[m * UP + m].y = 0.f;
        }
      }
    }
    tc::fence_before_sync();
  } else {
  // ---- TMEM -> P (the diagonal 2UP x 2UP blocks) ------------------------------
    if (warp < 4) {
      const int m = 32 * warp + lane;
      const int s = m / M2, r = m - s * M2;
  #pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        float v[32];
        tc::tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + 32 * cc, v);
  #pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = 32 * cc + j;
          if (s < NG && n / M2 == s) P[T::p_index(s, r, n - s * M2)] = v[j];
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    // ---- P -> G, row by row ------------------------------------------------------
    for (int e = tid; e < NG * UP * UP; e += NT) {
      const int s = e / (UP * UP), ij = e - s * UP * UP, i = ij / UP, j = ij - i * UP;
      float2 g = make_float2(0.f, 0.f);
      if (s < nact && i < U && j < U) {
        g.x = P[T::p_index(s, i, j)] + P[T::p_index(s, UP + i, UP + j)];
        g.y = (i == j) ? 0.f : P[T::p_index(s, UP + i, j)] - P[T::p_index(s, i, UP + j)];
      }
      Gs[e] = g;
    }
  }
  }  // PH_FUSED, PH_GRAM
  if constexpr (PH == PH_SOLVE) {  // G and its finiteness from the workspace
    for (int e = tid; e < NG * UP * UP; e += NT) Gs[e] = ws->G[(size_t)it * NG * UP * UP + e];
    if (tid < NG) st_s[tid] = ws->st[it * NG + tid];
  }
  __syncthreads();
  // per-system finiteness of G (covers H) and of the symbols
  if (warp < NG) {
    bool fin = true;
    if constexpr (PH != PH_SOLVE)
      for (int e = lane; e < UP * UP; e += 32) fin = fin && cfinite(Gs[warp * UP * UP + e]);
    if constexpr (PH != PH_GRAM)
      for (int e = lane; e < K * UP; e += 32) fin = fin && cfinite(Ss[warp * K * UP + e]);
    fin = __all_sync(FULL, fin);
    if constexpr (PH == PH_SOLVE) {  // the Gram phase's verdict stands
      if (lane == 0 && st_s[warp] == ST_OK && !fin) st_s[warp] = ST_NONFINITE;
    } else {
      if (lane == 0) st_s[warp] = fin ? ST_OK : ST_NONFINITE;
    }
  }
  __syncthreads();
  if constexpr (PH == PH_GRAM) {  // G and its finiteness to the workspace
    for (int e = tid; e < NG * UP * UP; e += NT) ws->G[(size_t)it * NG * UP * UP + e] = Gs[e];
    if (tid < NG) ws->st[it * NG + tid] = st_s[tid];
    return true;
  }

  const bool refine = d.refine && !d.mrt;
  if constexpr (UP >= 24) {
    // ---- solve: the whole CTA in the quad-row layout (dp_quad.cuh) ------------
    // With refinement T = A^{-1} replaces G in Gs (the residual is formed
    // from H itself).  The quad solve reads G in conjugate-transposed order,
    // which for U > 32 is how the TMEM readout above stored it; for U <= 32
    // the readout stored G itself, and G is Hermitian.
    quad_solve<UP>(Gs, Ss, Zs, st_s, sc_s, sk_s, nact, d, sys0, d.Es, U, K,
                   d.mrt != 0, kLemmaMaxRatioLP, reinterpret_cast<float2 *>(base + L.region),
                   sc_s + NG, refine ? Gs : nullptr, d.refine == 2 ? sens_s : nullptr, tid);
  } else {
  // ---- solve: one warp per system --------------------------------------------
    if (warp < nact) {
      float sc = 0.f, sens = 0.f;
      const int st = warp_solve<UP>(Gs + warp * UP * UP, Ss + warp * K * UP, Zs + warp * K * UP, UP,
                                    sys_kappa(d, sys0 + warp), sys_rho2(d, sys0 + warp), d.Es, U,
                                    K, lane, st_s[warp] == ST_OK,
                                    sc, d.mrt != 0, d.refine == 2 ? &sens : nullptr);
      if (lane == 0) {
        st_s[warp] = st;
        sc_s[warp] = sc;
        sens_s[warp] = sens;
      }
    }
  }
  // What the reduced-precision result gets.  refine = 1: one refinement step
  // of z for every system.  refine = 2: a system the sensitivity estimate
  // flags (eps sens >= kRefineTrigger) is escalated -- its Gram recomputed in
  // FP32 and solved again -- because refining z leaves the precoding factor's
  // error (t comes from the 16-bit inverse), which is of the same order.
  __syncthreads();
  if (tid < NG) {
    constexpr float eps = BF16 ? 0x1p-8f : 0x1p-11f;
    int steps = 0, esc = 0;
    if (refine && tid < nact && !sk_s[tid] && st_s[tid] == ST_OK) {
      if (d.refine == 1) steps = 1;
      else if (eps * sens_s[tid] >= kRefineTrigger) esc = 1;
    }
    rf_s[tid] = steps;
    es_s[tid] = esc;
    nes_s[tid] = !esc;
  }
  fence_proxy_async_smem();
  const bool any_rf = __syncthreads_or(tid < NG && rf_s[tid]) != 0;
  const bool any_es = __syncthreads_or(tid < NG && es_s[tid]) != 0;

  if constexpr (PH == PH_FUSED) ok = tc_apply<UP>(cx, d, H, X, nact, ok, any_es ? nes_s : nullptr);

  if (any_es && ok) {
    // ---- escalation: FP32 Gram (SIMT, register-tiled as the FP32 path's),
    // then the solve and the apply again, for the escalated systems only
    constexpr int RS = Geo<UP>::RS;
    constexpr int CH0 = (int)(T::REGION / (RS * 4));
    constexpr int CH = CH0 > 128 ? 128 : CH0;
    float *Hs = reinterpret_cast<float *>(base + L.region);
    for (int s = 0; s < nact; ++s) {
      if (!es_s[s]) continue;
      const float2 *hn = H + (size_t)n_s[s] * d.B * U;
      GramAcc<UP> gacc;
      gacc.init(tid);
      __syncthreads();  // the region is free (previous system, apply)
      zero_row_pads<UP>(Hs, CH, U, tid);
      for (int r0 = 0; r0 < nr_s[s]; r0 += CH) {
        const int nrows = min(CH, nr_s[s] - r0);
        __syncthreads();
        fetch_rows<UP>(Hs, hn, lo_s[s] + r0, nrows, U, false, nullptr, tid);
        __syncthreads();
        gacc.accumulate(Hs, nrows);
      }
      gacc.finish(Gs + s * UP * UP, tid);
    }
    __syncthreads();
    if constexpr (UP >= 24) {
      quad_solve<UP>(Gs, Ss, Zs, st_s, sc_s, nes_s, nact, d, sys0, d.Es, U, K,
                     d.mrt != 0, kLemmaMaxRatio, reinterpret_cast<float2 *>(base + L.region),
                     sc_s + NG, nullptr, nullptr, tid);
    } else {
      if (warp < nact && es_s[warp]) {
        float sc = 0.f;
        const int st = warp_solve<UP>(Gs + warp * UP * UP, Ss + warp * K * UP,
                                      Zs + warp * K * UP, UP, sys_kappa(d, sys0 + warp),
                                      sys_rho2(d, sys0 + warp), d.Es, U, K, lane, true, sc,
                                      d.mrt != 0);
        if (lane == 0) {
          st_s[warp] = st;
          sc_s[warp] = sc;
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if constexpr (PH == PH_FUSED) ok = tc_apply<UP>(cx, d, H, X, nact, ok, es_s);
  }
  if constexpr (PH == PH_SOLVE) {  // z, scale and status to the workspace
    __syncthreads();
    for (int e = tid; e < NG * K * UP; e += NT) {
      const int s = e / (K * UP), r = e - s * K * UP;
      ws->Z[((size_t)it * NG + s) * ws->kmax * UP + r] = Zs[e];
    }
    if (tid < NG) {
      ws->sc[it * NG + tid] = sc_s[tid];
      ws->st[it * NG + tid] = (tid < nact && !sk_s[tid]) ? st_s[tid] : ST_OK;
    }
    if (tid < nact && !sk_s[tid]) {
      status[sys0 + tid] = st_s[tid];
      if (scale_out) scale_out[sys0 + tid] = st_s[tid] == ST_OK ? sc_s[tid] : 0.f;
    }
    return true;
  }

  for (int step = 1; PH == PH_FUSED && any_rf && ok && step <= 3; ++step) {
    if (tid < NG) act_s[tid] = (tid < nact && rf_s[tid] >= step) ? 1 : 0;
    if (!__syncthreads_or(tid < NG && act_s[tid])) break;
    // ---- a step of iterative refinement of z ---------------------------------
    // With the exact H in FP32: r = s - (H H^H z + kappa z), where H^H z is
    // the last apply's X / scale; dz = A_lp^{-1} r with the low-precision
    // A_lp = G_lp + kappa I (U <= 16: A_lp rebuilt from G in Gs; U >= 24: its
    // inverse T kept in Gs); z += dz; apply again.
    float2 *Dz = reinterpret_cast<float2 *>(base + L.region);  // [NG][K][UP]
    for (int s = 0; s < nact; ++s) {
      if (!act_s[s]) continue;
      const float inv = 1.f / sc_s[s];
      const float2 *hs = H + ((size_t)n_s[s] * d.B + lo_s[s]) * U;
      const float2 *xs = X + (size_t)n_s[s] * K * d.B + lo_s[s];  // written above: plain loads
      float2 *ss = Ss + s * K * UP;
      const float2 *zz = Zs + s * K * UP;
      bool fin = true;
      for (int e = tid; e < K * UP; e += NT) {
        const int k = e / UP, u = e - k * UP;
        if (u >= U) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int b = 0; b < nr_s[s]; ++b)
          cmac(acc, __ldg(hs + (size_t)b * U + u), xs[(size_t)k * d.B + b]);
        const float2 z0 = zz[e];
        // s itself from the input (Ss holds the previous step's residual)
        float2 r = __ldg(S + ((size_t)n_s[s] * K + k) * U + u);
        const float ks = sys_kappa(d, sys0 + s);
        r.x -= acc.x * inv + ks * z0.x;
        r.y -= acc.y * inv + ks * z0.y;
        fin = fin && cfinite(r);
        ss[e] = r;
      }
      const int okr = __syncthreads_and(fin);
      if (tid == 0 && !okr) {  // a non-finite residual stops this system's refinement
        act_s[s] = 0;
        rf_s[s] = 0;
      }
    }
    __syncthreads();
    if constexpr (UP >= 24) {
      // dz[k][i] = sum_j T_ij r_k[j], T Hermitian: conj(T_ji) along the
      // lanes' consecutive i
      for (int e = tid; e < NG * K * UP; e += NT) {
        const int s = e / (K * UP), r = e - s * K * UP, k = r / UP, i = r - k * UP;
        float2 acc = make_float2(0.f, 0.f);
        if (s < nact && act_s[s] && i < U) {
          const float2 *Tm = Gs + (size_t)s * UP * UP;
          const float2 *rk = Ss + (size_t)s * K * UP + k * UP;
          for (int j = 0; j < U; ++j) cmac_cj(acc, Tm[j * UP + i], rk[j]);
        }
        Dz[e] = acc;
      }
    } else {
      if (warp < nact && act_s[warp]) {
        float unused;
        warp_solve<UP>(Gs + warp * UP * UP, Ss + warp * K * UP, Dz + warp * K * UP, UP,
                       sys_kappa(d, sys0 + warp), sys_rho2(d, sys0 + warp), d.Es, U, K, lane,
                       true, unused);
      }
    }
    __syncthreads();
    for (int e = tid; e < NG * K * UP; e += NT) {
      const int s = e / (K * UP), u = e % UP;
      if (s < nact && act_s[s] && u < U) {
        Zs[e].x += Dz[e].x;
        Zs[e].y += Dz[e].y;
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    ok = tc_apply<UP>(cx, d, H, X, nact, ok, act_s);
  }

  if (!ok) {
    for (int s = 0; s < nact; ++s) {
      if (sk_s[s]) continue;
      zero_rows<UP>(nr_s[s], K, X + (size_t)n_s[s] * K * d.B, d.B, lo_s[s], tid);
      if (tid == 0) st_s[s] = ST_TIMEOUT;
    }
  }
  __syncthreads();
  if (tid < nact && !sk_s[tid]) {
    status[sys0 + tid] = st_s[tid];
    if (scale_out) scale_out[sys0 + tid] = st_s[tid] == ST_OK ? sc_s[tid] : 0.f;
  }
  return ok;
}


template <int UP, bool BF16>
__global__ void __launch_bounds__(NT, TcGeo<UP>::MIN_BLOCKS)
    k_fused_tc(InstDesc in, int Kmax) {
  extern __shared__ unsigned char smem_raw[];
  const int total = in.d.n_sc * in.d.nsys;
  const int sys0 = blockIdx.x * TcGeo<UP>::NG;
  const int nact = min(TcGeo<UP>::NG, total - sys0);
  TcCtx cx;
  tc_setup<UP>(cx, smem_raw, Kmax);
  tc_group<UP, BF16>(cx, in, sys0, nact);
  tc_teardown(cx);
}

// Fix-up after the warp-specialized kernel (automatic precision escalation):
// the groups it listed (fix_list[0 .. *fix_count), group g = systems
// [g NG, g NG + NG)), redone by the group kernel; with an empty list every CTA
// leaves at once.
template <int UP, bool BF16>
__global__ void __launch_bounds__(NT, TcGeo<UP>::MIN_BLOCKS)
    k_fixup_tc(InstDesc in, const int *__restrict__ fix_list, int *fix_count, int Kmax) {
  extern __shared__ unsigned char smem_raw[];
  const int n = *fix_count;
  // the list is emptied for the next call by the last CTA to have read it
  // (fix_count[1] counts the readers), so the caller needs no reset
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(fix_count + 1, 1) == (int)gridDim.x - 1) {
      fix_count[0] = 0;
      fix_count[1] = 0;
    }
  }
  if ((int)blockIdx.x >= n) return;
  const int total = in.d.n_sc * in.d.nsys;
  TcCtx cx;
  tc_setup<UP>(cx, smem_raw, Kmax);
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int sys0 = fix_list[it] * TcGeo<UP>::NG;
    if (!tc_group<UP, BF16>(cx, in, sys0, min(TcGeo<UP>::NG, total - sys0))) break;
  }
  tc_teardown(cx);
}

// Persistent form: CTAs pull work items (groups of systems of any instance of
// this bucket) from an atomic queue until it is empty.
template <int UP, bool BF16, int PH = PH_FUSED>
__global__ void __launch_bounds__(NT, TcGeo<UP>::MIN_BLOCKS)
    k_batch_tc(const InstDesc *__restrict__ insts, const WorkItem *__restrict__ items,
               int n_items, int *__restrict__ queue, int Kmax, const int *__restrict__ fix_list,
               const int *__restrict__ fix_count, SplitWs ws) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int next;
  // fix-up form (automatic refinement after the warp-specialized kernel):
  // only the items that kernel listed
  const int n = fix_count ? *fix_count : n_items;
  if (n == 0) return;
  TcCtx cx;
  tc_setup<UP>(cx, smem_raw, Kmax);
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(queue, 1);
    __syncthreads();
    const int it = next;
    if (it >= n) break;
    const int item = fix_list ? fix_list[it] : it;
    const WorkItem w = items[item];
    if (!tc_group<UP, BF16, PH>(cx, insts[w.inst], w.sys0, w.nact, &ws, item)) break;
  }
  tc_teardown(cx);
}

template <int UP, bool BF16>
cudaError_t launch_tc_t(const SysDesc &d, const float2 *H, const float2 *S, float2 *X,
                        int *status, float *scale_out, cudaStream_t s) {
  const TcSmem L = tc_smem_layout<UP>(d.K);
  cudaError_t e = cudaFuncSetAttribute(k_fused_tc<UP, BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fused_tc<UP, BF16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const int total = d.n_sc * d.nsys;
  const int grid = (total + TcGeo<UP>::NG - 1) / TcGeo<UP>::NG;
  InstDesc in{d, H, S, X, status, scale_out};
  k_fused_tc<UP, BF16><<<grid, NT, L.total, s>>>(in, d.K);
  return cudaGetLastError();
}

template <int UP, bool BF16, int PH>
cudaError_t launch_batch_tc_ph(const InstDesc *insts, const WorkItem *items, int n_items,
                               int *queue, int Kmax, int grid, cudaStream_t s,
                               const int *fix_list, const int *fix_count, const SplitWs &ws) {
  const TcSmem L = tc_smem_layout<UP>(Kmax);
  cudaError_t e = cudaFuncSetAttribute(k_batch_tc<UP, BF16, PH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_tc<UP, BF16, PH>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k_batch_tc<UP, BF16, PH><<<grid, NT, L.total, s>>>(insts, items, n_items, queue, Kmax,
                                                      fix_list, fix_count, ws);
  return cudaGetLastError();
}

template <int UP, bool BF16>
cudaError_t launch_batch_tc_t(const InstDesc *insts, const WorkItem *items, int n_items,
                              int *queue, int Kmax, int grid, cudaStream_t s,
                              const int *fix_list, const int *fix_count, int phase,
                              const SplitWs &ws) {
  switch (phase) {
    case PH_GRAM:
      return launch_batch_tc_ph<UP, BF16, PH_GRAM>(insts, items, n_items, queue, Kmax, grid, s,
                                                   fix_list, fix_count, ws);
    case PH_SOLVE:
      return launch_batch_tc_ph<UP, BF16, PH_SOLVE>(insts, items, n_items, queue, Kmax, grid, s,
                                                    fix_list, fix_count, ws);
    case PH_APPLY:
      return launch_batch_tc_ph<UP, BF16, PH_APPLY>(insts, items, n_items, queue, Kmax, grid, s,
                                                    fix_list, fix_count, ws);
    default:
      return launch_batch_tc_ph<UP, BF16, PH_FUSED>(insts, items, n_items, queue, Kmax, grid, s,
                                                    fix_list, fix_count, ws);
  }
}

template <int UP>
cudaError_t launch_tc_u(const SysDesc &d, bool bf16, const float2 *H, const float2 *S, float2 *X,
                        int *status, float *scale_out, cudaStream_t s) {
  return bf16 ? launch_tc_t<UP, true>(d, H, S, X, status, scale_out, s)
              : launch_tc_t<UP, false>(d, H, S, X, status, scale_out, s);
}

template <int UP, bool BF16>
cudaError_t launch_fixup_tc_t(const SysDesc &d, const float2 *H, const float2 *S, float2 *X,
                              int *status, const int *fix_list, int *fix_count, int grid,
                              cudaStream_t s) {
  const TcSmem L = tc_smem_layout<UP>(d.K);
  cudaError_t e = cudaFuncSetAttribute(k_fixup_tc<UP, BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fixup_tc<UP, BF16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  InstDesc in{d, H, S, X, status, nullptr};
  k_fixup_tc<UP, BF16><<<grid, NT, L.total, s>>>(in, fix_list, fix_count, d.K);
  return cudaGetLastError();
}

template <int UP>
int tc_blocks_t(bool bf16, int Kmax) {
  // the occupancy API reports one CTA per SM for these kernels, below what
  // the SM holds (three CTAs of the U = 16 form were measured resident), so
  // the count comes from the limits themselves
  const size_t bytes = tc_smem_layout<UP>(Kmax).total;
  const void *k = bf16 ? (const void *)k_batch_tc<UP, true> : (const void *)k_batch_tc<UP, false>;
  cudaError_t e = bf16 ? cudaFuncSetAttribute(k_batch_tc<UP, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)bytes)
                       : cudaFuncSetAttribute(k_batch_tc<UP, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)bytes);
  if (e == cudaSuccess)
    e = bf16 ? cudaFuncSetAttribute(k_batch_tc<UP, true>,
                                    cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared)
             : cudaFuncSetAttribute(k_batch_tc<UP, false>,
                                    cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared);
  return e == cudaSuccess ? resident_blocks(k, NT, bytes, TMEM_COLS) : 0;
}

}  // namespace

template <int UP>
cudaError_t TcOps<UP>::fused(const SysDesc &d, bool bf16, const float2 *H, const float2 *S,
                             float2 *X, int *status, float *scale_out, cudaStream_t s) {
  return launch_tc_u<UP>(d, bf16, H, S, X, status, scale_out, s);
}
template <int UP>
cudaError_t TcOps<UP>::batch(bool bf16, const InstDesc *insts, const WorkItem *items,
                             int n_items, int *queue, int Kmax, int grid, cudaStream_t s,
                             const int *fix_list, const int *fix_count, int phase,
                             const SplitWs &ws) {
  return bf16 ? launch_batch_tc_t<UP, true>(insts, items, n_items, queue, Kmax, grid, s, fix_list,
                                            fix_count, phase, ws)
              : launch_batch_tc_t<UP, false>(insts, items, n_items, queue, Kmax, grid, s,
                                             fix_list, fix_count, phase, ws);
}
template <int UP>
cudaError_t TcOps<UP>::fixup(const SysDesc &d, bool bf16, const float2 *H, const float2 *S,
                             float2 *X, int *status, const int *fix_list, int *fix_count,
                             int grid, cudaStream_t s) {
  return bf16 ? launch_fixup_tc_t<UP, true>(d, H, S, X, status, fix_list, fix_count, grid, s)
              : launch_fixup_tc_t<UP, false>(d, H, S, X, status, fix_list, fix_count, grid, s);
}
template <int UP>
int TcOps<UP>::blocks(bool bf16, int Kmax) {
  return tc_blocks_t<UP>(bf16, Kmax);
}

}  // namespace dp
