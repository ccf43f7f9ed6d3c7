// dp_tcpipe.cu -- the tensor-core precoder as a warp-specialized persistent
// pipeline, for U <= 16 users (padded to 8 or 16), 1 <= K <= 16 symbols and
// channel rows that 1-D bulk copies can fetch (U even, H 16-byte aligned).
//
// Per system the arithmetic is that of the group kernel in dp_tc.cu, bit for
// bit (Sec. III-B: G = H H^H as the real product P = R R^T of the realified
// channel on the tensor cores; Thm. 1 with Lemma 1 for the precoding factor;
// z = A^{-1} s; x_c = scale H_c^H z as a split-FP16 tensor-core product).
// What differs is the schedule.  One CTA per SM walks its groups of
// NG = 128 / (2 UP) systems through three roles that hand work over with
// mbarriers, never with a CTA-wide barrier:
//
//   producer  (warp 12)    1-D bulk copies of H rows into a 3-stage ring: the
//                          Gram chunks of group g, then the apply tiles of
//                          group g - 1 (read again, now from L2);
//   converters (warps 0-7) BF16/FP16 Gram operand from the ring; split-FP16
//                          apply operands; TMEM -> scaled X.  Each warp
//                          streams on its own, synchronized only by
//                          mbarriers;
//   MMA issuer (warp 13)   one thread issues every tcgen05.mma and commit;
//   solvers   (warps 8-11) TMEM -> G in registers (one system per 2 UP
//                          lanes, each lane half a row), Gauss-Jordan
//                          inverse, t, scale, z = T s; z and scale to
//                          shared memory.
//
// The solve of group g thus runs while the converters apply group g - 1 and
// stream the Gram of group g + 1, and the next groups' H is always in flight.
// Every wait is bounded; a wait that gives up sets an abort flag that every
// role samples, the kernel drains its copies and MMAs, marks the systems it
// did not finish ST_TIMEOUT (outputs zeroed) and frees its TMEM.
#include "dp_blocks.cuh"
#include "dp_internal.h"
#include "dp_tc.cuh"

namespace dp {
namespace {

constexpr int PP_CV = 8;                              // converter warps
constexpr int PP_SV = 4;                              // solver warps
constexpr int PP_PRODUCER = PP_CV + PP_SV;            // producer warp
constexpr int PP_ISSUER = PP_PRODUCER + 1;            // MMA-issuing warp
constexpr int PP_THREADS = 32 * (PP_ISSUER + 1);
constexpr int PP_NRAW = 3;                            // raw H stages
constexpr int PP_RAW = 32768;                         // bytes per raw stage
constexpr int PP_TILE = 16384;                        // 128 rows x 128 B, SW128
constexpr int PP_BOP = 4096;                          // 32 rows x 128 B
constexpr int PP_KMAX = 16;
constexpr int PP_GCH = 64;                            // antennas per Gram chunk
constexpr int PP_MT = 128;                            // antennas per apply tile
constexpr uint32_t PP_TMEM = 256;                     // Gram 128 + 2 x apply 32
constexpr uint32_t PP_ACC = 128;                      // first apply column
constexpr int BAR_SV = 1;                             // solvers' named barrier (0: CTA)

// mbarrier slots (arrival counts in brackets)
enum : int {
  B_RAWFULL = 0,                      // [1 + bytes] producer
  B_RAWEMPTY = B_RAWFULL + PP_NRAW,   // [8] converters
  B_GOPFULL = B_RAWEMPTY + PP_NRAW,   // [8] converters, 2 stages
  B_GOPEMPTY = B_GOPFULL + 2,         // [1] MMA commit, 2 stages
  B_GRAMDONE = B_GOPEMPTY + 2,        // [1] MMA commit
  B_GRAMFREE,                         // [1] solvers
  B_ZREADY,                           // [1] solvers, 2 buffers
  B_ZFREE = B_ZREADY + 2,             // [8] converters, 2 buffers
  B_AOPFULL = B_ZFREE + 2,            // [8] converters, 2 stages
  B_ACCDONE = B_AOPFULL + 2,          // [1] MMA commit, 2 accumulators
  B_FIN = B_ACCDONE + 2,              // [1] MMA commit
  B_COUNT
};

template <int UP>
struct PpGeo {
  static constexpr int NG = 128 / (2 * UP);  // systems per group
  static constexpr int M2 = 2 * UP;          // realified rows per system
  static constexpr int SEG = 2 * UP;         // solver lanes per system
  static constexpr int SPW = NG / PP_SV;     // systems per solver warp
  static constexpr int KSTEPS = (2 * UP + 15) / 16;  // apply K-steps per term
  // byte offsets in the 1024-aligned dynamic shared memory
  static constexpr int RAW = 0;
  static constexpr int GOP = RAW + PP_NRAW * PP_RAW;            // 2 Gram operand tiles
  static constexpr int AOP = GOP + 2 * PP_TILE;                 // 2 apply tiles [hi | lo]
  static constexpr int BOPS = AOP + 2 * PP_TILE;                // 2 x (hi, lo, hi 2^-11)
  static constexpr int GS = BOPS + 2 * 3 * PP_BOP;              // G per solver system
  static constexpr int SZ = GS + NG * UP * UP * 8;              // s, then z: 2 x NG x [K][UP]
  static constexpr int INFO = SZ + 2 * NG * PP_KMAX * UP * 8;   // st, sc, zexp: 2 x NG each
  static constexpr int BARS = INFO + 3 * 2 * NG * 4;
  static constexpr int MISC = BARS + B_COUNT * 8;               // tmem base, abort, stall flag, per-warp done
  static constexpr int BYTES = MISC + 48 + 1024;                // + alignment slack
  static_assert(NG % PP_SV == 0 && SPW >= 1, "whole systems per solver warp");
  static_assert((32 * PP_CV) % (NG * UP) == 0, "a converter thread's Gram items share a system");
  static_assert(NG * PP_GCH * UP * 8 <= PP_RAW && PP_MT * UP * 8 <= PP_RAW, "raw stage");
  static_assert(BARS % 8 == 0, "mbarrier alignment");
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

// Named barrier over n threads that also ANDs a predicate across them: every
// thread of a role leaves with the same verdict.
__device__ __forceinline__ bool bar_and(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// AND of a predicate over this lane's segment of SEG lanes.
template <int SEG>
__device__ __forceinline__ bool seg_all(bool v, int lane) {
  const unsigned b = __ballot_sync(FULL, v);
  const unsigned m = SEG == 32 ? FULL : (((1u << SEG) - 1u) << (lane / SEG * SEG));
  return (b & m) == m;
}

// Where a launch's groups come from: a single plan's systems taken NG at a
// time (items == nullptr, instance in0), or a batch bucket's work items (an
// instance and up to NG of its systems each).  Every role walks groups
// blockIdx.x, blockIdx.x + gridDim.x, ... in the same order.
struct PpSrc {
  InstDesc in0;
  const InstDesc *insts;
  const WorkItem *items;
  int n_groups;
  int *fix_list;   // batch, automatic refinement: groups holding ST_REFINE
  int *fix_count;  // systems, appended once per group by the solvers
};
struct PpGroup {
  const InstDesc *in;
  int sys0, nact;
};
template <int UP, bool BAT>
__device__ __forceinline__ PpGroup pp_group(const PpSrc &src, int g) {
  if constexpr (BAT) {
    const WorkItem w = src.items[g];
    return PpGroup{src.insts + w.inst, w.sys0, w.nact};
  }
  const int total = src.in0.d.n_sc * src.in0.d.nsys;
  return PpGroup{&src.in0, g * PpGeo<UP>::NG, min(PpGeo<UP>::NG, total - g * PpGeo<UP>::NG)};
}

// The instance of a group: a single plan's reads its descriptor straight from
// the kernel parameters.
template <bool BAT>
__device__ __forceinline__ const InstDesc &pp_in(const PpSrc &src, const PpGroup &G) {
  if constexpr (BAT) return *G.in;
  else return src.in0;
}

// A system of a group: subcarrier, first antenna, antennas; live = exists and
// is not left to the B_c x B_c kernel.
struct PpSys {
  int n, lo, nr;
  bool live;
};
__device__ __forceinline__ PpSys pp_sys(const SysDesc &d, const PpGroup &G, int s) {
  PpSys r{0, 0, 0, false};
  if (s < G.nact) {
    const int sys = G.sys0 + s;
    r.n = sys / d.nsys;
    int lo, hi;
    sys_rows(d, sys - r.n * d.nsys, lo, hi);
    if (!sys_is_small(d, hi - lo)) {
      r.lo = lo;
      r.nr = hi - lo;
      r.live = true;
    }
  }
  return r;
}
// Largest antenna count over the live systems of a group (0: nothing to do;
// every role skips such a group).
template <int UP>
__device__ int pp_group_rows(const SysDesc &d, const PpGroup &G) {
  int m = 0;
  for (int s = 0; s < PpGeo<UP>::NG; ++s) {
    const PpSys y = pp_sys(d, G, s);
    if (y.live) m = max(m, y.nr);
  }
  return m;
}

// ------------------------------------------------------------- producer ---
template <int UP, bool BAT>
__device__ void pp_producer(const PpSrc &src, unsigned char *base, uint64_t *bars,
                            volatile int *abort_f) {
  using T = PpGeo<UP>;
  uint32_t use = 0;
  bool ok = true;
  auto stage = [&](uint32_t bytes) -> unsigned char * {
    const int slot = use % PP_NRAW;
    if (use >= PP_NRAW) ok = mbar_wait_ab(&bars[B_RAWEMPTY + slot], ((use / PP_NRAW) - 1) & 1, abort_f);
    if (ok && *abort_f) ok = false;
    if (!ok) return nullptr;
    mbar_arrive_expect_tx(&bars[B_RAWFULL + slot], bytes);
    return base + T::RAW + slot * PP_RAW;
  };
  int prev = -1;
  for (int g = blockIdx.x; ok; g += gridDim.x) {
    const bool have = g < src.n_groups;
    const PpGroup G = have ? pp_group<UP, BAT>(src, g) : PpGroup{nullptr, 0, 0};
    const int rows = have ? pp_group_rows<UP>(pp_in<BAT>(src, G).d, G) : 0;
    if (have && rows == 0) continue;
    if (have) {
      const InstDesc &gi = pp_in<BAT>(src, G);
      const SysDesc &d = gi.d;
      const size_t rowb = (size_t)d.U * 8;
      for (int c = 0; c * PP_GCH < rows && ok; ++c) {
        uint32_t bytes = 0;
        for (int s = 0; s < T::NG; ++s) {
          const PpSys y = pp_sys(d, G, s);
          const int r = y.live ? min(PP_GCH, y.nr - c * PP_GCH) : 0;
          if (r > 0) bytes += (uint32_t)(r * rowb);
        }
        unsigned char *dst = stage(bytes);
        if (!dst) break;
        const uint64_t *bar = &bars[B_RAWFULL + use % PP_NRAW];
        for (int s = 0; s < T::NG; ++s) {
          const PpSys y = pp_sys(d, G, s);
          const int r = y.live ? min(PP_GCH, y.nr - c * PP_GCH) : 0;
          if (r > 0)
            tma_load_1d(dst + s * PP_GCH * rowb,
                        gi.H + ((size_t)y.n * d.B + y.lo + c * PP_GCH) * d.U,
                        (uint32_t)(r * rowb), const_cast<uint64_t *>(bar));
        }
        ++use;
      }
    }
    if (prev >= 0 && ok) {
      const PpGroup P = pp_group<UP, BAT>(src, prev);
      const InstDesc &pi = pp_in<BAT>(src, P);
      const SysDesc &d = pi.d;
      const size_t rowb = (size_t)d.U * 8;
      for (int s = 0; s < T::NG && ok; ++s) {
        const PpSys y = pp_sys(d, P, s);
        if (!y.live) continue;
        for (int m0 = 0; m0 < y.nr && ok; m0 += PP_MT) {
          const int r = min(PP_MT, y.nr - m0);
          unsigned char *dst = stage((uint32_t)(r * rowb));
          if (!dst) break;
          tma_load_1d(dst, pi.H + ((size_t)y.n * d.B + y.lo + m0) * d.U, (uint32_t)(r * rowb),
                      &bars[B_RAWFULL + use % PP_NRAW]);
          ++use;
        }
      }
    }
    if (!have) break;
    prev = g;
  }
  if (!ok) *abort_f = 1;
  // every copy issued has landed before the CTA may leave (the last use of
  // each slot is its newest phase)
  for (uint32_t k = 0; k < PP_NRAW && k < use; ++k) {
    const uint32_t last = use - 1 - ((use - 1 - k) % PP_NRAW);
    mbar_wait(&bars[B_RAWFULL + k], (last / PP_NRAW) & 1);
  }
}

// ----------------------------------------------------------- converters ---
struct PpPend {  // an apply tile whose MMAs may be in flight
  float2 *Xn;
  int m0, mrows, at;
  uint32_t tile;
  float os;
  bool good;
};

// Scaled X of one tile: this warp's 32 antenna rows (its TMEM lane quarter),
// symbols 8 h .. 8 h + 7 (h = which of the two warps of the quarter).
__device__ bool pp_readout(const PpPend &p, int K, int B, uint32_t taddr, uint64_t *bars,
                           volatile int *abort_f, int warp, int lane) {
  bool w = mbar_wait_ab(&bars[B_ACCDONE + p.at], (p.tile >> 1) & 1, abort_f);
  w = __all_sync(FULL, w) != 0;
  if (!w) {
    *abort_f = 1;
    return false;
  }
  const int quad = warp & 3, h = warp >> 2;
  const int r = 32 * quad + lane;
  float2 *xc = p.Xn + p.m0 + r;
  if (!p.good) {
    if (r < p.mrows) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (8 * h + q < K) xc[(size_t)(8 * h + q) * B] = make_float2(0.f, 0.f);
    }
    return true;
  }
  tc::fence_after_sync();
  float v[16];
  tc::tmem_ld16(taddr + ((uint32_t)(32 * quad) << 16) + PP_ACC + 32 * p.at + 16 * h, v);
  tc::fence_before_sync();
  if (r < p.mrows) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (8 * h + q < K)
        xc[(size_t)(8 * h + q) * B] = make_float2(v[2 * q] * p.os, v[2 * q + 1] * p.os);
  }
  return true;
}

template <int UP, bool BF16, bool BAT>
__device__ void pp_converter(const PpSrc &src, unsigned char *base, uint64_t *bars,
                             uint32_t taddr, volatile int *abort_f, volatile int *done_w) {
  using T = PpGeo<UP>;
  constexpr int NG = T::NG, M2 = T::M2, NTH = 32 * PP_CV;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int *st_i = reinterpret_cast<const int *>(base + T::INFO);
  const float *sc_i = reinterpret_cast<const float *>(base + T::INFO + 2 * NG * 4);
  const int *ze_i = reinterpret_cast<const int *>(base + T::INFO + 4 * NG * 4);
  const float2 *Zs = reinterpret_cast<const float2 *>(base + T::SZ);
  uint32_t raw_i = 0, gop_i = 0, tile_i = 0, bsys_i = 0;
  int o = 0, prev = -1;
  bool run = true;
  // hand a filled stage to the MMA issuer and the ring slot back to the
  // producer (one arrival per warp)
  auto release = [&](uint64_t *full, int slot) {
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(full);
      mbar_arrive(&bars[B_RAWEMPTY + slot]);
    }
  };
  for (int g = blockIdx.x; run; g += gridDim.x) {
    const bool have = g < src.n_groups;
    const PpGroup G = have ? pp_group<UP, BAT>(src, g) : PpGroup{nullptr, 0, 0};
    const int rows = have ? pp_group_rows<UP>(pp_in<BAT>(src, G).d, G) : 0;
    if (have && rows == 0) continue;

    // ---- Gram of group g (ordinal o): chunks of 64 antennas ------------------
    if (have) {
      const SysDesc &gd = pp_in<BAT>(src, G).d;
      const int U = gd.U;
      // the thread's items all belong to one system (NTH is a multiple of
      // NG * UP), whose rows it keeps in registers
      const int s_mine = (tid / UP) % NG;
      const PpSys y_mine = pp_sys(gd, G, s_mine);
      const int nr_mine = y_mine.live ? y_mine.nr : 0;
      const int nch = (rows + PP_GCH - 1) / PP_GCH;
      for (int c = 0; c < nch && run; ++c) {
        const int slot = raw_i % PP_NRAW, st = gop_i & 1;
        bool w = !*abort_f && mbar_wait_ab(&bars[B_RAWFULL + slot], (raw_i / PP_NRAW) & 1, abort_f);
        if (w && gop_i >= 2) w = mbar_wait_ab(&bars[B_GOPEMPTY + st], ((gop_i >> 1) - 1) & 1, abort_f);
        if (__all_sync(FULL, w)) {
          const unsigned char *rs = base + T::RAW + slot * PP_RAW;
          unsigned char *tile = base + T::GOP + st * PP_TILE;
          for (int item = tid; item < 8 * NG * UP; item += NTH) {
            const int u = item % UP, s = s_mine, g8 = item / (UP * NG);
            const int left = nr_mine - (c * PP_GCH + 8 * g8);
            const bool live = nr_mine > 0 && u < U;
            const float2 *sp =
                reinterpret_cast<const float2 *>(rs + (size_t)s * PP_GCH * U * 8) + 8 * g8 * U + u;
            float2 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              v[j] = (live && j < left) ? sp[j * U] : make_float2(0.f, 0.f);
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
        } else {
          *abort_f = 1;
          run = false;
          break;
        }
        release(&bars[B_GOPFULL + st], slot);
        ++raw_i;
        ++gop_i;
      }
      if (!run) break;
    }

    // ---- apply of the previous group (ordinal o - 1) -------------------------
    if (prev >= 0) {
      const PpGroup P = pp_group<UP, BAT>(src, prev);
      const InstDesc &pi = pp_in<BAT>(src, P);
      const int U = pi.d.U, K = pi.d.K, B = pi.d.B;
      const int po = o - 1, zb = po & 1;
      bool w = !*abort_f && mbar_wait_ab(&bars[B_ZREADY + zb], (po >> 1) & 1, abort_f);
      if (!__all_sync(FULL, w)) {
        *abort_f = 1;
        break;
      }
      PpPend pend{nullptr, 0, 0, 0, 0, 0.f, false};
      bool has_pend = false;
      for (int s = 0; s < NG && run; ++s) {
        const PpSys y = pp_sys(pi.d, P, s);
        if (!y.live) continue;
        float2 *Xn = pi.X + (size_t)y.n * K * B + y.lo;
        const bool good = st_i[zb * NG + s] == ST_OK;
        float os = 0.f;
        const uint32_t bb = bsys_i & 1;
        if (good) {
          // B operands: 32 rows (16 symbols x Re/Im) x 8 chunks of 4 users
          const float2 *zs = Zs + (size_t)(zb * NG + s) * PP_KMAX * UP;
          const int zexp = ze_i[zb * NG + s];
          const float zn = ldexpf(1.f, -zexp);
          os = ldexpf(sc_i[zb * NG + s], zexp);
          unsigned char *b_op = base + T::BOPS + bb * 3 * PP_BOP;
          for (int e = tid; e < 32 * 8; e += NTH) {
            const int row = e >> 3, c8 = e & 7;
            const int q = row >> 1, im = row & 1;
            float v[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int u = 4 * c8 + j;
              float2 z = make_float2(0.f, 0.f);
              if (q < K && u < U && 8 * c8 < 2 * UP) z = zs[q * UP + u];
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
            *reinterpret_cast<uint4 *>(b_op + PP_BOP + off) = lo;
            *reinterpret_cast<uint4 *>(b_op + 2 * PP_BOP + off) = hs;
          }
        }
        for (int m0 = 0; m0 < y.nr; m0 += PP_MT) {
          const int slot = raw_i % PP_NRAW, at = tile_i & 1;
          const int mrows = min(PP_MT, y.nr - m0);
          bool wt = !*abort_f && mbar_wait_ab(&bars[B_RAWFULL + slot], (raw_i / PP_NRAW) & 1, abort_f);
          if (!__all_sync(FULL, wt)) {
            *abort_f = 1;
            run = false;
            break;
          }
          if (good) {
            // A tile: row r = antenna, chunks [0, UP/4) = hi, [UP/4, UP/2) = lo
            // (scaled by 2^11); chunk p holds users 4p..4p+3 (Re, Im)
            const unsigned char *rs = base + T::RAW + slot * PP_RAW;
            unsigned char *a_op = base + T::AOP + at * PP_TILE;
            for (int e = tid; e < PP_MT * (UP / 4); e += NTH) {
              const int r = e / (UP / 4), p = e % (UP / 4);
              float v[8];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < mrows && 4 * p + 2 * h < U)
                  f = *reinterpret_cast<const float4 *>(rs + (size_t)r * U * 8 + (4 * p + 2 * h) * 8);
                v[4 * h] = f.x;
                v[4 * h + 1] = f.y;
                v[4 * h + 2] = f.z;
                v[4 * h + 3] = f.w;
              }
              uint4 hi, lo;
              uint32_t *ph = &hi.x, *pl = &lo.x;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const __half2 h2 = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
                const float2 hf = __half22float2(h2);
                const __half2 l2 = __floats2half2_rn((v[2 * j] - hf.x) * 0x1p11f,
                                                     (v[2 * j + 1] - hf.y) * 0x1p11f);
                ph[j] = *reinterpret_cast<const uint32_t *>(&h2);
                pl[j] = *reinterpret_cast<const uint32_t *>(&l2);
              }
              *reinterpret_cast<uint4 *>(a_op + tc::sw128_offset(r, p)) = hi;
              *reinterpret_cast<uint4 *>(a_op + tc::sw128_offset(r, UP / 4 + p)) = lo;
            }
          }
          release(&bars[B_AOPFULL + at], slot);
          ++raw_i;
          // the previous tile's accumulator, while this tile's MMAs run
          if (has_pend && !pp_readout(pend, K, B, taddr, bars, abort_f, warp, lane)) {
            run = false;
            break;
          }
          pend = PpPend{Xn, m0, mrows, at, tile_i, os, good};
          has_pend = true;
          ++tile_i;
        }
        ++bsys_i;
      }
      if (!run) break;
      if (has_pend && !pp_readout(pend, K, B, taddr, bars, abort_f, warp, lane)) break;
      // this warp is done with the group's z, scale and status
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars[B_ZFREE + zb]);
        done_w[warp] = o;  // this warp's share of groups 0 .. o - 1 is written
      }
    }
    if (!have) break;
    prev = g;
    ++o;
  }
}

// ----------------------------------------------------------- MMA issuer ---
// One thread issues the Gram and apply MMAs in the converters' order.
template <int UP, bool BF16, bool BAT>
__device__ void pp_issuer(const PpSrc &src, unsigned char *base, uint64_t *bars, uint32_t taddr,
                          volatile int *abort_f) {
  using T = PpGeo<UP>;
  constexpr int NG = T::NG;
  const int *st_i = reinterpret_cast<const int *>(base + T::INFO);
  const uint32_t gop_u = smem_u32(base + T::GOP), aop_u = smem_u32(base + T::AOP),
                 bop_u = smem_u32(base + T::BOPS);
  const uint32_t idesc_g = tc::idesc_f16(128, 128, BF16);
  const uint32_t idesc_a = tc::idesc_f16(128, 32, false);
  uint32_t gop_i = 0, tile_i = 0, bsys_i = 0;
  int o = 0, prev = -1;
  bool ok = true;
  const int stall_us = BAT ? 0 : src.in0.d.dbg_stall_us;
  if (stall_us > 0) {
    // failure injection: wait on a flag that nothing sets, bounded in time;
    // running out counts as a timed-out wait
    const volatile int *never = reinterpret_cast<const volatile int *>(base + T::MISC + 8);
    const uint64_t t0 = globaltimer_ns(), lim = (uint64_t)stall_us * 1000u;
    while (!*never && globaltimer_ns() - t0 < lim) __nanosleep(256);
    ok = *never != 0;
  }
  for (int g = blockIdx.x; ok; g += gridDim.x) {
    const bool have = g < src.n_groups;
    const PpGroup G = have ? pp_group<UP, BAT>(src, g) : PpGroup{nullptr, 0, 0};
    const int rows = have ? pp_group_rows<UP>(pp_in<BAT>(src, G).d, G) : 0;
    if (have && rows == 0) continue;
    if (have) {
      const int nch = (rows + PP_GCH - 1) / PP_GCH;
      for (int c = 0; c < nch && ok; ++c) {
        const int st = gop_i & 1;
        ok = !*abort_f && mbar_wait_ab(&bars[B_GOPFULL + st], (gop_i >> 1) & 1, abort_f);
        // the solvers have read the previous group's Gram out of TMEM
        if (ok && c == 0 && o >= 1) ok = mbar_wait_ab(&bars[B_GRAMFREE], (o - 1) & 1, abort_f);
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll
        for (int kk = 0; kk < PP_GCH / 16; ++kk) {
          const uint64_t desc = tc::desc_kmajor_sw128(gop_u + st * PP_TILE + kk * 32);
          tc::mma_f16(taddr, desc, desc, idesc_g, c > 0 || kk > 0);
        }
        tc::commit(&bars[B_GOPEMPTY + st]);
        if (c == nch - 1) tc::commit(&bars[B_GRAMDONE]);
        ++gop_i;
      }
    }
    if (prev >= 0 && ok) {
      const PpGroup P = pp_group<UP, BAT>(src, prev);
      const int zb = (o - 1) & 1;
      for (int s = 0; s < NG && ok; ++s) {
        const PpSys y = pp_sys(pp_in<BAT>(src, P).d, P, s);
        if (!y.live) continue;
        const uint32_t b0 = bop_u + (bsys_i & 1) * 3 * PP_BOP;
        for (int m0 = 0; m0 < y.nr && ok; m0 += PP_MT) {
          const int at = tile_i & 1;
          ok = !*abort_f && mbar_wait_ab(&bars[B_AOPFULL + at], (tile_i >> 1) & 1, abort_f);
          if (!ok) break;
          if (st_i[zb * NG + s] == ST_OK) {  // written before the converters' arrival
            tc::fence_after_sync();
            const uint32_t acc = taddr + PP_ACC + 32 * at;
            const uint32_t a0 = aop_u + at * PP_TILE;
#pragma unroll
            for (int kk = 0; kk < T::KSTEPS; ++kk) {
              const uint32_t ko = kk * 32;
              tc::mma_f16(acc, tc::desc_kmajor_sw128(a0 + ko), tc::desc_kmajor_sw128(b0 + ko),
                          idesc_a, kk > 0);
              tc::mma_f16(acc, tc::desc_kmajor_sw128(a0 + ko),
                          tc::desc_kmajor_sw128(b0 + PP_BOP + ko), idesc_a, true);
              tc::mma_f16(acc, tc::desc_kmajor_sw128(a0 + 4 * UP + ko),
                          tc::desc_kmajor_sw128(b0 + 2 * PP_BOP + ko), idesc_a, true);
            }
          }
          tc::commit(&bars[B_ACCDONE + at]);
          ++tile_i;
        }
        ++bsys_i;
      }
    }
    if (!have) break;
    prev = g;
    ++o;
  }
  if (!ok) *abort_f = 1;
  // every MMA issued has completed before TMEM is freed
  tc::commit(&bars[B_FIN]);
  if (!mbar_wait(&bars[B_FIN], 0)) *abort_f = 1;
}

// --------------------------------------------------------------- solver ---
// Solver warp sw takes systems sw * SPW .. of each group, one per segment of
// 2 UP lanes in the split-row form: lane (i, h) holds half h of row i.  The
// system's symbols are loaded into its z buffer, which the whitening then
// overwrites with z.
template <int UP, bool BF16, bool BAT>
__device__ void pp_solver(const PpSrc &src, unsigned char *base, uint64_t *bars, uint32_t taddr,
                          volatile int *abort_f) {
  using T = PpGeo<UP>;
  constexpr int NG = T::NG, SEG = T::SEG, SPW = T::SPW, HALF = UP / 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sw = warp - PP_CV, stid = tid - 32 * PP_CV;  // solver warp, thread
  const int seg = lane / SEG, sl = lane % SEG, i = sl % UP, h = sl / UP;
  const int sysi = sw * SPW + seg;  // this lane's system within the group
  float2 *Gw = reinterpret_cast<float2 *>(base + T::GS) + (size_t)sysi * UP * UP;
  int *st_i = reinterpret_cast<int *>(base + T::INFO);
  float *sc_i = reinterpret_cast<float *>(base + T::INFO + 2 * NG * 4);
  int *ze_i = reinterpret_cast<int *>(base + T::INFO + 4 * NG * 4);
  int *fix_f = reinterpret_cast<int *>(base + T::MISC + 12);  // the group has a marked system
  int o = 0;
  for (int g = blockIdx.x; g < src.n_groups; g += gridDim.x) {
    const PpGroup G = pp_group<UP, BAT>(src, g);
    if (pp_group_rows<UP>(pp_in<BAT>(src, G).d, G) == 0) continue;
    const InstDesc &in = pp_in<BAT>(src, G);
    const SysDesc &d = in.d;
    const int U = d.U, K = d.K;
    const int sys = G.sys0 + sysi, zb = o & 1;
    const float kappa = sys_kappa(d, sys);
    const PpSys y = pp_sys(in.d, G, sysi);
    float2 *Sz = reinterpret_cast<float2 *>(base + T::SZ) + (size_t)(zb * NG + sysi) * PP_KMAX * UP;
    // the converters are done with this buffer's previous group (o - 2)
    bool w = !*abort_f;
    if (w && o >= 2) w = mbar_wait_ab(&bars[B_ZFREE + zb], ((o >> 1) - 1) & 1, abort_f);
    // symbols of this system (zero pads), fetched while the Gram runs
    bool fin_s = true;
    if (w) {
      for (int e = sl; e < K * UP; e += SEG) {
        const int k = e / UP, u = e - k * UP;
        float2 v = make_float2(0.f, 0.f);
        if (y.live && u < U) v = __ldg(in.S + ((size_t)y.n * K + k) * U + u);
        fin_s = fin_s && cfinite(v);
        Sz[k * UP + u] = v;
      }
    }
    // this warp's 32 rows of P (its systems' diagonal blocks)
    if (w) w = mbar_wait_ab(&bars[B_GRAMDONE], o & 1, abort_f);
    w = __all_sync(FULL, w) != 0;
    float v[32];
    if (w) {
      tc::fence_after_sync();
      tc::tmem_ld32(taddr + ((uint32_t)(32 * sw) << 16) + 32 * sw, v);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = 0.f;
    }
    tc::fence_before_sync();
    if (!bar_and(BAR_SV, 32 * PP_SV, w)) {
      *abort_f = 1;
      break;
    }
    if (stid == 0) mbar_arrive(&bars[B_GRAMFREE]);

    // half h of G row i: Re G_ij = P_ij + P_{U'+i,U'+j}, Im G_ij = P_{U'+i,j} -
    // P_{i,U'+j} (U' = UP).  Lane (i, 0) holds TMEM row i, lane (i, 1) row
    // U' + i; each sends the partner the two entries of the partner's half.
    float pw[SEG];
#pragma unroll
    for (int c = 0; c < SEG; ++c) pw[c] = (SEG == 32 || seg == 0) ? v[c] : v[(SEG % 32) + c];
    float2 row[HALF];
    bool fin_g = true;
#pragma unroll
    for (int jj = 0; jj < HALF; ++jj) {
      const float s1 = h == 0 ? pw[HALF + jj] : pw[UP + jj];
      const float s2 = h == 0 ? pw[UP + HALF + jj] : pw[jj];
      const float r1 = __shfl_xor_sync(FULL, s1, UP, SEG);
      const float r2 = __shfl_xor_sync(FULL, s2, UP, SEG);
      const int j = h * HALF + jj;
      const float re = h == 0 ? pw[jj] + r1 : r1 + pw[UP + HALF + jj];
      const float im = h == 0 ? r2 - pw[UP + jj] : pw[HALF + jj] - r2;
      float2 gij = make_float2(0.f, 0.f);
      if (i < U && j < U) gij = make_float2(re, j == i ? 0.f : im);
      fin_g = fin_g && cfinite(gij);
      Gw[i * UP + j] = gij;
      row[jj] = gij;
      if (j == i) row[jj].x += kappa;
    }
    __syncwarp();
    const bool finite_in = seg_all<SEG>(fin_s && fin_g, lane);
    float sc = 0.f, zm = 0.f, sens = 0.f;
    const int st = split_solve<UP>(row, Gw, Sz, Sz, UP, kappa, sys_rho2(d, sys), d.Es, U, K, sl,
                                   finite_in, true, sc, zm, d.mrt != 0,
                                   d.refine == 2 ? &sens : nullptr);
    // automatic refinement: a flagged system is applied unrefined here and
    // marked; the fix-up launch of the group kernel redoes its group
    constexpr float eps = BF16 ? 0x1p-8f : 0x1p-11f;
    const bool mark = d.refine == 2 && st == ST_OK && eps * sens >= kRefineTrigger;
    int zexp = 0;
    if (zm > 0.f) frexpf(zm, &zexp);
    if (sl == 0) {
      st_i[zb * NG + sysi] = st;
      sc_i[zb * NG + sysi] = sc;
      ze_i[zb * NG + sysi] = zexp;
      if (y.live) {
        in.status[sys] = mark ? (int)ST_REFINE : st;
        if (in.scale_out) in.scale_out[sys] = st == ST_OK ? sc : 0.f;
        if (mark) atomicOr(fix_f, 1);
      }
    }
    if (!bar_and(BAR_SV, 32 * PP_SV, true)) break;
    if (stid == 0) {
      if (*fix_f) {  // a batch lists the group once for its fix-up launch
        if (src.fix_list) src.fix_list[atomicAdd(src.fix_count, 1)] = g;
        *fix_f = 0;
      }
      mbar_arrive(&bars[B_ZREADY + zb]);
    }
    ++o;
  }
}

// --------------------------------------------------------------- kernel ---
template <int UP, bool BF16, bool BAT>
__global__ void __launch_bounds__(PP_THREADS, 1)
    k_pipe_tc(PpSrc src) {
  using T = PpGeo<UP>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + T::BARS);
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + T::MISC);
  volatile int *abort_f = reinterpret_cast<volatile int *>(base + T::MISC + 4);
  volatile int *done_w = reinterpret_cast<volatile int *>(base + T::MISC + 16);  // [PP_CV]
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int b = 0; b < B_COUNT; ++b) {
      const bool per_warp = (b >= B_RAWEMPTY && b < B_RAWEMPTY + PP_NRAW) ||
                            (b >= B_GOPFULL && b < B_GOPFULL + 2) ||
                            (b >= B_ZFREE && b < B_ZFREE + 2) ||
                            (b >= B_AOPFULL && b < B_AOPFULL + 2);
      mbar_init(&bars[b], per_warp ? PP_CV : 1);
    }
    *abort_f = 0;
    *reinterpret_cast<volatile int *>(base + T::MISC + 8) = 0;  // the flag nothing sets
    *reinterpret_cast<volatile int *>(base + T::MISC + 12) = 0;
    for (int w = 0; w < PP_CV; ++w) done_w[w] = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, PP_TMEM);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tmem_holder;

  if (warp < PP_CV) {
    pp_converter<UP, BF16, BAT>(src, base, bars, taddr, abort_f, done_w);
  } else if (warp < PP_CV + PP_SV) {
    pp_solver<UP, BF16, BAT>(src, base, bars, taddr, abort_f);
  } else if (warp == PP_PRODUCER) {
    if ((tid & 31) == 0) pp_producer<UP, BAT>(src, base, bars, abort_f);
  } else if ((tid & 31) == 0) {
    pp_issuer<UP, BF16, BAT>(src, base, bars, taddr, abort_f);
  }
  __syncwarp();  // the producer warp's lanes meet again before the CTA barrier
  tc::fence_before_sync();
  __syncthreads();

  if (*abort_f) {  // systems of the groups not completed: ST_TIMEOUT, zero rows
    int done = done_w[0];
    for (int w = 1; w < PP_CV; ++w) done = min(done, (int)done_w[w]);
    int o = 0;
    for (int g = blockIdx.x; g < src.n_groups; g += gridDim.x) {
      const PpGroup G = pp_group<UP, BAT>(src, g);
      if (pp_group_rows<UP>(pp_in<BAT>(src, G).d, G) == 0) continue;
      if (o >= done) {
        const InstDesc &in = pp_in<BAT>(src, G);
        const SysDesc &d = in.d;
        for (int s = 0; s < T::NG; ++s) {
          const PpSys y = pp_sys(d, G, s);
          if (!y.live) continue;
          float2 *Xn = in.X + (size_t)y.n * d.K * d.B + y.lo;
          for (int e = tid; e < y.nr * d.K; e += PP_THREADS) {
            const int q = e / y.nr, r = e - q * y.nr;
            Xn[(size_t)q * d.B + r] = make_float2(0.f, 0.f);
          }
          if (tid == 0) {
            in.status[G.sys0 + s] = ST_TIMEOUT;
            if (in.scale_out) in.scale_out[G.sys0 + s] = 0.f;
          }
        }
      }
      ++o;
    }
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, PP_TMEM);
  }
}

template <int UP, bool BF16>
cudaError_t launch_pipe_t(const SysDesc &d, const float2 *H, const float2 *S, float2 *X,
                          int *status, float *scale_out, int *fix_list, int *fix_count,
                          cudaStream_t s) {
  using T = PpGeo<UP>;
  const int total = d.n_sc * d.nsys;
  const int ngroups = (total + T::NG - 1) / T::NG;
  if (ngroups == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_pipe_tc<UP, BF16, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, T::BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int grid = ngroups < nsm ? ngroups : nsm;
  PpSrc src{InstDesc{d, H, S, X, status, scale_out}, nullptr, nullptr, ngroups, fix_list,
            fix_count};
  k_pipe_tc<UP, BF16, false><<<grid, PP_THREADS, T::BYTES, s>>>(src);
  return cudaGetLastError();
}

template <int UP, bool BF16>
cudaError_t launch_batch_pipe_t(const InstDesc *insts, const WorkItem *items, int n_items,
                                int *fix_list, int *fix_count, int grid, cudaStream_t s) {
  using T = PpGeo<UP>;
  if (n_items == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_pipe_tc<UP, BF16, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, T::BYTES);
  if (e != cudaSuccess) return e;
  PpSrc src{InstDesc{}, insts, items, n_items, fix_list, fix_count};
  k_pipe_tc<UP, BF16, true><<<grid, PP_THREADS, T::BYTES, s>>>(src);
  return cudaGetLastError();
}

}  // namespace

bool pipe_tc_supported(const SysDesc &d, int UP) {
  return (UP == 8 || UP == 16) && d.tma_ok && d.K >= 1 && d.K <= PP_KMAX && d.refine != 1;
}

int pipe_systems_per_group(int UP) { return UP == 8 ? PpGeo<8>::NG : PpGeo<16>::NG; }

cudaError_t launch_batch_pipe_tc(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                                 int n_items, int *fix_list, int *fix_count, int grid,
                                 cudaStream_t s) {
  switch (UP) {
    case 8:
      return bf16 ? launch_batch_pipe_t<8, true>(insts, items, n_items, fix_list, fix_count, grid, s)
                  : launch_batch_pipe_t<8, false>(insts, items, n_items, fix_list, fix_count, grid, s);
    case 16:
      return bf16 ? launch_batch_pipe_t<16, true>(insts, items, n_items, fix_list, fix_count, grid, s)
                  : launch_batch_pipe_t<16, false>(insts, items, n_items, fix_list, fix_count, grid, s);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pipe_tc(const SysDesc &d, int UP, bool bf16, const float2 *H,
                           const float2 *S, float2 *X, int *status, float *scale_out,
                           cudaStream_t s, int *fix_list, int *fix_count) {
  switch (UP) {
    case 8:
      return bf16 ? launch_pipe_t<8, true>(d, H, S, X, status, scale_out, fix_list, fix_count, s)
                  : launch_pipe_t<8, false>(d, H, S, X, status, scale_out, fix_list, fix_count, s);
    case 16:
      return bf16 ? launch_pipe_t<16, true>(d, H, S, X, status, scale_out, fix_list, fix_count, s)
                  : launch_pipe_t<16, false>(d, H, S, X, status, scale_out, fix_list, fix_count,
                                             s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace dp
