// dp_rowsolve.cu -- the solve phase (steps a3-a5: Thm. 1, Lemma 1, Eq. (14))
// of the split tensor-core form for systems of 24..64 padded users.
//
// A CTA of 256 threads is four groups of 64 threads (40..64 users) or eight
// groups of one warp (24 or 32 users); each group pulls systems on its own
// and solves one at a time.  Thread i of a group holds row i of
// A = G + kappa I (UP complex registers; the pad block of A is the identity).
//
// The inverse is a blocked Gauss-Jordan without pivoting, 8 pivots per step
// (every pivot an LDL^H pivot of A, checked positive and finite):
//   * the owners of the 8 pivot rows K publish them (R = A_K,:) to shared
//     memory; one named barrier of the group;
//   * each warp inverts the 8 x 8 pivot block M = A_KK with shuffles, two
//     entries per lane, by the scalar Gauss-Jordan steps (A_ij -= (A_ip /
//     A_pp) A_pj, row p scaled by 1 / A_pp, column p set to -A_ip / A_pp, A_pp
//     to 1 / A_pp);
//   * each row forms w = A_iK M^-1 (an owner: its row of M^-1) and takes
//     A_i: -= w R outside K and A_iK = -w (an owner: A_i: = w R outside K and
//     its row of M^-1 on K) -- eight scalar pivots at once.
// The rows are kept in a frame rotated by 8 columns per step, so that the
// pivot block sits in registers 0..7; the update writes the next frame, and
// the row is back in its order after UP / 8 steps.
//
// Then t by Lemma 1 while its subtraction cancels by at most 256x (else by
// the definition, through T in shared memory), the sensitivity estimate that
// flags a system for an FP32 Gram (escalation: the group recomputes G from H
// in FP32 and solves again), scale = sqrt(rho2 / (Es t)), and z_k = T s_k from
// each thread's row, four symbols at a time.
#include "dp_blocks.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

constexpr int RS_B = 8;   // pivots per block step
constexpr int RS_KW = 4;  // symbols whitened at once
template <int UP>
struct RsGeo {
  static_assert(UP % 8 == 0 && UP >= 24 && UP <= 64, "row solve: 24..64 padded users");
  static constexpr int CW = UP;                          // columns per thread (a whole row)
  static constexpr int GT = UP <= 32 ? 32 : 64;          // threads per group (one per row)
  static constexpr int WARPS = GT / 32;
  static constexpr int GROUPS = 256 / GT;                // systems in flight per CTA
  static constexpr int THREADS = GROUPS * GT;
  static constexpr int MINB = UP <= 24 ? 2 : 1;          // CTAs per SM (registers)
  // systems per work item: the group kernel's stacking of 128 / (2 UP)
  // systems per tile (one for more than 32 users)
  static constexpr int NG = (128 / (2 * UP)) > 0 ? 128 / (2 * UP) : 1;
  static constexpr int RLD = UP + 2;                     // padded row of R
  static constexpr int GJW = 2 * RS_B * RLD + WARPS * RS_B * RS_B;  // two R, M^-1 per warp
  static constexpr int TS = UP + 1;                      // padded row of T (definition of t)
  static constexpr int SCR = GJW > UP * TS ? GJW : UP * TS;  // T aliases the Gauss-Jordan area
};

// Named barrier of group g (ids 1..2; 0 is __syncthreads).
template <int GT>
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory");
}

// Sum over the group's threads (fixed order); red: one float per warp.
template <int GT>
__device__ __forceinline__ float group_sum(float v, float *red, int g, int lt) {
  v = warp_sum(v);
  group_sync<GT>(g);
  if ((lt & 31) == 0) red[lt >> 5] = v;
  group_sync<GT>(g);
  float s = red[0];
#pragma unroll
  for (int w = 1; w < GT / 32; ++w) s += red[w];
  return s;
}

template <int GT>
__device__ __forceinline__ bool group_all(bool v, float *red, int g, int lt) {
  return group_sum<GT>(v ? 0.f : 1.f, red, g, lt) == 0.f;
}

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Blocked Gauss-Jordan inverse of the group's system (see the top of the
// file).  Thread i holds row i in a[] (original column order at entry and
// exit).  gj: the group's scratch (two [8][RLD] copies of R, M^-1 per warp).
// Returns whether a pivot was not a positive finite number (the same value in
// every thread of the group).
template <int UP>
__device__ __forceinline__ bool row_gj(float2 (&a)[UP], int i, float2 *gj, int g, int lt) {
  using G = RsGeo<UP>;
  constexpr int LD = G::RLD;
  const int lane = lt & 31;
  float2 *mw = gj + 2 * RS_B * LD + (lt >> 5) * RS_B * RS_B;
  bool bad = false;
  const int r = lane >> 2, c0 = 2 * (lane & 3);  // this lane's two entries of M
#pragma unroll 1
  for (int kb = 0; kb < UP; kb += RS_B) {
    float2 *R = gj + ((kb / RS_B) & 1) * (RS_B * LD);
    const int l0 = i - kb;
    const bool own = l0 >= 0 && l0 < RS_B;
    if (own) {
#pragma unroll
      for (int c = 0; c < UP; ++c) R[l0 * LD + c] = a[c];
    }
    group_sync<G::GT>(g);
    float2 m0 = R[r * LD + c0], m1 = R[r * LD + c0 + 1];
#pragma unroll
    for (int p = 0; p < RS_B; ++p) {
      const int rsrc = p * 4 + (lane & 3);
      const float2 q0 = shfl2(m0, rsrc), q1 = shfl2(m1, rsrc);
      const float2 mc = (p & 1) ? m1 : m0;
      const float2 pc = shfl2(mc, r * 4 + (p >> 1));
      const float piv = __shfl_sync(0xffffffffu, mc.x, p * 4 + (p >> 1));
      bad = bad || !(piv > 0.f) || !isfinite(piv);
      const float ip = 1.f / piv;
      if (r == p) {
        m0 = (c0 == p) ? make_float2(ip, 0.f) : cscale(m0, ip);
        m1 = (c0 + 1 == p) ? make_float2(ip, 0.f) : cscale(m1, ip);
      } else {
        const float2 f = cscale(pc, ip);
        if (c0 == p) m0 = make_float2(-f.x, -f.y);
        else cmsub(m0, f, q0);
        if (c0 + 1 == p) m1 = make_float2(-f.x, -f.y);
        else cmsub(m1, f, q1);
      }
    }
    mw[r * RS_B + c0] = m0;
    mw[r * RS_B + c0 + 1] = m1;
    __syncwarp();
    // w = A_iK M^-1 (an owner: m = e_l0, w negated: its new row is +w R)
    float2 wv[RS_B];
#pragma unroll
    for (int l = 0; l < RS_B; ++l) wv[l] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < RS_B; ++q) {
      const float2 mq = own ? make_float2(q == l0 ? 1.f : 0.f, 0.f) : a[q];
      const float4 *mr = reinterpret_cast<const float4 *>(mw + q * RS_B);
#pragma unroll
      for (int l = 0; l < RS_B; l += 2) {
        const float4 v = mr[l / 2];
        cmac(wv[l], mq, make_float2(v.x, v.y));
        cmac(wv[l + 1], mq, make_float2(v.z, v.w));
      }
    }
#pragma unroll
    for (int l = 0; l < RS_B; ++l)
      if (own) wv[l] = make_float2(-wv[l].x, -wv[l].y);
    // A_i: -= w R outside the pivot block, pivot row by pivot row
#pragma unroll
    for (int c = RS_B; c < UP; ++c)
      if (own) a[c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < RS_B; ++l) {
      const float4 *rl = reinterpret_cast<const float4 *>(R + l * LD);
#pragma unroll
      for (int c = RS_B; c < UP; c += 2) {
        const float4 v = rl[c / 2];
        cmsub(a[c], wv[l], make_float2(v.x, v.y));
        cmsub(a[c + 1], wv[l], make_float2(v.z, v.w));
      }
    }
    // the next frame: columns shift by 8, the pivot block's -w at the end
#pragma unroll
    for (int c = RS_B; c < UP; ++c) a[c - RS_B] = a[c];
#pragma unroll
    for (int l = 0; l < RS_B; ++l) a[UP - RS_B + l] = make_float2(-wv[l].x, -wv[l].y);
  }
  return bad;
}

template <int UP>
__global__ void __launch_bounds__(RsGeo<UP>::THREADS, RsGeo<UP>::MINB)
    k_solve_rows(const InstDesc *__restrict__ insts, const WorkItem *__restrict__ items,
                 int n_items, int *__restrict__ queue, SplitWs ws, float eps_lp) {
  using R = RsGeo<UP>;
  constexpr int CW = R::CW, GT = R::GT;
  extern __shared__ __align__(16) float2 rs_smem[];
  __shared__ int item_s[R::GROUPS];
  __shared__ float red_s[R::GROUPS][R::WARPS];
  const int tid = threadIdx.x, g = tid / GT, lt = tid % GT;
  const int i = lt;  // row of A (a whole row per thread)
  const bool row = i < UP;
  // per group: Gauss-Jordan scratch (aliased by T), symbols with RS_KW - 1 rows of slack
  const size_t gsz = (size_t)R::SCR + (size_t)(ws.kmax + RS_KW - 1) * UP;
  float2 *rb = rs_smem + (size_t)g * gsz;
  float2 *Ts = rb;                    // [UP][TS], after the inverse
  float2 *Sg = rb + R::SCR;           // [K][UP]
  float *red = red_s[g];

  for (;;) {
    // the queue counts systems: system sq of item it (NG per item)
    if (lt == 0) item_s[g] = atomicAdd(queue, 1);
    group_sync<GT>(g);
    const int q = item_s[g], it = q / R::NG, sq = q - it * R::NG, wi = q;
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const InstDesc &in = insts[w.inst];
    const SysDesc &d = in.d;
    const int U = d.U, K = d.K;
    const int sys = w.sys0 + sq, n = sys / d.nsys;
    int lo, hi;
    sys_rows(d, sys - n * d.nsys, lo, hi);
    if (sq >= w.nact || sys_is_small(d, hi - lo)) {  // none, or the B_c x B_c kernel's
      group_sync<GT>(g);
      continue;
    }
    const float kappa = sys_kappa(d, sys);
    const bool mrt = d.mrt != 0;
    const float2 *Gm = ws.G + (size_t)wi * UP * UP;  // Gm[n][m] = conj(G_mn) (or G_mn)
    // symbols (zero pads) and their finiteness
    bool fin = true;
    for (int e = lt; e < K * UP; e += GT) {
      const int k = e / UP, u = e - k * UP;
      float2 v = make_float2(0.f, 0.f);
      if (u < U) v = __ldg(in.S + ((size_t)n * K + k) * U + u);
      fin = fin && cfinite(v);
      Sg[e] = v;
    }
    int st = ws.st[wi];  // the Gram phase's verdict
    if (!group_all<GT>(fin, red, g, lt) && st == ST_OK) st = ST_NONFINITE;

    // row i of A: A_ij = conj(Gm[j][i])
    float2 a[CW];
    float g2 = 0.f;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int j = c;
      float2 v = make_float2(0.f, 0.f);
      if (row && i < U && j < U) v = cconj(__ldg(Gm + (size_t)j * UP + i));
      if (j == i) v = (i < U) ? make_float2(v.x + (mrt ? 0.f : kappa), 0.f) : make_float2(1.f, 0.f);
      a[c] = v;
      const float re = v.x - ((j == i && !mrt) ? kappa : 0.f);
      if (row && i < U && j < U) g2 = fmaf(re, re, fmaf(v.y, v.y, g2));
    }
    const float gfro = group_sum<GT>(g2, red, g, lt);

    float sc = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      const bool escalated = pass > 0;
      bool bad = false;
      if (!mrt && st == ST_OK)
        bad = row_gj<UP>(a, i, rb, g, lt);
      // precoding factor: Lemma 1, or the definition where it cancels
      float dg = 0.f, fr = 0.f;
      if (row && i < U) {
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int j = c;
          if (j == i) dg = a[c].x;
          if (j < U) fr = fmaf(a[c].x, a[c].x, fmaf(a[c].y, a[c].y, fr));
        }
      }
      const float tr = group_sum<GT>(dg, red, g, lt);
      const float fro = group_sum<GT>(fr, red, g, lt);
      float t = mrt ? tr : tr - kappa * fro;
      const float lemma_max = escalated ? kLemmaMaxRatio : kLemmaMaxRatioLP;
      if (st == ST_OK && !mrt && kappa * fro > lemma_max * tr) {
        // t = tr(T G T) = sum_ij (T G)_ij conj(T_ij): T through shared memory
        if (row) {
#pragma unroll
          for (int c = 0; c < CW; ++c) Ts[i * R::TS + c] = a[c];
        }
        group_sync<GT>(g);
        float part = 0.f;
        if (row && i < U) {
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            const int j = c;
            if (j >= U) continue;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < U; ++k)  // G_kj = conj(Gm[j][k])
              cmac(acc, Ts[i * R::TS + k], cconj(__ldg(Gm + (size_t)j * UP + k)));
            part = fmaf(acc.x, a[c].x, fmaf(acc.y, a[c].y, part));
          }
        }
        t = group_sum<GT>(part, red, g, lt);
      }
      int st1 = st;
      if (st1 == ST_OK && bad) st1 = ST_NOT_PD;
      if (st1 == ST_OK && (!(t > 0.f) || !isfinite(t))) st1 = ST_NOT_PD;
      // automatic escalation (refine = 2): the 16-bit Gram's sensitivity
      const float sens = (st1 == ST_OK && !mrt) ? sqrtf(gfro * fro) / U : 0.f;
      if (!escalated && d.refine == 2 && st1 == ST_OK && eps_lp * sens >= kRefineTrigger) {
        // FP32 Gram from H: row i of G = sum_b h_b[i] conj(h_b[j])
        // over the system's antennas (h_b = antenna row b)
        const float2 *hn = in.H + ((size_t)n * d.B + lo) * U;
#pragma unroll
        for (int c = 0; c < CW; ++c) a[c] = make_float2(0.f, 0.f);
        if (row && i < U) {
#pragma unroll 1
          for (int b = 0; b < hi - lo; ++b) {
            const float2 hv = __ldg(hn + (size_t)b * U + i);
#pragma unroll
            for (int c = 0; c < CW; ++c) {
              const int j = c;
              if (j < U) cmac_cj(a[c], __ldg(hn + (size_t)b * U + j), hv);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int j = c;
          if (j == i) a[c] = (i < U) ? make_float2(a[c].x + kappa, 0.f) : make_float2(1.f, 0.f);
        }
        continue;
      }
      st = st1;
      if (st == ST_OK) sc = sqrtf(sys_rho2(d, sys) / (d.Es * t));
      break;
    }

    // whitening z_k = T s_k (MRT: z = s), straight to the workspace
    float2 *Zw = ws.Z + (size_t)wi * ws.kmax * UP;
    for (int k0 = 0; k0 < K; k0 += RS_KW) {  // RS_KW symbols at once (independent sums)
      float2 acc[RS_KW];
#pragma unroll
      for (int q = 0; q < RS_KW; ++q) acc[q] = make_float2(0.f, 0.f);
      if (row && st == ST_OK && mrt) {
#pragma unroll
        for (int q = 0; q < RS_KW; ++q)
          if (k0 + q < K) acc[q] = Sg[(k0 + q) * UP + i];
      } else if (row && st == ST_OK) {
#pragma unroll
        for (int c = 0; c < CW; c += 2) {
#pragma unroll
          for (int q = 0; q < RS_KW; ++q) {  // rows past K read the slack
            const float4 v = *reinterpret_cast<const float4 *>(Sg + (k0 + q) * UP + c);
            cmac(acc[q], a[c], make_float2(v.x, v.y));
            cmac(acc[q], a[c + 1], make_float2(v.z, v.w));
          }
        }
      }
      if (row) {
#pragma unroll
        for (int q = 0; q < RS_KW; ++q)
          if (k0 + q < K) Zw[(k0 + q) * UP + i] = (i < U) ? acc[q] : make_float2(0.f, 0.f);
      }
    }
    if (lt == 0) {
      ws.sc[wi] = sc;
      ws.st[wi] = st;
      in.status[sys] = st;
      if (in.scale_out) in.scale_out[sys] = st == ST_OK ? sc : 0.f;
    }
    group_sync<GT>(g);  // the group is done with its shared rows, symbols and T
  }
}

template <int UP>
cudaError_t launch_rows_t(const InstDesc *insts, const WorkItem *items, int n_items, int *queue,
                          const SplitWs &ws, bool bf16, int n_sm, cudaStream_t s) {
  using R = RsGeo<UP>;
  const size_t bytes =
      (size_t)R::GROUPS * ((size_t)R::SCR + (size_t)(ws.kmax + RS_KW - 1) * UP) * 8;
  cudaError_t e = cudaFuncSetAttribute(k_solve_rows<UP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_solve_rows<UP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(n_sm * R::MINB, n_items * R::NG));
  k_solve_rows<UP><<<grid, R::THREADS, bytes, s>>>(insts, items, n_items, queue, ws,
                                                   bf16 ? 0x1p-8f : 0x1p-11f);
  return cudaGetLastError();
}

}  // namespace

bool row_solve_supported(int UP) { return UP >= 24 && UP <= 64 && UP % 8 == 0; }

cudaError_t launch_solve_rows(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                              int n_items, int *queue, const SplitWs &ws, int n_sm,
                              cudaStream_t s) {
  switch (UP) {
    case 24: return launch_rows_t<24>(insts, items, n_items, queue, ws, bf16, n_sm, s);
    case 32: return launch_rows_t<32>(insts, items, n_items, queue, ws, bf16, n_sm, s);
    case 40: return launch_rows_t<40>(insts, items, n_items, queue, ws, bf16, n_sm, s);
    case 48: return launch_rows_t<48>(insts, items, n_items, queue, ws, bf16, n_sm, s);
    case 56: return launch_rows_t<56>(insts, items, n_items, queue, ws, bf16, n_sm, s);
    case 64: return launch_rows_t<64>(insts, items, n_items, queue, ws, bf16, n_sm, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dp
