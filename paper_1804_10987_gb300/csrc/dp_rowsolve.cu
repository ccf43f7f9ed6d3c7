// dp_rowsolve.cu -- the solve phase (steps a3-a5: Thm. 1, Lemma 1, Eq. (14))
// of the split tensor-core form for systems of 40..64 padded users, one row
// of A per thread.
//
// A CTA of 256 threads is four groups of 64 threads; each group pulls work
// items on its own and solves one system at a time.  Thread i of a group
// holds row i of A = G + kappa I (UP complex registers; the pad block of A is
// the identity).  Gauss-Jordan without pivoting, every element with the
// arithmetic of the other solves (A_ij -= (A_ip / A_pp) A_pj, row p scaled by
// 1 / A_pp, column p set to -A_ip / A_pp, A_pp to 1 / A_pp).  The pivot row is
// published by its owner into a double-buffered shared row, one named barrier
// of the group per pivot; every thread reads it as broadcasts, two entries per
// load.  The columns rotate by 4 after every 4 pivots, so that the pivot
// column sits at a register index known at compile time (the row returns to
// its order after UP pivots).
//
// Then t by Lemma 1 while its subtraction cancels by at most 256x (else by
// the definition, through T in shared memory), the sensitivity estimate that
// flags a system for an FP32 Gram (escalation: the group recomputes G from H
// in FP32 and solves again), scale = sqrt(rho2 / (Es t)), and z_k = T s_k from
// each thread's row.
#include "dp_blocks.cuh"
#include "dp_internal.h"

namespace dp {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_GROUP = 64;   // threads per group (one row each)
constexpr int RS_R = 4;        // pivots between rotations

template <int UP>
struct RsGeo {
  static_assert(UP % 8 == 0 && UP > 32 && UP <= 64, "row solve: 40..64 padded users");
  static constexpr int CW = UP;                     // columns per thread
  static_assert(CW % RS_R == 0 && CW % 2 == 0, "whole rotation blocks");
  static constexpr int GROUPS = RS_THREADS / RS_GROUP;
  static constexpr int ROWB = 2 * UP;               // two published rows (complex)
  static constexpr int TS = UP + 1;                 // padded row of T (definition of t)
};

// Named barrier of group g (ids 1..2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(RS_GROUP) : "memory");
}

// Sum over the group's threads (fixed order); red: 2 floats of the group.
__device__ __forceinline__ float group_sum(float v, float *red, int g, int lt) {
  v = warp_sum(v);
  group_sync(g);
  if ((lt & 31) == 0) red[lt >> 5] = v;
  group_sync(g);
  return red[0] + red[1];
}

__device__ __forceinline__ bool group_all(bool v, float *red, int g, int lt) {
  return group_sum(v ? 0.f : 1.f, red, g, lt) == 0.f;
}

// Rotate a row left by RS_R columns.
template <int CW>
__device__ __forceinline__ void rotate(float2 (&a)[CW]) {
  float2 t[RS_R];
#pragma unroll
  for (int c = 0; c < RS_R; ++c) t[c] = a[c];
#pragma unroll
  for (int c = 0; c < CW - RS_R; ++c) a[c] = a[c + RS_R];
#pragma unroll
  for (int c = 0; c < RS_R; ++c) a[CW - RS_R + c] = t[c];
}

// Gauss-Jordan inverse of the group's system: thread i holds row i in a[]
// (original column order at entry and exit).  rb: two published rows.
// Returns whether a pivot was not a positive finite number (the same value in
// every thread of the group).
template <int UP>
__device__ __forceinline__ bool row_gj(float2 (&a)[UP], int i, float2 *rb, int g) {
  bool bad = false;
  if (i == 0) {
#pragma unroll
    for (int c = 0; c < UP; ++c) rb[c] = a[c];
  }
  group_sync(g);
#pragma unroll 1
  for (int blk = 0; blk < UP / RS_R; ++blk) {
#pragma unroll
    for (int pl = 0; pl < RS_R; ++pl) {
      const int p = RS_R * blk + pl;  // pivot; its column sits at register pl
      const float2 *rp = rb + (pl & 1) * UP;
      const float piv = rp[pl].x;
      bad = bad || !(piv > 0.f) || !isfinite(piv);
      const float ip = 1.f / piv;
      const float2 fv = cscale(a[pl], ip);
      const float4 *rq = reinterpret_cast<const float4 *>(rp);
      if (i == p) {
#pragma unroll
        for (int c = 0; c < UP; c += 2) {
          const float4 w = rq[c / 2];
          a[c] = (c == pl) ? make_float2(ip, 0.f) : make_float2(w.x * ip, w.y * ip);
          a[c + 1] = (c + 1 == pl) ? make_float2(ip, 0.f) : make_float2(w.z * ip, w.w * ip);
        }
      } else {
#pragma unroll
        for (int c = 0; c < UP; c += 2) {
          const float4 w = rq[c / 2];
          if (c == pl) a[c] = make_float2(-fv.x, -fv.y);
          else cmsub(a[c], fv, make_float2(w.x, w.y));
          if (c + 1 == pl) a[c + 1] = make_float2(-fv.x, -fv.y);
          else cmsub(a[c + 1], fv, make_float2(w.z, w.w));
        }
      }
      if (i == p + 1) {  // publish the next pivot row (in its pivot's rotation)
        float2 *wp = rb + ((pl + 1) & 1) * UP;
        if (pl == RS_R - 1) {
#pragma unroll
          for (int c = 0; c < UP; ++c) wp[c] = a[(c + RS_R) % UP];
        } else {
#pragma unroll
          for (int c = 0; c < UP; ++c) wp[c] = a[c];
        }
      }
      group_sync(g);
    }
    rotate<UP>(a);
  }
  return bad;
}

template <int UP>
__global__ void __launch_bounds__(RS_THREADS, 1)
    k_solve_rows(const InstDesc *__restrict__ insts, const WorkItem *__restrict__ items,
                 int n_items, int *__restrict__ queue, SplitWs ws, float eps_lp) {
  using R = RsGeo<UP>;
  constexpr int CW = R::CW;
  extern __shared__ __align__(16) float2 rs_smem[];
  __shared__ int item_s[R::GROUPS];
  __shared__ float red_s[R::GROUPS][2];
  const int tid = threadIdx.x, g = tid / RS_GROUP, lt = tid % RS_GROUP;
  const int i = lt, h = 0;            // row of A (one whole row per thread)
  const bool row = i < UP;
  const size_t gsz = (size_t)R::ROWB + (size_t)ws.kmax * UP + (size_t)UP * R::TS;
  float2 *rb = rs_smem + (size_t)g * gsz;
  float2 *Sg = rb + R::ROWB;                  // [K][UP]
  float2 *Ts = Sg + (size_t)ws.kmax * UP;     // [UP][TS]
  float *red = red_s[g];

  for (;;) {
    if (lt == 0) item_s[g] = atomicAdd(queue, 1);
    group_sync(g);
    const int it = item_s[g];
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const InstDesc &in = insts[w.inst];
    const SysDesc &d = in.d;
    const int U = d.U, K = d.K;
    const int sys = w.sys0, n = sys / d.nsys;
    int lo, hi;
    sys_rows(d, sys - n * d.nsys, lo, hi);
    if (w.nact < 1 || sys_is_small(d, hi - lo)) {  // the B_c x B_c kernel's system
      group_sync(g);
      continue;
    }
    const float kappa = d.kappa;
    const bool mrt = d.mrt != 0;
    const float2 *Gm = ws.G + (size_t)it * UP * UP;  // Gm[n][m] = conj(G_mn)
    // symbols (zero pads) and their finiteness
    bool fin = true;
    for (int e = lt; e < K * UP; e += RS_GROUP) {
      const int k = e / UP, u = e - k * UP;
      float2 v = make_float2(0.f, 0.f);
      if (u < U) v = __ldg(in.S + ((size_t)n * K + k) * U + u);
      fin = fin && cfinite(v);
      Sg[e] = v;
    }
    int st = ws.st[it];  // the Gram phase's verdict
    if (!group_all(fin, red, g, lt) && st == ST_OK) st = ST_NONFINITE;

    // half h of row i of A: A_ij = conj(Gm[j][i])
    float2 a[CW];
    float g2 = 0.f;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int j = h * CW + c;
      float2 v = make_float2(0.f, 0.f);
      if (row && i < U && j < U) v = cconj(__ldg(Gm + (size_t)j * UP + i));
      if (j == i) v = (i < U) ? make_float2(v.x + (mrt ? 0.f : kappa), 0.f) : make_float2(1.f, 0.f);
      a[c] = v;
      const float re = v.x - ((j == i && !mrt) ? kappa : 0.f);
      if (row && i < U && j < U) g2 = fmaf(re, re, fmaf(v.y, v.y, g2));
    }
    const float gfro = group_sum(g2, red, g, lt);

    float sc = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      const bool escalated = pass > 0;
      bool bad = false;
      if (!mrt && st == ST_OK) bad = row_gj<UP>(a, i, rb, g);
      // precoding factor: Lemma 1, or the definition where it cancels
      float dg = 0.f, fr = 0.f;
      if (row && i < U) {
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int j = h * CW + c;
          if (j == i) dg = a[c].x;
          if (j < U) fr = fmaf(a[c].x, a[c].x, fmaf(a[c].y, a[c].y, fr));
        }
      }
      const float tr = group_sum(dg, red, g, lt);
      const float fro = group_sum(fr, red, g, lt);
      float t = mrt ? tr : tr - kappa * fro;
      const float lemma_max = escalated ? kLemmaMaxRatio : kLemmaMaxRatioLP;
      if (st == ST_OK && !mrt && kappa * fro > lemma_max * tr) {
        // t = tr(T G T) = sum_ij (T G)_ij conj(T_ij): T through shared memory
        if (row) {
#pragma unroll
          for (int c = 0; c < CW; ++c) Ts[i * R::TS + h * CW + c] = a[c];
        }
        group_sync(g);
        float part = 0.f;
        if (row && i < U) {
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            const int j = h * CW + c;
            if (j >= U) continue;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < U; ++k)  // G_kj = conj(Gm[j][k])
              cmac(acc, Ts[i * R::TS + k], cconj(__ldg(Gm + (size_t)j * UP + k)));
            part = fmaf(acc.x, a[c].x, fmaf(acc.y, a[c].y, part));
          }
        }
        t = group_sum(part, red, g, lt);
      }
      int st1 = st;
      if (st1 == ST_OK && bad) st1 = ST_NOT_PD;
      if (st1 == ST_OK && (!(t > 0.f) || !isfinite(t))) st1 = ST_NOT_PD;
      // automatic escalation (refine = 2): the 16-bit Gram's sensitivity
      const float sens = (st1 == ST_OK && !mrt) ? sqrtf(gfro * fro) / U : 0.f;
      if (!escalated && d.refine == 2 && st1 == ST_OK && eps_lp * sens >= kRefineTrigger) {
        // FP32 Gram from H: half h of row i of G = sum_b h_b[i] conj(h_b[j])
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
              const int j = h * CW + c;
              if (j < U) cmac_cj(a[c], __ldg(hn + (size_t)b * U + j), hv);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int j = h * CW + c;
          if (j == i) a[c] = (i < U) ? make_float2(a[c].x + kappa, 0.f) : make_float2(1.f, 0.f);
        }
        continue;
      }
      st = st1;
      if (st == ST_OK) sc = sqrtf(d.rho2_sys / (d.Es * t));
      break;
    }

    // whitening z_k = T s_k (MRT: z = s), straight to the workspace
    float2 *Zw = ws.Z + (size_t)it * ws.kmax * UP;
    if (row) {
      for (int k = 0; k < K; ++k) {
        float2 acc = make_float2(0.f, 0.f);
        if (st == ST_OK) {
          if (mrt) {
            if (h == 0) acc = Sg[k * UP + i];
          } else {
            const float4 *sk = reinterpret_cast<const float4 *>(Sg + k * UP + h * CW);
#pragma unroll
            for (int c = 0; c < CW; c += 2) {
              const float4 v = sk[c / 2];
              cmac(acc, a[c], make_float2(v.x, v.y));
              cmac(acc, a[c + 1], make_float2(v.z, v.w));
            }
          }
        }
        Zw[k * UP + i] = (i < U) ? acc : make_float2(0.f, 0.f);
      }
    }
    if (lt == 0) {
      ws.sc[it] = sc;
      ws.st[it] = st;
      in.status[sys] = st;
      if (in.scale_out) in.scale_out[sys] = st == ST_OK ? sc : 0.f;
    }
    group_sync(g);  // the group is done with its shared rows, symbols and T
  }
}

template <int UP>
cudaError_t launch_rows_t(const InstDesc *insts, const WorkItem *items, int n_items, int *queue,
                          const SplitWs &ws, bool bf16, int grid, cudaStream_t s) {
  using R = RsGeo<UP>;
  const size_t bytes =
      (size_t)R::GROUPS * ((size_t)R::ROWB + (size_t)ws.kmax * UP + (size_t)UP * R::TS) * 8;
  cudaError_t e = cudaFuncSetAttribute(k_solve_rows<UP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_solve_rows<UP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k_solve_rows<UP><<<grid, RS_THREADS, bytes, s>>>(insts, items, n_items, queue, ws,
                                                   bf16 ? 0x1p-8f : 0x1p-11f);
  return cudaGetLastError();
}

}  // namespace

bool row_solve_supported(int UP) { return UP > 32 && UP <= 64 && UP % 8 == 0; }

cudaError_t launch_solve_rows(int UP, bool bf16, const InstDesc *insts, const WorkItem *items,
                              int n_items, int *queue, const SplitWs &ws, int grid,
                              cudaStream_t s) {
  switch (UP) {
    case 40: return launch_rows_t<40>(insts, items, n_items, queue, ws, bf16, grid, s);
    case 48: return launch_rows_t<48>(insts, items, n_items, queue, ws, bf16, grid, s);
    case 56: return launch_rows_t<56>(insts, items, n_items, queue, ws, bf16, grid, s);
    case 64: return launch_rows_t<64>(insts, items, n_items, queue, ws, bf16, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dp
