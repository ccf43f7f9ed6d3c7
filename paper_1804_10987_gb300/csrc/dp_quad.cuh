// dp_quad.cuh -- the regularize / factor / precoding-factor / whitening steps
// (a3-a5: Thm. 1, Lemma 1, Eq. (14)) for systems of 24..64 padded users,
// solved by a whole CTA of NT = 256 threads in the "quad-row" layout.
//
// Row i of A = G + kappa I is split over four adjacent lanes: quarter q holds
// columns [q QW, (q + 1) QW), QW = UP / 4, in registers.  With UP <= 32 a CTA
// holds two systems (system s on threads [128 s, 128 s + 4 UP)), with UP > 32
// one (threads [0, 4 UP)).  Gauss-Jordan without pivoting runs over all UP
// pivots: the pad block of A (rows and columns U..UP) is the identity, so the
// pads stay exact and every system of the CTA pivots in step.  One CTA
// barrier per pivot: after its update for pivot p the owners of row p + 1
// publish it into a double-buffered shared row, and column p reaches the
// other lanes of a row by a shuffle from the lane that holds it.  Every
// element takes the same arithmetic as the row-per-lane Gauss-Jordan of
// dp_blocks.cuh (warp_gj_inverse): A_ij -= (A_ip / A_pp) A_pj, row p scaled
// by 1 / A_pp, column p set to -A_ip / A_pp, A_pp to 1 / A_pp.
//
// Then t = tr(A^{-1} G A^{-1}) by Lemma 1, tr(T) - kappa ||T||_F^2, while
// its subtraction cancels by at most 1 / (1 - lemma_max), else by the
// definition sum_ij (T G)_ij conj(T_ij); scale = sqrt(rho2 / (Es t)); and
// z_k = T s_k from each lane's quarter of row i, summed over the four lanes.
#pragma once

#include "dp_blocks.cuh"

namespace dp {

template <int UP>
struct Quad {
  static_assert(UP % 8 == 0 && UP >= 24 && UP <= 64, "quad-row solve: 24..64 padded users");
  static constexpr int QW = UP / 4;                    // columns per lane
  static constexpr int NS = UP <= 32 ? 2 : 1;          // systems per CTA
  static constexpr int TPS = NT / NS;                  // thread slots per system
  // stride of a published row's quarters (complex entries), padded so that
  // the four 16-byte reads of one request fall in distinct bank groups
  static constexpr int QS = (QW == 6 || QW == 14) ? QW + 4 : QW + 2;
  static constexpr int ROWBUF = 4 * QS;                // one published row
  // shared scratch: 2 published rows per system, then (definition of t) T
  // with rows padded by one entry
  static constexpr int TS = UP + 1;
  static constexpr size_t SCRATCH_BYTES =
      (size_t)NS * UP * TS * 8 > (size_t)NS * 2 * ROWBUF * 8 ? (size_t)NS * UP * TS * 8
                                                            : (size_t)NS * 2 * ROWBUF * 8;
  static_assert(NS * TPS == NT && 4 * UP <= TPS, "thread slots");
  static_assert(QW % 2 == 0, "pivot parity is compile-time");
};

// Per-system sum over the CTA (warps of system s are [s TPS / 32, (s + 1)
// TPS / 32)), fixed order.  red: NT / 32 floats.  Every thread calls it.
template <int NS>
__device__ __forceinline__ float quad_sys_sum(float v, float *red, int tid) {
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  constexpr int W = NT / 32 / NS;
  const int s = tid / (NT / NS);
  float r = 0.f;
#pragma unroll
  for (int w = 0; w < W; ++w) r += red[s * W + w];
  return r;
}

// The NS systems of a CTA (systems >= nact or with skip_s set are left
// alone).  Gs: [NS][UP][UP] with zero pads; Ss: [NS][K][UP] with zero pads;
// Zs: [NS][K][UP] (written for every live system: z, or zeros on failure);
// st_s: in: ST_OK or the input's failure; out: the system's status; sc_s:
// out: scale (0 on failure).  scratch: Quad<UP>::SCRATCH_BYTES of shared
// memory; sd, sys0: the descriptor and the first system (for each system's
// kappa and rho^2); red: NT / 32 floats; Tout: if non-NULL, T = A^{-1} [NS][UP][UP]
// (rows and columns >= U undefined); sens_s: if non-NULL, out: the
// sensitivity estimate ||G||_F ||T||_F / U of every live system (0 for MRT
// and on failure).  Every thread of the CTA calls it.
template <int UP>
__device__ void quad_solve(const float2 *Gs, const float2 *Ss, float2 *Zs, int *st_s,
                           float *sc_s, const int *skip_s, int nact, const SysDesc &sd,
                           int sys0, float Es, int U, int K, bool mrt, float lemma_max,
                           float2 *scratch,
                           float *red, float2 *Tout, float *sens_s, int tid) {
  using Q = Quad<UP>;
  constexpr int QW = Q::QW, QS = Q::QS, NS = Q::NS;
  const int s = tid / Q::TPS, t = tid - s * Q::TPS;
  const int i = t >> 2, q = t & 3;
  const int lane = tid & 31;
  const bool row = i < UP;  // warp-uniform: 4 UP is a multiple of 32
  const bool sys_live = s < nact && !skip_s[s];
  // this system's regularizer and power (per cluster for FD-WF)
  const float kappa = sys_kappa(sd, sys0 + s), rho2 = sys_rho2(sd, sys0 + s);
  const bool live = sys_live && st_s[s] == ST_OK;
  const float2 *G = Gs + (size_t)s * UP * UP;
  float2 *rb = scratch + (size_t)s * 2 * Q::ROWBUF;  // [2][4][QS]

  // A = G + kappa I (MRT: A = G), pads: identity.  A_ij = conj(G_ji): the
  // lanes of a request then read consecutive entries
  float2 a[QW];
#pragma unroll
  for (int c = 0; c < QW; ++c) {
    const int j = q * QW + c;
    float2 v = make_float2(0.f, 0.f);
    if (row) {
      if (i < U && j < U) v = cconj(G[j * UP + i]);
      if (i == j) v = (i < U) ? make_float2(v.x + (mrt ? 0.f : kappa), 0.f) : make_float2(1.f, 0.f);
    }
    a[c] = v;
  }
  float g2 = 0.f;  // ||G||_F^2 over the U x U block
  if (row && i < U) {
#pragma unroll
    for (int c = 0; c < QW; ++c) {
      const int j = q * QW + c;
      const float re = a[c].x - ((j == i && !mrt) ? kappa : 0.f);
      if (j < U) g2 = fmaf(re, re, fmaf(a[c].y, a[c].y, g2));
    }
  }

  bool bad = false;
  if (!mrt) {
    if (row && i == 0) {
#pragma unroll
      for (int c = 0; c < QW; ++c) rb[q * QS + c] = a[c];
    }
    __syncthreads();
    const int src = (lane & ~3);
    for (int qp = 0; qp < 4; ++qp) {
#pragma unroll
      for (int pr = 0; pr < QW; ++pr) {
        const int p = qp * QW + pr;
        const float2 *rp = rb + (pr & 1) * Q::ROWBUF;
        float2 f;  // A_ip, held by lane (i, qp) at register pr
        f.x = __shfl_sync(FULL, a[pr].x, src | qp);
        f.y = __shfl_sync(FULL, a[pr].y, src | qp);
        if (row) {
          const float piv = rp[qp * QS + pr].x;
          bad = bad || !(piv > 0.f) || !isfinite(piv);
          const float ip = 1.f / piv;
          const float2 fv = cscale(f, ip);
          const float4 *rq = reinterpret_cast<const float4 *>(rp + q * QS);
          // row p two entries at a time, used as read (few live registers)
          if (i == p) {
#pragma unroll
            for (int c = 0; c < QW; c += 2) {
              const float4 w = rq[c / 2];
              a[c] = (c == pr && q == qp) ? make_float2(ip, 0.f) : make_float2(w.x * ip, w.y * ip);
              a[c + 1] = (c + 1 == pr && q == qp) ? make_float2(ip, 0.f)
                                                  : make_float2(w.z * ip, w.w * ip);
            }
          } else {
#pragma unroll
            for (int c = 0; c < QW; c += 2) {
              const float4 w = rq[c / 2];
              if (c == pr && q == qp) a[c] = make_float2(-fv.x, -fv.y);
              else cmsub(a[c], fv, make_float2(w.x, w.y));
              if (c + 1 == pr && q == qp) a[c + 1] = make_float2(-fv.x, -fv.y);
              else cmsub(a[c + 1], fv, make_float2(w.z, w.w));
            }
          }
          if (i == p + 1) {  // publish the next pivot row
            float2 *wp = rb + ((pr + 1) & 1) * Q::ROWBUF + q * QS;
#pragma unroll
            for (int c = 0; c < QW; c += 2)
              *reinterpret_cast<float4 *>(wp + c) = make_float4(a[c].x, a[c].y, a[c + 1].x,
                                                                a[c + 1].y);
          }
        }
        __syncthreads();
      }
    }
  }

  // ---- precoding factor -----------------------------------------------------
  float dg = 0.f, fr = 0.f;
  if (row && i < U) {
#pragma unroll
    for (int c = 0; c < QW; ++c) {
      const int j = q * QW + c;
      if (j == i) dg = a[c].x;
      if (j < U) fr = fmaf(a[c].x, a[c].x, fmaf(a[c].y, a[c].y, fr));
    }
  }
  const float tr = quad_sys_sum<NS>(dg, red, tid);
  const float fro = quad_sys_sum<NS>(fr, red, tid);
  const float gfro = sens_s ? quad_sys_sum<NS>(g2, red, tid) : 0.f;
  float tt = mrt ? tr : tr - kappa * fro;
  const bool need = live && !mrt && kappa * fro > lemma_max * tr;
  if (__syncthreads_or(need)) {
    // the definition tr(T G T): T into scratch (rows padded), then lane
    // (i, q) sums conj(T_ij) (T G)_ij over its columns j
    float2 *Ts = scratch + (size_t)s * UP * Q::TS;
    if (row) {
#pragma unroll
      for (int c = 0; c < QW; ++c) Ts[i * Q::TS + q * QW + c] = a[c];
    }
    __syncthreads();
    float part = 0.f;
    if (row && i < U) {
#pragma unroll
      for (int c = 0; c < QW; ++c) {
        const int j = q * QW + c;
        if (j >= U) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < U; ++k) cmac(acc, Ts[i * Q::TS + k], G[k * UP + j]);
        part = fmaf(acc.x, a[c].x, fmaf(acc.y, a[c].y, part));
      }
    }
    const float talt = quad_sys_sum<NS>(part, red, tid);
    if (need) tt = talt;
  }
  int st = live ? (bad ? ST_NOT_PD : ST_OK) : (sys_live ? st_s[s] : ST_OK);
  float sc = 0.f;
  if (st == ST_OK && live) {
    if (!(tt > 0.f) || !isfinite(tt)) st = ST_NOT_PD;
    else sc = sqrtf(rho2 / (Es * tt));
  }

  // ---- whitening z_k = T s_k (MRT: z = s) ------------------------------------
  if (row && sys_live) {
    const float2 *sk = Ss + (size_t)s * K * UP;
    float2 *zk = Zs + (size_t)s * K * UP;
    for (int k = 0; k < K; ++k) {
      float2 acc = make_float2(0.f, 0.f);
      if (st == ST_OK) {
        if (mrt) {
          if (q == 0) acc = sk[k * UP + i];
        } else {
#pragma unroll
          for (int c = 0; c < QW; ++c) cmac(acc, a[c], sk[k * UP + q * QW + c]);
        }
      }
      acc.x += __shfl_xor_sync(FULL, acc.x, 1);
      acc.y += __shfl_xor_sync(FULL, acc.y, 1);
      acc.x += __shfl_xor_sync(FULL, acc.x, 2);
      acc.y += __shfl_xor_sync(FULL, acc.y, 2);
      if (q == 0) zk[k * UP + i] = (i < U) ? acc : make_float2(0.f, 0.f);
    }
  } else {
    // lanes of rows past UP and of absent systems still join the shuffles'
    // warps: every lane of a warp takes the same branch (rows are
    // warp-uniform and a warp belongs to one system)
  }
  if (Tout && row && sys_live) {
    float2 *T = Tout + (size_t)s * UP * UP;
#pragma unroll
    for (int c = 0; c < QW; ++c) T[i * UP + q * QW + c] = a[c];
  }
  __syncthreads();  // every lane is done with Gs, Ss and the scratch
  if (t == 0 && sys_live) {
    st_s[s] = st;
    sc_s[s] = sc;
    if (sens_s) sens_s[s] = (st == ST_OK && live && !mrt) ? sqrtf(gfro * fro) / (float)U : 0.f;
  }
  __syncthreads();
}

}  // namespace dp
