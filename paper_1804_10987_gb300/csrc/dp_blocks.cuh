// dp_blocks.cuh -- device building blocks of the FP32 precoding path.
//
// Shared-memory tile of one system's channel: rows = antennas b, each row the
// U user entries H[b][0..U) as complex floats, padded to UP (a multiple of 8)
// with zeros, row stride RS = 2 UP + 4 floats.  The 16-byte pad makes a
// thread-per-row walk (the apply) hit distinct bank groups within every
// quarter warp, while the Gram's same-row reads broadcast.
#pragma once

#include "dp_common.cuh"

namespace dp {

constexpr int NT = 256;  // threads per CTA of the per-system kernels

// Lemma 1 is used for t while kappa ||T||_F^2 <= kLemmaMaxRatio tr(T), i.e.
// while its subtraction amplifies rounding errors by at most 1 / (1 - 0.875)
// = 8; beyond that t is formed as tr(T G T).
constexpr float kLemmaMaxRatio = 0.875f;
// The reduced-precision (BF16 / FP16 Gram) path keeps Lemma 1 up to an
// amplification of 256: with FP32 sums of U <= 64 terms that bounds its
// rounding contribution to t near 256 * 64 * 2^-24 ~ 1e-3 in the worst case
// and ~1e-5 typically, against the same path's 1e-3 bar, where the 16-bit
// Gram itself contributes ~1e-4.  Beyond it t is formed as tr(T G T).
constexpr float kLemmaMaxRatioLP = 1.0f - 1.0f / 256.0f;

constexpr int pow2_floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

template <int UP>
struct Geo {
  static_assert(UP % 8 == 0 && UP >= 8 && UP <= 64, "UP must be 8..64, a multiple of 8");
  static constexpr int RS = 2 * UP + 4;
  static constexpr int M = UP / 4;                 // 4 x 4 tiles per side of G
  static constexpr int NTILES = M * (M + 1) / 2;   // lower-triangular tiles
  static constexpr int NBG0 = pow2_floor(NT / NTILES);
  // antenna groups per tile: a power of two <= 32 so that a group is a
  // lane-aligned slice of one warp and reduces with xor shuffles
  static constexpr int NBG = NBG0 > 32 ? 32 : (NBG0 < 1 ? 1 : NBG0);
  static_assert(NTILES * NBG <= NT, "one Gram item per thread");
};

// ------------------------------------------------------------ row fetch ---
// Fetch rows [lo, lo + nrows) of one subcarrier's channel Hn (rows of U
// complex) into the padded tile Hs.  With tma, warp 0 posts the byte count on
// bar and issues one 1-D bulk copy per row (the caller waits on bar);
// otherwise all threads copy with plain loads (the caller syncs).
template <int UP>
__device__ __forceinline__ void fetch_rows(float *Hs, const float2 *__restrict__ Hn, int lo,
                                           int nrows, int U, bool tma, uint64_t *bar, int tid) {
  constexpr int RS = Geo<UP>::RS;
  if (tma) {
    if (tid < 32) {
      if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)nrows * (uint32_t)U * 8u);
      __syncwarp();
      for (int r = tid; r < nrows; r += 32)
        tma_load_1d(Hs + r * RS, Hn + (size_t)(lo + r) * U, (uint32_t)U * 8u, bar);
    }
  } else {
    for (int e = tid; e < nrows * U; e += NT) {
      int r = e / U, u = e - r * U;
      float2 v = __ldg(Hn + (size_t)(lo + r) * U + u);
      *reinterpret_cast<float2 *>(Hs + r * RS + 2 * u) = v;
    }
  }
}

// Zero the pad columns [U, UP) of rows [0, nrows) (once per buffer: bulk
// copies write only the first U entries of a row).
template <int UP>
__device__ __forceinline__ void zero_row_pads(float *Hs, int nrows, int U, int tid) {
  constexpr int RS = Geo<UP>::RS;
  const int w = RS - 2 * U;
  for (int e = tid; e < nrows * w; e += NT) {
    int r = e / w, c = e - r * w;
    Hs[r * RS + 2 * U + c] = 0.f;
  }
}

// ------------------------------------------------------------------ Gram ---
// G = sum over the tile's rows of h_b h_b^H (h_b = row b), accumulated by
// 4 x 4 register tiles of the lower triangle; each tile is split over NBG
// antenna groups (rows b = bg mod NBG), reduced with xor shuffles at the end.
template <int UP>
struct GramAcc {
  float2 acc[4][4];
  int ti, tj, bg;
  bool active;

  __device__ __forceinline__ void init(int tid) {
    constexpr int NB = Geo<UP>::NBG, NTL = Geo<UP>::NTILES;
    active = tid < NTL * NB;
    int tile = tid / NB;
    bg = tid % NB;
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= tile) ++i;
    ti = i;
    tj = tile - i * (i + 1) / 2;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = make_float2(0.f, 0.f);
  }

  // Rows [0, nrows) of Hs; nrows may vary between calls (chunks), the group
  // assignment restarts at row 0 of every chunk.
  __device__ __forceinline__ void accumulate(const float *Hs, int nrows) {
    constexpr int NB = Geo<UP>::NBG, RS = Geo<UP>::RS;
    if (!active) return;
    for (int r = bg; r < nrows; r += NB) {
      const float4 *row = reinterpret_cast<const float4 *>(Hs + r * RS);
      float4 a0 = row[2 * ti], a1 = row[2 * ti + 1];
      float4 b0 = row[2 * tj], b1 = row[2 * tj + 1];
      float2 a[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                     make_float2(a1.z, a1.w)};
      float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                     make_float2(b1.z, b1.w)};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) cmac_cj(acc[p][q], b[q], a[p]);  // += a_p conj(b_q)
    }
  }

  // Reduce over the antenna groups and store the tile and its Hermitian
  // mirror into G [UP][UP] (shared).  Every thread of the CTA must call it.
  __device__ __forceinline__ void finish(float2 *G, int tid) {
    constexpr int NB = Geo<UP>::NBG;
    if (!active) return;
    const int lane = tid & 31;
    const unsigned mask = (NB == 32) ? FULL : (((1u << NB) - 1u) << (lane & ~(NB - 1)));
#pragma unroll
    for (int o = NB / 2; o >= 1; o >>= 1)
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[p][q].x += __shfl_xor_sync(mask, acc[p][q].x, o);
          acc[p][q].y += __shfl_xor_sync(mask, acc[p][q].y, o);
        }
    if (bg != 0) return;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * ti + p, j = 4 * tj + q;
        if (ti == tj && q > p) continue;
        float2 v = acc[p][q];
        if (i == j) v.y = 0.f;
        G[i * UP + j] = v;
        G[j * UP + i] = cconj(v);
      }
  }
};

// ------------------------------------------------------------ reductions ---
// Deterministic CTA sum (fixed shuffle tree, then warps in order).
__device__ __forceinline__ float cta_sum(float v, float *red, int tid) {
  v = warp_sum(v);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// MRT's precoding factor t = tr(G) over a CTA (G [UP][UP] in shared memory),
// and z = s (Ss, Zs [K][UP]).
template <int UP>
__device__ float cta_mrt(const float2 *G, const float2 *Ss, float2 *Zs, int U, int K, float *red,
                         int tid) {
  float v = 0.f;
  for (int i = tid; i < U; i += NT) v += G[i * UP + i].x;
  for (int e = tid; e < K * UP; e += NT) Zs[e] = Ss[e];
  return cta_sum(v, red, tid);
}

// ------------------------------------------------- CTA-wide inversion ------
// In-place Gauss-Jordan inversion of the Hermitian positive definite A
// [UP][UP] (leading U x U block), no pivoting: for a positive definite matrix
// the pivots are the LDL^H pivots and stay positive.  Returns ST_OK or
// ST_NOT_PD on a pivot that is not a positive finite number.  Caller has
// synced after writing A.
template <int UP>
__device__ int cta_gj_inverse(float2 *A, int U, int tid) {
  for (int p = 0; p < U; ++p) {
    const float piv = A[p * UP + p].x;
    if (!(piv > 0.f) || !isfinite(piv)) return ST_NOT_PD;  // uniform over the CTA
    const float ip = 1.f / piv;
    for (int e = tid; e < U * UP; e += NT) {
      const int i = e / UP, j = e - i * UP;
      if (j < U && i != p && j != p) {
        float2 f = cscale(A[i * UP + p], ip);
        cmsub(A[i * UP + j], f, A[p * UP + j]);
      }
    }
    __syncthreads();
    if (tid < U) {
      if (tid != p) A[p * UP + tid] = cscale(A[p * UP + tid], ip);
    } else if (tid < 2 * U) {
      const int i = tid - U;
      if (i != p) A[i * UP + p] = cscale(A[i * UP + p], -ip);
    } else if (tid == 2 * U) {
      A[p * UP + p] = make_float2(ip, 0.f);
    }
    __syncthreads();
  }
  return ST_OK;
}

// The same Gauss-Jordan with A held in registers: thread (bi, bj) of a 16 x 16
// grid (NT = 256) owns the RB x RB block of rows bi RB + r and columns
// bj RB + c (RB = ceil(UP / 16)).  Before pivot p the owners publish row p
// and column p into rc [2][2][UP] (double-buffered by pivot parity: one CTA
// barrier per pivot).  The arithmetic of every element is that of
// cta_gj_inverse, so the results are identical.  A is read at entry and
// holds A^{-1} at exit; the caller has synced after writing A.
template <int UP>
__device__ int cta_gj_inverse_reg(float2 *A, int U, int tid, float2 *rc) {
  static_assert(NT == 256, "a 16 x 16 thread grid");
  constexpr int RB = (UP + 15) / 16;
  const int bi = tid >> 4, bj = tid & 15;
  float2 a[RB][RB];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int c = 0; c < RB; ++c) {
      const int i = bi * RB + r, j = bj * RB + c;
      a[r][c] = (i < UP && j < UP) ? A[i * UP + j] : make_float2(0.f, 0.f);
    }
  int st = ST_OK;
  for (int p = 0; p < U; ++p) {
    float2 *rowp = rc + (p & 1) * 2 * UP, *colp = rowp + UP;
    const int pb = p / RB, pr = p - pb * RB;
    if (bi == pb) {  // row p
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r == pr)
#pragma unroll
          for (int c = 0; c < RB; ++c)
            if (bj * RB + c < UP) rowp[bj * RB + c] = a[r][c];
    }
    if (bj == pb) {  // column p
#pragma unroll
      for (int c = 0; c < RB; ++c)
        if (c == pr)
#pragma unroll
          for (int r = 0; r < RB; ++r)
            if (bi * RB + r < UP) colp[bi * RB + r] = a[r][c];
    }
    __syncthreads();
    const float piv = rowp[p].x;
    if (!(piv > 0.f) || !isfinite(piv)) {  // uniform over the CTA
      st = ST_NOT_PD;
      break;
    }
    const float ip = 1.f / piv;
    // every owned element takes the elimination update with row p and its
    // row's multiplier (zero past U: pads stay exact); then the owners of
    // row p and column p overwrite those entries with the pivot formulas
    float2 rowv[RB], fv[RB];
#pragma unroll
    for (int c = 0; c < RB; ++c) {
      const int j = bj * RB + c;
      rowv[c] = j < U ? rowp[j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = bi * RB + r;
      fv[r] = i < U ? cscale(colp[i], ip) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < RB; ++c) cmsub(a[r][c], fv[r], rowv[c]);
    if (bi == pb) {  // row p: T_pj = A_pj / A_pp, T_pp = 1 / A_pp
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r == pr)
#pragma unroll
          for (int c = 0; c < RB; ++c) {
            const int j = bj * RB + c;
            if (j < U) a[r][c] = (j == p) ? make_float2(ip, 0.f) : cscale(rowv[c], ip);
          }
    }
    if (bj == pb) {  // column p: T_ip = -A_ip / A_pp
#pragma unroll
      for (int c = 0; c < RB; ++c)
        if (c == pr)
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            const int i = bi * RB + r;
            if (i < U && i != p) a[r][c] = cscale(colp[i], -ip);
          }
    }
  }
  __syncthreads();  // the last pivot's readers are done with rc; A is rewritten
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int c = 0; c < RB; ++c) {
      const int i = bi * RB + r, j = bj * RB + c;
      if (i < UP && j < UP) A[i * UP + j] = a[r][c];
    }
  __syncthreads();
  return st;
}

// t = tr(Q^H Q) of Thm. 1 for T = A^{-1}: Lemma 1, tr(T) - kappa ||T||_F^2,
// unless its subtraction cancels (kappa ||T||_F^2 > kLemmaMaxRatio tr(T));
// then the definition through Eq. (14), tr(T G T) = sum_ij (T G)_ij conj(T_ij).
template <int UP>
__device__ float cta_trace_tgt(const float2 *T, const float2 *G, float kappa, int U, float *red,
                               int tid) {
  float dg = 0.f, fr = 0.f;
  for (int e = tid; e < U * UP; e += NT) {
    const int i = e / UP, j = e - i * UP;
    if (j < U) {
      const float2 t = T[i * UP + j];
      fr = fmaf(t.x, t.x, fmaf(t.y, t.y, fr));
      if (i == j) dg += t.x;
    }
  }
  const float tr = cta_sum(dg, red, tid);
  const float fro = cta_sum(fr, red, tid);
  if (kappa * fro <= kLemmaMaxRatio * tr) return tr - kappa * fro;
  float part = 0.f;
  for (int e = tid; e < U * UP; e += NT) {
    const int i = e / UP, j = e - i * UP;
    if (j < U) {
      float2 acc = make_float2(0.f, 0.f);
      for (int k = 0; k < U; ++k) cmac(acc, T[i * UP + k], G[k * UP + j]);
      const float2 t = T[i * UP + j];
      part = fmaf(acc.x, t.x, fmaf(acc.y, t.y, part));
    }
  }
  return cta_sum(part, red, tid);
}

// Zs[k][i] = sum_j T_ij s[k][j] for k < K, i < U (T Hermitian: T_ij =
// conj(T_ji), read along the row the lanes walk).
template <int UP>
__device__ void cta_whiten(const float2 *T, const float2 *Ss, float2 *Zs, int U, int K, int tid) {
  for (int e = tid; e < K * UP; e += NT) {
    const int k = e / UP, i = e - k * UP;
    float2 acc = make_float2(0.f, 0.f);
    if (i < U)
      for (int j = 0; j < U; ++j) cmac_cj(acc, T[j * UP + i], Ss[k * UP + j]);
    Zs[k * UP + i] = acc;
  }
}

// ----------------------------------------------------------------- apply ---
// acc[r][q] += sum_u conj(h_r[u]) z_q[u] for R antenna rows and NQ symbols:
// h rows in shared memory (UP complex, 16-byte aligned), z_q = zs + q * UP.
// Fully unrolled with compile-time R, NQ: every broadcast z load feeds R
// complex multiply-adds and no predicate sits in the inner loop.
template <int UP, int R, int NQ>
__device__ __forceinline__ void apply_tile(const float *const (&hrow)[R], const float2 *zs,
                                           float2 (&acc)[R][NQ]) {
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[r][q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int u = 0; u < UP; u += 2) {
    float4 g[R];
#pragma unroll
    for (int r = 0; r < R; ++r) g[r] = *reinterpret_cast<const float4 *>(hrow[r] + 2 * u);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 z = *reinterpret_cast<const float4 *>(zs + q * UP + u);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cmac_cj(acc[r][q], make_float2(g[r].x, g[r].y), make_float2(z.x, z.y));
        cmac_cj(acc[r][q], make_float2(g[r].z, g[r].w), make_float2(z.z, z.w));
      }
    }
  }
}

// X[k][b_r] = scale * sum_u conj(H[b_r][u]) z_k[u] for k in [k0, k1), rows
// r < R (row r stored only if r < nvalid), symbols in blocks of up to 7.
template <int UP, int R>
__device__ __forceinline__ void apply_rows_k(const float *const (&hrow)[R], int nvalid,
                                             const float2 *zs, int k0, int k1, float scale,
                                             float2 *const (&xcol)[R], int ldx) {
  for (int kb = k0; kb < k1; kb += 7) {
    const int nq = min(7, k1 - kb);
    const float2 *z = zs + kb * UP;
#define DP_APPLY_CASE(NQ)                                                \
  case NQ: {                                                             \
    float2 acc[R][NQ];                                                   \
    apply_tile<UP, R, NQ>(hrow, z, acc);                                 \
    _Pragma("unroll") for (int r = 0; r < R; ++r) {                      \
      if (r < nvalid) {                                                  \
        _Pragma("unroll") for (int q = 0; q < NQ; ++q)                   \
            xcol[r][(size_t)(kb + q) * ldx] = cscale(acc[r][q], scale);  \
      }                                                                  \
    }                                                                    \
    break;                                                               \
  }
    switch (nq) {
      DP_APPLY_CASE(7)
      DP_APPLY_CASE(6)
      DP_APPLY_CASE(5)
      DP_APPLY_CASE(4)
      DP_APPLY_CASE(3)
      DP_APPLY_CASE(2)
      DP_APPLY_CASE(1)
      default: break;
    }
#undef DP_APPLY_CASE
  }
}

// X[k][lo + r] = scale * sum_u conj(H[r][u]) z[k][u] for the tile rows r <
// nrows; z from shared Zs [K][UP] (pad entries zero).  Thread per row pair
// (r, r + NT), all symbols; stores are coalesced along b.
template <int UP, int KB>
__device__ void apply_rows(const float *Hs, int nrows, const float2 *Zs, int K, float scale,
                           float2 *__restrict__ Xn, int B, int lo, int tid) {
  constexpr int RS = Geo<UP>::RS;
  static_assert(KB == 7, "blocks of seven symbols");
  for (int r = tid; r < nrows; r += 2 * NT) {
    const int r1 = r + NT < nrows ? r + NT : r;
    const float *hrow[2] = {Hs + r * RS, Hs + r1 * RS};
    float2 *xcol[2] = {Xn + lo + r, Xn + lo + r1};
    apply_rows_k<UP, 2>(hrow, r + NT < nrows ? 2 : 1, Zs, 0, K, scale, xcol, B);
  }
}

template <int UP>
__device__ void zero_rows(int nrows, int K, float2 *__restrict__ Xn, int B, int lo, int tid) {
  for (int e = tid; e < nrows * K; e += NT) {
    const int k = e / nrows, r = e - k * nrows;
    Xn[(size_t)k * B + lo + r] = make_float2(0.f, 0.f);
  }
}

// Load S_n [K][U] into Ss [K][UP] (zero pads); returns (via the CTA vote)
// whether every entry is finite.
template <int UP>
__device__ bool load_symbols(const float2 *__restrict__ Sn, float2 *Ss, int U, int K, int tid) {
  bool fin = true;
  for (int e = tid; e < K * UP; e += NT) {
    const int k = e / UP, u = e - k * UP;
    float2 v = make_float2(0.f, 0.f);
    if (u < U) {
      v = __ldg(Sn + (size_t)k * U + u);
      fin = fin && cfinite(v);
    }
    Ss[e] = v;
  }
  return __syncthreads_and(fin) != 0;
}

// ------------------------------------------------ lane-segment reductions ---
// Butterflies over aligned segments of SEG lanes (SEG a power of two <= 32).
template <int SEG>
__device__ __forceinline__ float seg_sum(float v) {
#pragma unroll
  for (int o = SEG / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
template <int SEG>
__device__ __forceinline__ float seg_max(float v) {
#pragma unroll
  for (int o = SEG / 2; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// ------------------------------------------------- split-row warp solve ---
// A system of UP <= 16 padded users on a segment of SEG = 2 UP lanes: lane
// (i, h) = segment lane h UP + i holds columns [h UP/2, (h + 1) UP/2) of row
// i of A = G + kappa I.  Gauss-Jordan without pivoting (A is Hermitian
// positive definite), then t = tr(T G T) by Lemma 1 (by its definition,
// sum_ij (T G)_ij conj(T_ij), where kappa ||T||_F^2 comes close to tr(T)),
// scale = sqrt(rho2 / (Es t)) (Thm. 1) and z_k = T s_k.  Gw: G [UP][UP]
// (zero pads) for the definition; Ss: s_k at Ss[k UP + u] (zero pads);
// z_k[i] goes to zout[k ldz + i] (i < U) from lanes with h = 0 when store is
// set -- zout may be Ss itself.  zmax: max |Re|, |Im| over the system's z.
// Every lane of the warp takes part (with UP = 8 both segments run in step).
template <int UP>
__device__ __forceinline__ int split_solve(float2 (&row)[UP / 2], const float2 *Gw,
                                           const float2 *Ss, float2 *zout, int ldz, float kappa,
                                           float rho2, float Es, int U, int K, int sl,
                                           bool finite_in, bool store, float &scale,
                                           float &zmax, bool mrt = false,
                                           float *sens = nullptr) {
  constexpr int HALF = UP / 2, SEG = 2 * UP;
  static_assert(SEG <= 32, "a system fits a warp");
  const int i = sl % UP, h = sl / UP;
  int st = finite_in ? ST_OK : ST_NONFINITE;
  bool bad = false;
  // ||G||_F^2 from A = G + kappa I (for the sensitivity estimate)
  float g2 = 0.f;
  if (sens && i < U) {
#pragma unroll
    for (int jj = 0; jj < HALF; ++jj) {
      const int j = h * HALF + jj;
      const float re = row[jj].x - (j == i ? kappa : 0.f);
      if (j < U) g2 = fmaf(re, re, fmaf(row[jj].y, row[jj].y, g2));
    }
  }
  if (sens) g2 = seg_sum<SEG>(g2);
  // MRT (kappa = 0, no inverse): t = tr(G), z = s; row keeps G
#pragma unroll
  for (int p = 0; p < UP; ++p) {
    if (p >= U || mrt) break;
    const int hp = p / HALF, pc = p % HALF;
    const float piv = __shfl_sync(FULL, row[pc].x, p + hp * UP, SEG);
    bad = bad || !(piv > 0.f) || !isfinite(piv);
    const float ip = 1.f / piv;
    float2 oth;  // A_ip sits in half hp: this lane's or its partner's
    oth.x = __shfl_xor_sync(FULL, row[pc].x, UP, SEG);
    oth.y = __shfl_xor_sync(FULL, row[pc].y, UP, SEG);
    const float2 f = cscale(h == hp ? row[pc] : oth, ip);
    const int src = p + h * UP;  // row p, this lane's half
#pragma unroll
    for (int jj = 0; jj < HALF; ++jj) {
      float2 rp;
      rp.x = __shfl_sync(FULL, row[jj].x, src, SEG);
      rp.y = __shfl_sync(FULL, row[jj].y, src, SEG);
      const int j = h * HALF + jj;
      if (i == p) {
        row[jj] = (j == p) ? make_float2(ip, 0.f) : cscale(rp, ip);
      } else if (j == p) {
        row[jj] = make_float2(-f.x, -f.y);
      } else {
        cmsub(row[jj], f, rp);
      }
    }
  }
  if (st == ST_OK && bad) st = ST_NOT_PD;
  float sc = 0.f;
  {
    float dg = 0.f, fr = 0.f;
#pragma unroll
    for (int jj = 0; jj < HALF; ++jj) {
      if (h * HALF + jj == i) dg = row[jj].x;
      fr = fmaf(row[jj].x, row[jj].x, fmaf(row[jj].y, row[jj].y, fr));
    }
    if (i >= U) {
      dg = 0.f;
      fr = 0.f;
    }
    const float tr = seg_sum<SEG>(dg), fro = seg_sum<SEG>(fr);
    // sensitivity of z to a relative perturbation of G: ||G|| ||A^{-1}||,
    // estimated as ||G||_F ||T||_F / U
    if (sens) *sens = (mrt || st != ST_OK || bad) ? 0.f : sqrtf(g2 * fro) / (float)U;
    float t = mrt ? tr : tr - kappa * fro;
    const bool need = !mrt && kappa * fro > kLemmaMaxRatio * tr;
    if (__any_sync(FULL, need && st == ST_OK)) {
      // (T G)_ij from both halves of row i of T, one column j at a time
      float part = 0.f;
#pragma unroll 1
      for (int j = 0; j < U; ++j) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int kk = 0; kk < HALF; ++kk) cmac(acc, row[kk], Gw[(h * HALF + kk) * UP + j]);
        float2 oth;
        oth.x = __shfl_xor_sync(FULL, acc.x, UP, SEG);
        oth.y = __shfl_xor_sync(FULL, acc.y, UP, SEG);
        const float2 tg = cadd(acc, oth);
        if (j / HALF == h) {
          float2 tij = make_float2(0.f, 0.f);
#pragma unroll
          for (int jj = 0; jj < HALF; ++jj)
            if (h * HALF + jj == j) tij = row[jj];
          part = fmaf(tg.x, tij.x, fmaf(tg.y, tij.y, part));
        }
      }
      if (i >= U) part = 0.f;
      const float talt = seg_sum<SEG>(part);
      if (need) t = talt;
    }
    if (st == ST_OK) {
      if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
      else sc = sqrtf(rho2 / (Es * t));
    }
  }
  float zm = 0.f;
  for (int k = 0; k < K; ++k) {
    float2 acc = make_float2(0.f, 0.f);
    if (st == ST_OK && mrt) {
      if (h == 0) acc = Ss[k * UP + i];  // the partner adds zero
    } else if (st == ST_OK) {
#pragma unroll
      for (int jj = 0; jj < HALF; ++jj) cmac(acc, row[jj], Ss[k * UP + h * HALF + jj]);
    }
    float2 oth;
    oth.x = __shfl_xor_sync(FULL, acc.x, UP, SEG);
    oth.y = __shfl_xor_sync(FULL, acc.y, UP, SEG);
    const float2 z = cadd(acc, oth);
    if (i < U) zm = fmaxf(zm, fmaxf(fabsf(z.x), fabsf(z.y)));
    if (store && h == 0 && i < U) zout[(size_t)k * ldz + i] = z;
  }
  zmax = seg_max<SEG>(zm);
  scale = sc;
  return st;
}

// ----------------------------------------------------- warp-per-system solve ---
// Lane i holds row i of A = G + kappa I (UP complex registers).  In-place
// Gauss-Jordan without pivoting (A Hermitian positive definite: the pivots are
// the LDL^H pivots), row p broadcast by shuffles.  Leaves T = A^{-1}.
template <int UP>
__device__ __forceinline__ bool warp_gj_inverse(float2 (&row)[UP], int lane, int U) {
#pragma unroll
  for (int p = 0; p < UP; ++p) {
    if (p >= U) break;
    const float piv = __shfl_sync(FULL, row[p].x, p);
    if (!(piv > 0.f) || !isfinite(piv)) return false;
    const float ip = 1.f / piv;
    const float2 f = cscale(row[p], ip);
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      float2 rp;
      rp.x = __shfl_sync(FULL, row[j].x, p);
      rp.y = __shfl_sync(FULL, row[j].y, p);
      if (lane == p) {
        row[j] = (j == p) ? make_float2(ip, 0.f) : cscale(rp, ip);
      } else if (j == p) {
        row[j] = make_float2(-f.x, -f.y);
      } else {
        cmsub(row[j], f, rp);
      }
    }
  }
  return true;
}

// One system solved by one warp (steps a3-a5); up to 16 padded users in the
// split-row form above, else lane i holds row i of A = G + kappa I; Gauss-Jordan inverse in registers, t = tr(T G T), scale =
// sqrt(rho2 / (Es t)), z_k = T s_k written to zout[k * ldz + i] (i < U).
// Gs [UP][UP] and Ss [K][UP] in shared memory with zero pads.  Returns the
// status; on failure z = 0 and scale = 0.
template <int UP>
__device__ int warp_solve(const float2 *Gs, const float2 *Ss, float2 *zout, int ldz, float kappa,
                          float rho2, float Es, int U, int K, int lane, bool finite_in,
                          float &scale, bool mrt = false, float *sens = nullptr) {
  if constexpr (2 * UP <= 32) {  // split rows over 2 UP lanes
    constexpr int HALF = UP / 2, SEG = 2 * UP;
    const int sl = lane % SEG, i = sl % UP, h = sl / UP;
    float2 row[HALF];
#pragma unroll
    for (int jj = 0; jj < HALF; ++jj) {
      const int j = h * HALF + jj;
      row[jj] = (i < U) ? Gs[i * UP + j] : make_float2(0.f, 0.f);
      if (j == i) row[jj].x += kappa;
    }
    float zm;
    return split_solve<UP>(row, Gs, Ss, zout, ldz, kappa, rho2, Es, U, K, sl, finite_in,
                           lane < SEG, scale, zm, mrt, sens);
  }
  float2 row[UP];
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    row[j] = (lane < U) ? Gs[lane * UP + j] : make_float2(0.f, 0.f);
    if (j == lane) row[j].x += kappa;
  }
  int st = finite_in ? ST_OK : ST_NONFINITE;
  if (st == ST_OK && !mrt && !warp_gj_inverse<UP>(row, lane, U)) st = ST_NOT_PD;
  float sc = 0.f;
  if (st == ST_OK) {
    // Lemma 1: t = tr(T) - kappa ||T||_F^2.  When kappa ||T||_F^2 / tr(T) is
    // close to one the difference cancels (kappa dominating G); then t is
    // formed as the definition tr(T G T) = sum_ij (T G)_ij conj(T_ij).
    float dg = 0.f, fr = 0.f;
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      if (j == lane) dg = row[j].x;
      fr = fmaf(row[j].x, row[j].x, fmaf(row[j].y, row[j].y, fr));
    }
    if (lane >= U) {
      dg = 0.f;
      fr = 0.f;
    }
    const float tr = warp_sum(dg), fro = warp_sum(fr);
    float t = mrt ? tr : tr - kappa * fro;  // MRT: row holds G, t = tr(G)
    if (!mrt && kappa * fro > kLemmaMaxRatio * tr) {
      // the cancelling case: lane i forms (T G)_ij = sum_k T_ik G_kj one
      // column j at a time (runtime loop: few live registers)
      float part = 0.f;
#pragma unroll 1
      for (int j = 0; j < U; ++j) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < UP; ++k) cmac(acc, row[k], Gs[k * UP + j]);
        float2 tij = make_float2(0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < UP; ++jj)
          if (jj == j) tij = row[jj];
        part = fmaf(acc.x, tij.x, fmaf(acc.y, tij.y, part));
      }
      if (lane >= U) part = 0.f;
      t = warp_sum(part);
    }
    if (!(t > 0.f) || !isfinite(t)) st = ST_NOT_PD;
    else sc = sqrtf(rho2 / (Es * t));
  }
  for (int k = 0; k < K; ++k) {
    float2 acc = make_float2(0.f, 0.f);
    if (st == ST_OK && mrt) {
      acc = Ss[k * UP + (lane < UP ? lane : 0)];  // z = s
    } else if (st == ST_OK) {
#pragma unroll
      for (int j = 0; j < UP; ++j) cmac(acc, row[j], Ss[k * UP + j]);
    }
    if (lane < U) zout[(size_t)k * ldz + lane] = acc;
  }
  scale = sc;
  return st;
}

}  // namespace dp
