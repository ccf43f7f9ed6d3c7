// dp_tc.cu -- the reduced-precision fused precoder: Gram contraction on the
// 5th-generation tensor cores (tcgen05, BF16 or FP16 inputs, FP32
// accumulation in TMEM), solve and apply in FP32.
//
// One CTA takes a group of NG = 128 / (2 UP) systems.  The complex Gram of a
// system is one real product: with P = R R^T for R = [Re H; Im H] (2U rows,
// antennas along K), Re G = P11 + P22 and Im G = P21 - P12 (Sec. III-B,
// G = H H^H).  The group's realified rows are stacked into the M = 128 rows
// of one K-major operand that serves as both A and B (D = R R^T, N = 128);
// the block-diagonal blocks of D are the systems' P.  Antennas stream in
// chunks of 64: one bulk copy per system and chunk into an FP32 staging
// buffer, conversion to BF16/FP16 into a 128-byte-swizzled tile (two tiles
// alternate so conversion of chunk c+1 overlaps the MMAs of chunk c), four
// MMAs of K = 16 per chunk accumulating in TMEM.
// Then: TMEM -> shared P -> G, warp-per-system Gauss-Jordan solve in
// registers (Thm. 1, Lemma 1 through tr(T G T), z = A^{-1} s), and the FP32
// apply x_c = scale H_c^H z over the antenna rows fetched again (from L2).
#include "dp_blocks.cuh"
#include "dp_internal.h"
#include "dp_tc.cuh"

namespace dp {
namespace {

constexpr int KC = 64;          // antennas per chunk (one 128-byte K-block of 16-bit data)
constexpr int TILE_BYTES = 128 * 128;
constexpr int TMEM_COLS = 128;

template <int UP>
struct TcGeo {
  static constexpr int NG = (128 / (2 * UP)) > 0 ? 128 / (2 * UP) : 1;  // systems per CTA
  static constexpr int RS = Geo<UP>::RS;
  static constexpr int PS = 2 * UP + 1;                          // row stride of a P block
  static constexpr int STAGE_FLOATS = NG * KC * RS;              // padded rows (apply)
  static constexpr int P_FLOATS = NG * 2 * UP * PS;
  static_assert(P_FLOATS <= STAGE_FLOATS, "P aliases the staging buffer");
  static_assert(NG * KC * 2 * UP <= STAGE_FLOATS, "unpadded Gram staging fits");
};

struct TcSmem {
  size_t tiles, stage, G, S, Z, scale, status, info, bars, tmem, total;
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
  L.tiles = take(2 * TILE_BYTES, 1024);
  L.stage = take((size_t)T::STAGE_FLOATS * 4, 128);
  L.G = take((size_t)T::NG * UP * UP * 8, 16);
  L.S = take((size_t)T::NG * K * UP * 8 + 16, 16);
  L.Z = take((size_t)T::NG * K * UP * 8 + 16, 16);
  L.scale = take((size_t)T::NG * 4, 16);
  L.status = take((size_t)T::NG * 4, 16);
  L.info = take((size_t)T::NG * 3 * 4, 16);
  L.bars = take(3 * 8, 8);
  L.tmem = take(4, 4);
  L.total = o + 1024;  // slack to align the dynamic base to 1024 bytes
  return L;
}

template <int UP, bool BF16>
__global__ void __launch_bounds__(NT) k_fused_tc(SysDesc d, const float2 *__restrict__ H,
                                                 const float2 *__restrict__ S,
                                                 float2 *__restrict__ X,
                                                 int *__restrict__ status,
                                                 float *__restrict__ scale_out) {
  using T = TcGeo<UP>;
  constexpr int NG = T::NG, RS = T::RS, PS = T::PS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const TcSmem L = tc_smem_layout<UP>(d.K);
  unsigned char *tiles = base + L.tiles;
  float *stage = reinterpret_cast<float *>(base + L.stage);
  float *P = stage;  // alias: P is written after the last staged chunk was consumed
  float2 *Gs = reinterpret_cast<float2 *>(base + L.G);
  float2 *Ss = reinterpret_cast<float2 *>(base + L.S);
  float2 *Zs = reinterpret_cast<float2 *>(base + L.Z);
  float *sc_s = reinterpret_cast<float *>(base + L.scale);
  int *st_s = reinterpret_cast<int *>(base + L.status);
  int *lo_s = reinterpret_cast<int *>(base + L.info);  // first antenna of each system
  int *nr_s = lo_s + NG;                                // antennas of each system
  int *n_s = nr_s + NG;                                 // subcarrier of each system
  uint64_t *bar_tma = reinterpret_cast<uint64_t *>(base + L.bars);
  uint64_t *bar_mma = bar_tma + 1;  // two, one per tile
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(base + L.tmem);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int U = d.U, K = d.K;
  const int total = d.n_sc * d.nsys;
  const int sys0 = blockIdx.x * NG;
  const int nact = min(NG, total - sys0);
  const bool tma = d.tma_ok != 0;

  // rows of each system of the group
  if (tid < NG) {
    int lo = 0, hi = 0, n = 0;
    if (tid < nact) {
      const int sys = sys0 + tid;
      n = sys / d.nsys;
      sys_rows(d, sys - n * d.nsys, lo, hi);
    }
    lo_s[tid] = lo;
    nr_s[tid] = hi - lo;
    n_s[tid] = n;
  }
  __syncthreads();
  int kmax = 0;
  for (int s = 0; s < NG; ++s) kmax = max(kmax, nr_s[s]);
  const int nchunks = (kmax + KC - 1) / KC;

  // ---- set-up: barriers, TMEM, symbols -----------------------------------
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    mbar_init(bar_mma + 1, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, TMEM_COLS);
    tc::tmem_relinquish();
  }
  for (int e = tid; e < NG * K * UP; e += NT) {
    const int s = e / (K * UP), r = e - s * K * UP, k = r / UP, u = r - k * UP;
    float2 v = make_float2(0.f, 0.f);
    if (s < nact && u < U) v = __ldg(S + ((size_t)n_s[s] * K + k) * U + u);
    Ss[e] = v;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tmem_holder;

  // ---- Gram mainloop ----------------------------------------------------
  const uint32_t idesc = tc::idesc_f16(128, 128, BF16);
  const uint32_t tiles_u32 = smem_u32(tiles);
  bool timeout = false;
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    if (c > 0) {
      __syncthreads();  // everyone finished reading the staging buffer
      fence_proxy_async_smem();
    }
    // stage chunk c of every system (FP32, rows unpadded: row stride 2U floats)
    if (tma) {
      if (warp == 0) {
        uint32_t bytes = 0;
#pragma unroll
        for (int s = 0; s < NG; ++s) {
          const int m = min(KC, nr_s[s] - c * KC);
          if (m > 0) bytes += (uint32_t)m * U * 8u;
        }
        if (lane == 0) {
          if (bytes) mbar_arrive_expect_tx(bar_tma, bytes);
          else mbar_arrive(bar_tma);
        }
        __syncwarp();
        if (lane < NG) {
          const int s = lane;
          const int m = min(KC, nr_s[s] - c * KC);
          if (m > 0)
            tma_load_1d(stage + (size_t)s * KC * 2 * U,
                        H + ((size_t)n_s[s] * d.B + lo_s[s] + c * KC) * U, (uint32_t)m * U * 8u,
                        bar_tma);
        }
      }
      if (!mbar_wait(bar_tma, c & 1)) timeout = true;
    } else {
      for (int s = 0; s < NG; ++s) {
        const int m = min(KC, nr_s[s] - c * KC);
        const float2 *src = H + ((size_t)n_s[s] * d.B + lo_s[s] + c * KC) * U;
        for (int e = tid; e < m * U; e += NT)
          reinterpret_cast<float2 *>(stage + (size_t)s * KC * 2 * U)[e] = __ldg(src + e);
      }
    }
    // the MMAs of chunk c - 2 read this tile: wait for them
    if (c >= 2 && !mbar_wait(bar_mma + buf, ((c >> 1) - 1) & 1)) timeout = true;
    if (__syncthreads_or(timeout)) break;

    // convert: tile row m = s * 2UP + r (r < UP: Re H[.][r], else Im H[.][r - UP]),
    // 8 consecutive antennas per 16-byte chunk, zero outside the systems
    unsigned char *tile = tiles + buf * TILE_BYTES;
    for (int item = tid; item < 128 * 8; item += NT) {
      const int g8 = item >> 7, m = item & 127;
      const int s = m / (2 * UP), r = m - s * (2 * UP);
      const int u = r < UP ? r : r - UP, part = r < UP ? 0 : 1;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int b = c * KC + 8 * g8 + j;  // antenna within the system
        const int sc = s < NG ? s : 0;
        const bool ok = s < nact && u < U && b < nr_s[sc];
        const float *src = stage + (size_t)sc * KC * 2 * U + (size_t)(8 * g8 + j) * 2 * U;
        v[j] = ok ? src[2 * u + part] : 0.f;
      }
      uint4 q;
      q.x = tc::pack2<BF16>(v[0], v[1]);
      q.y = tc::pack2<BF16>(v[2], v[3]);
      q.z = tc::pack2<BF16>(v[4], v[5]);
      q.w = tc::pack2<BF16>(v[6], v[7]);
      *reinterpret_cast<uint4 *>(tile + tc::sw128_offset(m, g8)) = q;
    }
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
  }
  if (!timeout && nchunks > 0) {
    const int last = nchunks - 1;
    if (!mbar_wait(bar_mma + (last & 1), (last >> 1) & 1)) timeout = true;
  }
  timeout = __syncthreads_or(timeout) != 0;
  tc::fence_after_sync();

  if (timeout) {  // let anything in flight land, free TMEM, report
    mbar_wait(bar_tma, 0);
    mbar_wait(bar_mma, 0);
    mbar_wait(bar_mma + 1, 0);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc::fence_after_sync();
      tc::tmem_dealloc(taddr, TMEM_COLS);
    }
    for (int s = 0; s < nact; ++s) {
      zero_rows<UP>(nr_s[s], K, X + (size_t)n_s[s] * K * d.B, d.B, lo_s[s], tid);
      if (tid == 0) {
        status[sys0 + s] = ST_TIMEOUT;
        if (scale_out) scale_out[sys0 + s] = 0.f;
      }
    }
    return;
  }

  // ---- TMEM -> P (the diagonal 2UP x 2UP blocks) ---------------------------
  if (warp < 4) {
    const int m = 32 * warp + lane;
    const int s = m / (2 * UP), r = m - s * (2 * UP);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      float v[32];
      tc::tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + 32 * cc, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = 32 * cc + j;
        if (s < NG && n / (2 * UP) == s) P[(size_t)s * 2 * UP * PS + r * PS + (n - s * 2 * UP)] = v[j];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, TMEM_COLS);
  }

  // ---- P -> G (Hermitian, lower triangle mirrored) -------------------------
  for (int e = tid; e < NG * UP * UP; e += NT) {
    const int s = e / (UP * UP), ij = e - s * UP * UP, i = ij / UP, j = ij - i * UP;
    float2 g = make_float2(0.f, 0.f);
    if (s < nact && i < U && j < U) {
      const float *Pb = P + (size_t)s * 2 * UP * PS;
      const int a = i >= j ? i : j, b = i >= j ? j : i;  // lower-triangle source
      g.x = Pb[a * PS + b] + Pb[(UP + a) * PS + UP + b];
      g.y = (a == b) ? 0.f : Pb[(UP + a) * PS + b] - Pb[a * PS + UP + b];
      if (i < j) g.y = -g.y;
    }
    Gs[e] = g;
  }
  __syncthreads();
  // per-system finiteness of G (covers H) and of the symbols: a NaN of one
  // system must not fail the others
  if (warp < NG) {
    bool ok = true;
    for (int e = lane; e < UP * UP; e += 32) ok = ok && cfinite(Gs[warp * UP * UP + e]);
    for (int e = lane; e < K * UP; e += 32) ok = ok && cfinite(Ss[warp * K * UP + e]);
    ok = __all_sync(FULL, ok);
    if (lane == 0) st_s[warp] = ok ? ST_OK : ST_NONFINITE;
  }
  __syncthreads();

  // ---- solve: one warp per system ------------------------------------------
  if (warp < nact) {
    float sc = 0.f;
    const int st = warp_solve<UP>(Gs + warp * UP * UP, Ss + warp * K * UP, Zs + warp * K * UP, UP,
                                  d.kappa, d.rho2_sys, d.Es, U, K, lane, st_s[warp] == ST_OK,
                                  sc);
    if (lane == 0) {
      st_s[warp] = st;
      sc_s[warp] = sc;
    }
  }
  __syncthreads();

  // ---- apply: rows re-fetched (L2) into padded staging, thread per row ------
  zero_row_pads<UP>(stage, NG * KC, U, tid);
  fence_proxy_async_smem();
  __syncthreads();
  for (int c = 0; c < nchunks; ++c) {
    if (c > 0) {
      __syncthreads();
      fence_proxy_async_smem();
    }
    if (tma) {
      if (warp == 0) {
        uint32_t bytes = 0;
#pragma unroll
        for (int s = 0; s < NG; ++s) {
          const int m = min(KC, nr_s[s] - c * KC);
          if (m > 0 && st_s[s] == ST_OK) bytes += (uint32_t)m * U * 8u;
        }
        if (lane == 0) {
          if (bytes) mbar_arrive_expect_tx(bar_tma, bytes);
          else mbar_arrive(bar_tma);
        }
        __syncwarp();
        for (int s = 0; s < NG; ++s) {
          const int m = min(KC, nr_s[s] - c * KC);
          if (m <= 0 || st_s[s] != ST_OK) continue;
          const float2 *src = H + ((size_t)n_s[s] * d.B + lo_s[s] + c * KC) * U;
          for (int r = lane; r < m; r += 32)
            tma_load_1d(stage + ((size_t)s * KC + r) * RS, src + (size_t)r * U, (uint32_t)U * 8u,
                        bar_tma);
        }
      }
      if (!mbar_wait(bar_tma, (nchunks + c) & 1)) timeout = true;
    } else {
      for (int s = 0; s < NG; ++s) {
        const int m = min(KC, nr_s[s] - c * KC);
        if (m <= 0 || st_s[s] != ST_OK) continue;
        const float2 *src = H + ((size_t)n_s[s] * d.B + lo_s[s] + c * KC) * U;
        for (int e = tid; e < m * U; e += NT) {
          const int r = e / U, u = e - r * U;
          *reinterpret_cast<float2 *>(stage + ((size_t)s * KC + r) * RS + 2 * u) = __ldg(src + e);
        }
      }
    }
    if (__syncthreads_or(timeout)) {
      mbar_wait(bar_tma, (nchunks + c) & 1);
      break;
    }
    for (int e = tid; e < NG * KC; e += NT) {
      const int s = e / KC, r = e - s * KC;
      const int b = c * KC + r;
      if (s >= nact || b >= nr_s[s]) continue;
      float2 *Xn = X + (size_t)n_s[s] * K * d.B;
      if (st_s[s] != ST_OK) {
        for (int k = 0; k < K; ++k) Xn[(size_t)k * d.B + lo_s[s] + b] = make_float2(0.f, 0.f);
        continue;
      }
      const float *hrow = stage + ((size_t)s * KC + r) * RS;
      const float2 *zs = Zs + s * K * UP;
      const float scl = sc_s[s];
      for (int kb = 0; kb < K; kb += 7) {
        float2 acc[7];
#pragma unroll
        for (int kk = 0; kk < 7; ++kk) acc[kk] = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < UP; u += 2) {
          const float4 h = *reinterpret_cast<const float4 *>(hrow + 2 * u);
          const float2 h0 = make_float2(h.x, h.y), h1 = make_float2(h.z, h.w);
#pragma unroll
          for (int kk = 0; kk < 7; ++kk) {
            if (kb + kk < K) {
              const float4 z = *reinterpret_cast<const float4 *>(zs + (kb + kk) * UP + u);
              cmac_cj(acc[kk], h0, make_float2(z.x, z.y));
              cmac_cj(acc[kk], h1, make_float2(z.z, z.w));
            }
          }
        }
#pragma unroll
        for (int kk = 0; kk < 7; ++kk)
          if (kb + kk < K) Xn[(size_t)(kb + kk) * d.B + lo_s[s] + b] = cscale(acc[kk], scl);
      }
    }
  }
  if (timeout) {
    for (int s = 0; s < nact; ++s) {
      zero_rows<UP>(nr_s[s], K, X + (size_t)n_s[s] * K * d.B, d.B, lo_s[s], tid);
      if (tid == 0) st_s[s] = ST_TIMEOUT;
    }
  }
  __syncthreads();
  if (tid < nact) {
    status[sys0 + tid] = st_s[tid];
    if (scale_out) scale_out[sys0 + tid] = st_s[tid] == ST_OK ? sc_s[tid] : 0.f;
  }
}

template <int UP, bool BF16>
cudaError_t launch_tc_t(const SysDesc &d, const float2 *H, const float2 *S, float2 *X,
                        int *status, float *scale_out, cudaStream_t s) {
  const TcSmem L = tc_smem_layout<UP>(d.K);
  cudaError_t e = cudaFuncSetAttribute(k_fused_tc<UP, BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  const int total = d.n_sc * d.nsys;
  const int grid = (total + TcGeo<UP>::NG - 1) / TcGeo<UP>::NG;
  k_fused_tc<UP, BF16><<<grid, NT, L.total, s>>>(d, H, S, X, status, scale_out);
  return cudaGetLastError();
}

template <int UP>
cudaError_t launch_tc_u(const SysDesc &d, bool bf16, const float2 *H, const float2 *S, float2 *X,
                        int *status, float *scale_out, cudaStream_t s) {
  return bf16 ? launch_tc_t<UP, true>(d, H, S, X, status, scale_out, s)
              : launch_tc_t<UP, false>(d, H, S, X, status, scale_out, s);
}

}  // namespace

bool tc_supported(int UP) { return UP <= 32; }

cudaError_t launch_fused_tc(const SysDesc &d, int UP, bool bf16, const float2 *H, const float2 *S,
                            float2 *X, int *status, float *scale_out, cudaStream_t s) {
  switch (UP) {
    case 8: return launch_tc_u<8>(d, bf16, H, S, X, status, scale_out, s);
    case 16: return launch_tc_u<16>(d, bf16, H, S, X, status, scale_out, s);
    case 24: return launch_tc_u<24>(d, bf16, H, S, X, status, scale_out, s);
    case 32: return launch_tc_u<32>(d, bf16, H, S, X, status, scale_out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dp
