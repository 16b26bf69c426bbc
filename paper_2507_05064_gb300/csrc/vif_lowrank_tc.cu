// A = K_nm L_m^{-T} (Sec. 2.2, the low-rank factor of the predictive-process part) on the
// fifth-generation tensor cores, for the float32 (mixed) path.
//
// Row p of A is sum_k K(s_p, z_k) Linv[j][k] over k <= j, i.e. a GEMM of the kernel
// block K_nm (M = points, K = inducing points) with L_m^{-1} read as an N x K K-major
// operand (row j of L_m^{-1} is contiguous in k).  Float32 accuracy is kept with the
// three-term split x = hi + lo (hi, lo tf32, round to nearest): each product is
//   Khi Lhi + Khi Llo + Klo Lhi,
// which leaves an error of about 2^-21 relative per product.  The tensor core's float32
// accumulation rounds toward zero at every step (a coherent bias), so a TMEM
// accumulator never runs longer than one chunk of 32 inducing points (12 MMAs): each
// chunk's partial is added into float32 registers (round to nearest), and two TMEM
// accumulators alternate so that the MMAs of chunk c run while the partial of chunk
// c-1 is read out.
//
// CTA: 128 points (one TMEM lane each) x 256 output columns; 16 compute warps and one MMA
// warp.  Per chunk every compute thread evaluates 8 kernel values of one point, splits
// them and writes them into the swizzled A-operand tiles of the chunk's stage, then reads
// out the previous chunk's accumulator; thread 0 also brings the L_m^{-1} tiles (packed once
// per call, already in the swizzled image) of the next chunk with one bulk copy per tile.
// The MMA warp issues a chunk's 12 MMAs as soon as its tiles are staged and its
// accumulator read out, so the kernel evaluation and read-out of neighbouring chunks run
// while the tensor core works (hand-offs through mbarriers, no CTA-wide barrier per chunk).
// Chunks above the tile's last column are skipped (L_m^{-1} is lower triangular).
#include "vif_internal.cuh"
#include "vif_tc.cuh"

namespace vif {

namespace {

constexpr int AT_M = 128;                         // points per CTA
constexpr int AT_N = 256;                         // output columns per CTA
constexpr int AT_K = 32;                          // inducing points per chunk
constexpr int AT_MAXD = 16;
constexpr int AT_CT = 512;                        // compute threads
constexpr int AT_THREADS = AT_CT + 32;            // + the MMA warp
constexpr uint32_t AT_ATILE = AT_M * 128;         // bytes of one A-operand tile (hi or lo)
constexpr uint32_t AT_BTILE = AT_N * 128;         // bytes of one B-operand tile (hi or lo)
constexpr uint32_t AT_STAGE = 2 * AT_ATILE + 2 * AT_BTILE;
constexpr uint32_t AT_SMEM = 2 * AT_STAGE + 1024; // two stages + alignment slack
constexpr uint32_t AT_TMEM_COLS = 2 * AT_N;       // two accumulators

struct __align__(16) AtBars {
  uint64_t full[2];    // B tiles of the stage have landed
  uint64_t staged[2];  // A tiles of the stage written (one arrival per compute thread)
  uint64_t drained[2]; // accumulator s read out (one arrival per compute thread)
  uint64_t done[2];    // MMAs of the stage's chunk are done: stage free, accumulator s ready
  uint64_t fin;        // every MMA of the CTA is done
  uint32_t tmem;
  int abort;           // the MMA warp gave up waiting
  alignas(16) float zs[2][AT_K * AT_MAXD];   // 8-byte pairs are read from it
};

// Packed L_m^{-1}: tile (h, c, part) holds rows j = 256 h + r (r < 256) and columns
// k = 32 c + kk of L_m^{-1} (hi part = 0, lo part = 1) as a swizzled 256 x 32 tf32 image.
__global__ void linv_pack_tc_kernel(const double* __restrict__ Linv, int m, int ldl, float* __restrict__ pk,
                                    int nchunk, int64_t total) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int kk = (int)(e % AT_K);
  const int r = (int)((e / AT_K) % AT_N);
  const int64_t t = e / ((int64_t)AT_K * AT_N);     // (h * nchunk + c)
  const int c = (int)(t % nchunk), h = (int)(t / nchunk);
  const int j = h * AT_N + r, k = c * AT_K + kk;
  double v = 0.0;
  if (j < m && k < m && k <= j) v = Linv[(size_t)j * ldl + k];
  const float hi = tc::to_tf32((float)v);
  const float lo = tc::to_tf32((float)(v - (double)hi));
  float* tile = pk + (size_t)t * 2 * (AT_N * AT_K);
  const uint32_t off = tc::sw128_off32(r, kk) / 4;
  tile[off] = hi;
  tile[AT_N * AT_K + off] = lo;
}

// D > 0: compile-time input dimension; D = 0: any d <= AT_MAXD
template <int D>
__global__ __launch_bounds__(AT_THREADS, 1) void lowrank_A_tc_kernel(
    const float* __restrict__ Xs, const float* __restrict__ Zs, const float* __restrict__ pk, float* __restrict__ A,
    int64_t n, int d, int m, int mpad, int nchunk_all, int kind, float var, int* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ AtBars sb;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int h = blockIdx.y;
  const int64_t row0 = (int64_t)blockIdx.x * AT_M;
  const int ncols = min(AT_N, mpad - h * AT_N);                 // multiple of 32
  const int nchunk = min(nchunk_all, (h * AT_N + ncols - 1) / AT_K + 1);
  const uint32_t idesc = tc::idesc_tf32(AT_M, ncols);
  const float* pk_h = pk + (size_t)h * nchunk_all * 2 * (AT_N * AT_K);
  // kernel evaluation: point krow, values 8 kq .. 8 kq + 7 of each chunk (compute threads)
  const int krow = tid & (AT_M - 1), kq = (tid >> 7) & 3;
  const int64_t p = row0 + krow;
  // read-out: TMEM lanes dl .. dl + 31, columns dc .. dc + 63 of the accumulator
  const int dl = 32 * (warp & 3), dc = 64 * (warp >> 2);
  const int ngrp = max(0, min(2, (ncols - dc) / 32));

  if (warp == 0) tc::tmem_alloc(&sb.tmem, AT_TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&sb.full[s], 1);
      tc::mbar_init(&sb.staged[s], AT_CT);
      tc::mbar_init(&sb.drained[s], AT_CT);
      tc::mbar_init(&sb.done[s], 1);
    }
    tc::mbar_init(&sb.fin, 1);
    sb.abort = 0;
    tc::fence_mbar_init();
  }
  constexpr int DX = D > 0 ? D : AT_MAXD;
  float x[DX];
#pragma unroll
  for (int t = 0; t < DX; ++t) x[t] = (t < d && p < n) ? Xs[(size_t)p * d + t] : 0.f;
  constexpr int DP = (D > 0 && D % 2 == 0) ? D / 2 : 1;   // coordinate pairs (even D)
  unsigned long long xp[DP];
#pragma unroll
  for (int j = 0; j < DP; ++j) xp[j] = pack_f2(x[(2 * j) % DX], x[(2 * j + 1) % DX]);
  // inducing points of chunk c, element e = tid + 512 j of the chunk's 32 x d block
  auto zload = [&](int c, float (&zr)[1]) {
#pragma unroll
    for (int j = 0; j < 1; ++j) {
      const int e = tid + AT_CT * j;
      const int k = c * AT_K + e / max(d, 1);
      zr[j] = (c < nchunk && e < AT_K * d && k < m) ? Zs[(size_t)c * AT_K * d + e] : 0.f;
    }
  };
  float zpre[1];
  zload(0, zpre);
  unsigned long long acc2[32];   // column pairs (2j, 2j+1) of this thread's read-out range
#pragma unroll
  for (int j = 0; j < 32; ++j) acc2[j] = 0ull;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sb.tmem;

  bool failed = false;
  // add the partial of chunk j (accumulator j % 2) into acc
  auto drain = [&](int j) {
    // warp-uniform outcome: the TMEM loads below are warp-collective
    if (!__all_sync(0xffffffffu, tc::mbar_wait(&sb.done[j & 1], (j >> 1) & 1))) {
      failed = true;
      return;
    }
    tc::fence_after_sync();
    const uint32_t base = tmem + ((uint32_t)dl << 16) + (uint32_t)((j & 1) * AT_N + dc);
    // 16-column pieces (few live registers); the accumulator is released once all are read
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g < 2 * ngrp) {
        float v[16];
        tc::tmem_ld16(base + g * 16, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc2[g * 8 + i] = fadd2(acc2[g * 8 + i], pack_f2(v[2 * i], v[2 * i + 1]));
      }
    }
    tc::fence_before_sync();
    tc::mbar_arrive(&sb.drained[j & 1]);
  };
  // L_m^{-1} tiles of chunk c into stage c % 2 (thread 0)
  int copies_issued[2] = {0, 0};
  auto fetch_b = [&](int c) {
    const int s = c & 1;
    unsigned char* st = smem + s * AT_STAGE;
    const float* src = pk_h + (size_t)c * 2 * (AT_N * AT_K);
    tc::mbar_arrive_expect_tx(&sb.full[s], 2u * ncols * 128u);
    tc::bulk_g2s(st + 2 * AT_ATILE, src, ncols * 128u, &sb.full[s]);
    tc::bulk_g2s(st + 2 * AT_ATILE + AT_BTILE, src + AT_N * AT_K, ncols * 128u, &sb.full[s]);
    ++copies_issued[s];
  };
  if (tid == 0 && nchunk > 0) fetch_b(0);

  if (warp == AT_CT / 32) {
    // ------------------------------------------------------------ MMA warp (one lane)
    if (lane == 0) {
      for (int c = 0; c < nchunk; ++c) {
        const int s = c & 1;
        const uint32_t ph = (uint32_t)(c >> 1) & 1u;
        if (!tc::mbar_wait(&sb.staged[s], ph) || !tc::mbar_wait(&sb.full[s], ph) ||
            (c >= 2 && !tc::mbar_wait(&sb.drained[s], ph ^ 1u))) {
          failed = true;
          sb.abort = 1;
          break;
        }
        tc::fence_after_sync();
        unsigned char* st = smem + s * AT_STAGE;
        const uint32_t dt = tmem + (uint32_t)(s * AT_N);
        const uint32_t ah = tc::smem_addr(st), al = ah + AT_ATILE;
        const uint32_t bh = ah + 2 * AT_ATILE, bl = bh + AT_BTILE;
        // the small cross terms first, the hi x hi products last: every accumulation
        // step truncates relative to the running sum, so the steps taken once the sum
        // is large are kept to the four hi x hi ones
#pragma unroll
        for (int ks = 0; ks < AT_K / 8; ++ks) {
          const uint32_t o = ks * 32;
          tc::mma_tf32(dt, tc::desc_k_sw128(al + o), tc::desc_k_sw128(bh + o), idesc, ks > 0);
          tc::mma_tf32(dt, tc::desc_k_sw128(ah + o), tc::desc_k_sw128(bl + o), idesc, 1u);
        }
#pragma unroll
        for (int ks = 0; ks < AT_K / 8; ++ks) {
          const uint32_t o = ks * 32;
          tc::mma_tf32(dt, tc::desc_k_sw128(ah + o), tc::desc_k_sw128(bh + o), idesc, 1u);
        }
        tc::mma_commit(&sb.done[s]);
      }
      // every MMA issued by this CTA completes on `fin`
      tc::mma_commit(&sb.fin);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ compute warps
    for (int c = 0; c < nchunk; ++c) {
      const int s = c & 1;
      unsigned char* st = smem + s * AT_STAGE;
      unsigned char* a_hi = st;
      unsigned char* a_lo = st + AT_ATILE;
      // zs[s] was last read at iteration c-2; everyone passed the barrier of iteration c-1
#pragma unroll
      for (int j = 0; j < 1; ++j) {
        const int e = tid + AT_CT * j;
        if (e < AT_K * AT_MAXD) sb.zs[s][e] = zpre[j];
      }
      zload(c + 1, zpre);
      if (tc::bar_sync_or(1, AT_CT, failed || sb.abort)) {
        failed = true;
        break;
      }
      // stage s was last read by the MMAs of chunk c-2, which this thread saw finish when it
      // read out chunk c-2 at iteration c-1
      const int kmax = min(AT_K, m - c * AT_K);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float hv[4], lv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int kk = kq * 8 + q * 4 + u;
          float kv = 0.f;
          if (kk < kmax && p < n) {
            float r2 = 0.f;
            if constexpr (D > 0 && D % 2 == 0) {
              const float2* z2 = reinterpret_cast<const float2*>(&sb.zs[s][kk * D]);
              unsigned long long a2 = 0ull;
#pragma unroll
              for (int j = 0; j < DP; ++j) {
                const float2 zz = z2[j];
                const unsigned long long df = fsub2(xp[j], pack_f2(zz.x, zz.y));
                a2 = ffma2(df, df, a2);
              }
              const float2 h2 = unpack_f2(a2);
              r2 = h2.x + h2.y;
            } else if constexpr (D > 0) {
              const float* z = &sb.zs[s][kk * D];
#pragma unroll
              for (int t = 0; t < D; ++t) {
                const float df = x[t] - z[t];
                r2 = fmaf(df, df, r2);
              }
            } else {
              const float* z = &sb.zs[s][kk * d];
#pragma unroll
              for (int t = 0; t < AT_MAXD; ++t)
                if (t < d) {
                  const float df = x[t] - z[t];
                  r2 = fmaf(df, df, r2);
                }
            }
            kv = cov_r2_fast(r2, kind, var);
          }
          hv[u] = tc::to_tf32(kv);
          lv[u] = tc::to_tf32(kv - hv[u]);
        }
        const uint32_t off = tc::sw128_off32(krow, kq * 8 + q * 4);
        *reinterpret_cast<float4*>(a_hi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<float4*>(a_lo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(&sb.staged[s]);
      // read out chunk c-1 while chunk c multiplies; its MMAs were the last readers of
      // stage (c+1) % 2, which then takes the L_m^{-1} tiles of chunk c+1
      if (c >= 1 && !failed) drain(c - 1);
      if (tid == 0 && !failed && c + 1 < nchunk) fetch_b(c + 1);
    }
    if (!failed && nchunk > 0) drain(nchunk - 1);
    if (tid == 0) {
      // copies issued but possibly not landed (after a failure): wait for the last one of
      // each stage (bounded) so that none lands after the CTA has left
      for (int s = 0; s < 2; ++s)
        if (copies_issued[s] > 0) tc::mbar_wait(&sb.full[s], (uint32_t)(copies_issued[s] - 1) & 1u);
    }
  }
  // a wait that gave up may leave MMAs in flight: wait for them once more (bounded) before
  // the accumulators' TMEM is released; if they still have not finished, the TMEM is
  // kept rather than freed under running MMAs (the call reports the timeout and its
  // results are discarded)
  bool fin_ok = tc::mbar_wait(&sb.fin, 0);
  if (!fin_ok) {
    failed = true;
    fin_ok = tc::mbar_wait(&sb.fin, 0);
  }
  if (__syncthreads_or(failed)) {
    if (tid == 0 && status) flag_status(status, ST_TIMEOUT, blockIdx.x);
  } else if (warp < AT_CT / 32) {
    const int64_t row = row0 + dl + lane;
    if (row < n) {
      float* dst = A + (size_t)row * mpad + h * AT_N + dc;
#pragma unroll
      for (int g = 0; g < 2; ++g)
        if (g < ngrp) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const float2 a = unpack_f2(acc2[g * 16 + j]), b = unpack_f2(acc2[g * 16 + j + 1]);
            *reinterpret_cast<float4*>(dst + g * 32 + 2 * j) = make_float4(a.x, a.y, b.x, b.y);
          }
        }
    }
  }
  tc::fence_before_sync();
  const bool drained = __syncthreads_and(fin_ok);
  if (warp == 0 && drained) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, AT_TMEM_COLS);
  }
}

}  // namespace

cudaError_t lowrank_A_tc_init() {
  cudaError_t e = cudaFuncSetAttribute(lowrank_A_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)AT_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lowrank_A_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AT_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lowrank_A_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AT_SMEM);
  return e;
}

size_t lowrank_A_tc_pack_floats(int mpad) {
  const int nh = (mpad + AT_N - 1) / AT_N, nchunk = mpad / AT_K;
  return (size_t)nh * nchunk * 2 * AT_N * AT_K;
}

cudaError_t lowrank_A_tc(const float* Xs, const float* Zs, const double* Linv, int ldl, float* pack, float* A,
                         int64_t n, int d, int m, int mpad, int kind, double var, int* status, cudaStream_t s) {
  if (m <= 0) return cudaMemsetAsync(A, 0, sizeof(float) * (size_t)n * mpad, s);
  if (d > AT_MAXD || mpad % AT_K != 0 || mpad < m || mpad - m >= AT_K || n <= 0) return cudaErrorInvalidValue;
  // mpad = 32 ceil(m / 32), so the packed chunks and the chunks of m coincide
  const int nh = (mpad + AT_N - 1) / AT_N, nchunk = mpad / AT_K;
  const int64_t total = (int64_t)nh * nchunk * AT_N * AT_K;
  linv_pack_tc_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Linv, m, ldl, pack, nchunk, total);
  dim3 grid((unsigned)((n + AT_M - 1) / AT_M), (unsigned)nh);
  if (d == 8)
    lowrank_A_tc_kernel<8><<<grid, AT_THREADS, AT_SMEM, s>>>(Xs, Zs, pack, A, n, d, m, mpad, nchunk, kind,
                                                             (float)var, status);
  else if (d == 2)
    lowrank_A_tc_kernel<2><<<grid, AT_THREADS, AT_SMEM, s>>>(Xs, Zs, pack, A, n, d, m, mpad, nchunk, kind,
                                                             (float)var, status);
  else
    lowrank_A_tc_kernel<0><<<grid, AT_THREADS, AT_SMEM, s>>>(Xs, Zs, pack, A, n, d, m, mpad, nchunk, kind,
                                                             (float)var, status);
  return cudaGetLastError();
}

}  // namespace vif
