// A = K_nm L_m^{-T} (Sec. 2.2, the low-rank factor of the predictive-process part) on the
// fifth-generation tensor cores, for the float32 (mixed) path.
//
// Row p of A is sum_k K(s_p, z_k) Linv[j][k] over k <= j, i.e. a GEMM of the kernel
// block K_nm (M = points, K = inducing points) with L_m^{-1} read as an N x K K-major
// operand (row j of L_m^{-1} is contiguous in k).  Float32 accuracy is kept with the
// three-term split x = hi + lo (hi, lo float16, round to nearest): each product is
//   Khi Lhi + Khi Llo + Klo Lhi,
// which leaves an error of about 2^-21 relative per product.  Float16 has 11 significant
// bits like tf32 but a narrow exponent range, so both operands are brought to the top of
// it by powers of two: the kernel values are evaluated with variance 2^14 (correlations
// times 2^14), and row j of L_m^{-1} is scaled by 2^e_j so that its largest entry lies in
// [2^13, 2^14).  The read-out multiplies column j by var 2^-14 2^-e_j.  Entries below
// 2^-24 of their scale flush to zero, an absolute error far under float32 rounding.
// The tensor core's float32 accumulation rounds toward zero at every step (a coherent
// bias), so a TMEM accumulator never runs longer than one chunk of 64 inducing points
// (four hi x hi steps, eight cross-term steps): each chunk's partial is added into float32
// registers (round to nearest), and two TMEM accumulators alternate so that the MMAs of
// chunk c run while the partial of chunk c-1 is read out.
//
// CTA: 128 points (one TMEM lane each) x 256 output columns; 16 compute warps and one MMA
// warp.  Per chunk every compute thread evaluates 16 kernel values of one point, splits
// them and writes them into the swizzled A-operand tiles of the chunk's stage, then reads
// out the previous chunk's accumulator; thread 0 also brings the L_m^{-1} tiles (packed once
// per call, already in the swizzled image) of the next chunk with one bulk copy per tile.
// The MMA warp issues a chunk's 12 MMAs as soon as its tiles are staged and its
// accumulator read out, so the kernel evaluation and read-out of neighbouring chunks run
// while the tensor core works (hand-offs through mbarriers, no CTA-wide barrier per chunk).
// Chunks above the tile's last column are skipped (L_m^{-1} is lower triangular).
#include <cuda_fp16.h>

#include "vif_internal.cuh"
#include "vif_tc.cuh"

namespace vif {

namespace {

constexpr int AT_M = 128;                         // points per CTA
constexpr int AT_N = 256;                         // output columns per CTA
constexpr int AT_K = 64;                          // inducing points per chunk (128 bytes of f16)
constexpr int AT_MAXD = 16;
constexpr int AT_CT = 512;                        // compute threads
constexpr int AT_THREADS = AT_CT + 32;            // + the MMA warp
constexpr int AT_ZPT = AT_K * AT_MAXD / AT_CT;    // inducing-point coordinates per thread and chunk
constexpr uint32_t AT_ATILE = AT_M * 128;         // bytes of one A-operand tile (hi or lo)
constexpr uint32_t AT_BTILE = AT_N * 128;         // bytes of one B-operand tile (hi or lo)
constexpr uint32_t AT_STAGE = 2 * AT_ATILE + 2 * AT_BTILE;
constexpr uint32_t AT_SMEM = 2 * AT_STAGE + 1024; // two stages + alignment slack
constexpr uint32_t AT_TMEM_COLS = 2 * AT_N;       // two accumulators
constexpr float AT_KSCALE = 16384.f;              // kernel values are evaluated with this variance

struct __align__(16) AtBars {
  uint64_t full[2];    // B tiles of the stage have landed
  uint64_t staged[2];  // A tiles of the stage written (one arrival per compute thread)
  uint64_t drained[2]; // accumulator s read out (one arrival per compute thread)
  uint64_t done[2];    // MMAs of the stage's chunk are done: stage free, accumulator s ready
  uint64_t fin;        // every MMA of the CTA is done
  uint32_t tmem;
  int abort;           // the MMA warp gave up waiting
  alignas(16) float zs[2][AT_K * AT_MAXD];   // 16- and 8-byte groups are read from it
};

// byte offset of element (r, k) of a K-major 128-byte-swizzled tile of 16-bit values
__host__ __device__ constexpr uint32_t sw128_off16(uint32_t r, uint32_t k) {
  return r * 128u + ((((k >> 3) ^ (r & 7u)) & 7u) << 4) + (k & 7u) * 2u;
}

__device__ __forceinline__ uint32_t h2_rn(float a, float b) {   // a in the low half
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
// float16 (hi, lo) pairs of two values: a = hi + lo + O(2^-22 a)
__device__ __forceinline__ void split_h2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = h2_rn(a, b);
  const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  lo = h2_rn(a - hf.x, b - hf.y);
}

// Scales of the rows of L_m^{-1} (one warp per row j < 256 nh): s_j = 2^e_j with the
// row's largest |entry| s_j in [2^13, 2^14) (s_j = 1 for padding rows), and the read-out
// factor colf[j] = var 2^-14 / s_j of column j of A.
__global__ void linv_rowscale_kernel(const double* __restrict__ Linv, int m, int ldl, int rows, double var,
                                     float* __restrict__ rs, float* __restrict__ colf) {
  const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= rows) return;
  double mx = 0.0;
  if (j < m)
    for (int k = lane; k <= j; k += 32) mx = fmax(mx, fabs(Linv[(size_t)j * ldl + k]));
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    int e = 0;
    if (mx > 0.0 && mx <= 1e300) {
      int ex;
      frexp(mx, &ex);                       // mx in [2^(ex-1), 2^ex)
      e = min(100, max(-100, 14 - ex));
    }
    rs[j] = ldexpf(1.f, e);
    colf[j] = (float)(var * ldexp(1.0, -14 - e));
  }
}

// Packed L_m^{-1}: tile (h, c, part) holds rows j = 256 h + r (r < 256) and columns
// k = 64 c + kk of diag(s) L_m^{-1} (hi part = 0, lo part = 1) as a swizzled 256 x 64
// float16 image; one thread per 8 consecutive columns (16 bytes of each part).
__global__ void linv_pack_tc_kernel(const double* __restrict__ Linv, int m, int ldl, const float* __restrict__ rs,
                                    unsigned char* __restrict__ pk, int nchunk, int64_t total) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int g = (int)(e % (AT_K / 8));
  const int r = (int)((e / (AT_K / 8)) % AT_N);
  const int64_t t = e / ((int64_t)(AT_K / 8) * AT_N);     // (h * nchunk + c)
  const int c = (int)(t % nchunk), h = (int)(t / nchunk);
  const int j = h * AT_N + r, k0 = c * AT_K + 8 * g;
  const double sj = j < m ? (double)rs[j] : 0.0;
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float v[2];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int k = k0 + 2 * u + w;
      v[w] = (j < m && k < m && k <= j) ? (float)(sj * Linv[(size_t)j * ldl + k]) : 0.f;
    }
    // the float32 value of s_j Linv carries 24 bits; hi + lo keeps 22 of them
    split_h2(v[0], v[1], hi[u], lo[u]);
  }
  unsigned char* tile = pk + (size_t)t * 2 * AT_BTILE;
  const uint32_t off = sw128_off16(r, 8 * g);
  *reinterpret_cast<uint4*>(tile + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(tile + AT_BTILE + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// D > 0: compile-time input dimension; D = 0: any d <= AT_MAXD.  KIND: the covariance
// function (a compile-time constant, so that the evaluation loop holds one branch-free form)
template <int D, int KIND>
__global__ __launch_bounds__(AT_THREADS, 1) void lowrank_A_tc_kernel(
    const float* __restrict__ Xs, const float* __restrict__ Zs, const unsigned char* __restrict__ pk,
    const float* __restrict__ colf, float* __restrict__ A, int64_t n, int d, int m, int mpad, int nchunk_all,
    int* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ AtBars sb;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int h = blockIdx.y;
  const int64_t row0 = (int64_t)blockIdx.x * AT_M;
  const int ncols = min(AT_N, mpad - h * AT_N);                 // multiple of 32
  const int nchunk = min(nchunk_all, (h * AT_N + ncols - 1) / AT_K + 1);
  const uint32_t idesc = tc::idesc_f16(AT_M, ncols);
  const unsigned char* pk_h = pk + (size_t)h * nchunk_all * 2 * AT_BTILE;
  // kernel evaluation: point krow, values 16 kq .. 16 kq + 15 of each chunk (compute threads)
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
  // inducing points of chunk c, element e = tid + 512 j of the chunk's 64 x d block
  constexpr int ZPT = D > 0 ? (AT_K * D + AT_CT - 1) / AT_CT : AT_ZPT;
  auto zload = [&](int c, float (&zr)[ZPT]) {
#pragma unroll
    for (int j = 0; j < ZPT; ++j) {
      const int e = tid + AT_CT * j;
      const int k = c * AT_K + e / max(d, 1);
      zr[j] = (c < nchunk && e < AT_K * d && k < m) ? Zs[(size_t)c * AT_K * d + e] : 0.f;
    }
  };
  float zpre[ZPT];
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
    const unsigned char* src = pk_h + (size_t)c * 2 * AT_BTILE;
    tc::mbar_arrive_expect_tx(&sb.full[s], 2u * ncols * 128u);
    tc::bulk_g2s(st + 2 * AT_ATILE, src, ncols * 128u, &sb.full[s]);
    tc::bulk_g2s(st + 2 * AT_ATILE + AT_BTILE, src + AT_BTILE, ncols * 128u, &sb.full[s]);
    ++copies_issued[s];
  };
  if (tid == 0 && nchunk > 0) fetch_b(0);

  if (warp == AT_CT / 32) {
    // ------------------------------------------------------------ MMA warp
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
        for (int ks = 0; ks < AT_K / 16; ++ks) {
          const uint32_t o = ks * 32;
          tc::mma_f16(dt, tc::desc_k_sw128(al + o), tc::desc_k_sw128(bh + o), idesc, ks > 0);
          tc::mma_f16(dt, tc::desc_k_sw128(ah + o), tc::desc_k_sw128(bl + o), idesc, 1u);
        }
#pragma unroll
        for (int ks = 0; ks < AT_K / 16; ++ks) {
          const uint32_t o = ks * 32;
          tc::mma_f16(dt, tc::desc_k_sw128(ah + o), tc::desc_k_sw128(bh + o), idesc, 1u);
        }
        tc::mma_commit(&sb.done[s]);
      }
      // every MMA issued by this CTA completes on `fin`
      tc::mma_commit(&sb.fin);
    }
    __syncwarp();
    // the closing barriers of the compute warps (ids 2 and 3 span the whole CTA)
    bool fin_ok = tc::mbar_wait(&sb.fin, 0);
    if (!fin_ok) {
      failed = true;
      fin_ok = tc::mbar_wait(&sb.fin, 0);
    }
    tc::bar_sync_or(2, AT_THREADS, failed);
    tc::fence_before_sync();
    tc::bar_sync_or(3, AT_THREADS, !fin_ok);
    return;
  }
  // ------------------------------------------------------------ compute warps
  {
    for (int c = 0; c < nchunk; ++c) {
      const int s = c & 1;
      unsigned char* st = smem + s * AT_STAGE;
      unsigned char* a_hi = st;
      unsigned char* a_lo = st + AT_ATILE;
      // zs[s] was last read at iteration c-2; everyone passed the barrier of iteration c-1
#pragma unroll
      for (int j = 0; j < ZPT; ++j) {
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
      const bool pvalid = p < n;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        float kv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int kk = kq * 16 + q * 4 + u;
          // evaluated for every slot (inducing points past m read zeros, points past n have
          // x = 0) and masked afterwards: no branch in the loop
          {
            float r2 = 0.f;
            if constexpr (D > 0 && D % 4 == 0) {
              const float4* z4 = reinterpret_cast<const float4*>(&sb.zs[s][kk * D]);
              unsigned long long a2 = 0ull;
#pragma unroll
              for (int j = 0; j < D / 4; ++j) {
                const float4 zz = z4[j];
                const unsigned long long d0 = fsub2(xp[2 * j], pack_f2(zz.x, zz.y));
                const unsigned long long d1 = fsub2(xp[2 * j + 1], pack_f2(zz.z, zz.w));
                a2 = ffma2(d0, d0, a2);
                a2 = ffma2(d1, d1, a2);
              }
              const float2 h2 = unpack_f2(a2);
              r2 = h2.x + h2.y;
            } else if constexpr (D > 0 && D % 2 == 0) {
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
              for (int t = 0; t < AT_MAXD; ++t) {
                const float df = t < d ? x[t] - z[t] : 0.f;
                r2 = fmaf(df, df, r2);
              }
            }
            kv[u] = (kk < kmax && pvalid) ? cov_r2_fast(r2, KIND, AT_KSCALE) : 0.f;
          }
        }
        uint32_t hv[2], lv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) split_h2(kv[2 * u], kv[2 * u + 1], hv[u], lv[u]);
        const uint32_t off = sw128_off16(krow, kq * 16 + q * 4);
        *reinterpret_cast<uint2*>(a_hi + off) = make_uint2(hv[0], hv[1]);
        *reinterpret_cast<uint2*>(a_lo + off) = make_uint2(lv[0], lv[1]);
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
  if (tc::bar_sync_or(2, AT_THREADS, failed)) {
    if (tid == 0 && status) flag_status(status, ST_TIMEOUT, blockIdx.x);
  } else {
    const int64_t row = row0 + dl + lane;
    const int c0 = h * AT_N + dc;
    if (row < n) {
      float* dst = A + (size_t)row * mpad + c0;
#pragma unroll
      for (int g = 0; g < 2; ++g)
        if (g < ngrp) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(colf + c0 + g * 32 + 2 * j));
            const float2 a = unpack_f2(acc2[g * 16 + j]), b = unpack_f2(acc2[g * 16 + j + 1]);
            *reinterpret_cast<float4*>(dst + g * 32 + 2 * j) = make_float4(a.x * f.x, a.y * f.y, b.x * f.z, b.y * f.w);
          }
        }
    }
  }
  tc::fence_before_sync();
  const bool drained = !tc::bar_sync_or(3, AT_THREADS, !fin_ok);
  if (warp == 0 && drained) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, AT_TMEM_COLS);
  }
}

using AKernel = void (*)(const float*, const float*, const unsigned char*, const float*, float*, int64_t, int, int,
                        int, int, int*);

template <int D>
AKernel a_kernel_for_kind(int kind) {
  switch (kind) {
    case VIF_MATERN12: return lowrank_A_tc_kernel<D, VIF_MATERN12>;
    case VIF_MATERN32: return lowrank_A_tc_kernel<D, VIF_MATERN32>;
    case VIF_MATERN52: return lowrank_A_tc_kernel<D, VIF_MATERN52>;
    default: return lowrank_A_tc_kernel<D, VIF_SE>;
  }
}
AKernel a_kernel(int d, int kind) {
  return d == 8 ? a_kernel_for_kind<8>(kind) : d == 5 ? a_kernel_for_kind<5>(kind)
         : d == 2 ? a_kernel_for_kind<2>(kind) : a_kernel_for_kind<0>(kind);
}

}  // namespace

cudaError_t lowrank_A_tc_init() {
  cudaError_t e = cudaSuccess;
  for (int d : {0, 2, 5, 8})
    for (int kind : {VIF_MATERN12, VIF_MATERN32, VIF_MATERN52, VIF_SE})
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)a_kernel(d, kind), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)AT_SMEM);
  return e;
}

// packed L_m^{-1} tiles, then the row scales (256 nh floats) and the read-out factors
size_t lowrank_A_tc_pack_floats(int mpad) {
  const int nh = (mpad + AT_N - 1) / AT_N, nchunk = (mpad + AT_K - 1) / AT_K;
  return (size_t)nh * nchunk * 2 * AT_BTILE / sizeof(float) + 2 * (size_t)nh * AT_N;
}

cudaError_t lowrank_A_tc(const float* Xs, const float* Zs, const double* Linv, int ldl, float* pack, float* A,
                         int64_t n, int d, int m, int mpad, int kind, double var, int* status, cudaStream_t s) {
  if (m <= 0) return cudaMemsetAsync(A, 0, sizeof(float) * (size_t)n * mpad, s);
  if (d > AT_MAXD || mpad % 32 != 0 || mpad < m || mpad - m >= 32 || n <= 0) return cudaErrorInvalidValue;
  // mpad = 32 ceil(m / 32): the last chunk of 64 may hold 32 padding columns, packed as zeros
  const int nh = (mpad + AT_N - 1) / AT_N, nchunk = (mpad + AT_K - 1) / AT_K;
  unsigned char* tiles = reinterpret_cast<unsigned char*>(pack);
  float* rs = pack + (size_t)nh * nchunk * 2 * AT_BTILE / sizeof(float);
  float* colf = rs + (size_t)nh * AT_N;
  const int rows = nh * AT_N;
  linv_rowscale_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(Linv, m, ldl, rows, var, rs, colf);
  const int64_t total = (int64_t)nh * nchunk * AT_N * (AT_K / 8);
  linv_pack_tc_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Linv, m, ldl, rs, tiles, nchunk, total);
  dim3 grid((unsigned)((n + AT_M - 1) / AT_M), (unsigned)nh);
  a_kernel(d, kind)<<<grid, AT_THREADS, AT_SMEM, s>>>(Xs, Zs, tiles, colf, A, n, d, m, mpad, nchunk, status);
  return cudaGetLastError();
}

}  // namespace vif
