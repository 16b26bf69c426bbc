// G' = [F z]^T [F z] (the capacitance Gram of Sec. 2.2, C = I + F^T F with the
// response column appended) on the fifth-generation tensor cores, for the float32 path.
//
// Split-K SYRK over 128 x 128 tile pairs (ti >= tj) of the fpad columns: CTA (pair,
// slice) sums rows r0..r1 of F, 32 rows per chunk.  Warp specialisation: 8 staging warps
// bring the rows of chunk c+1 into a raw shared-memory buffer with cp.async, split every
// value of chunk c into tf32 hi + lo (round to nearest) and write them transposed into
// K-major 128-byte-swizzled tiles (row = column of F, K = row of F); 8 read-out warps (two
// per TMEM lane quarter) add each finished accumulator into the running sums while the
// staging warps prepare the next chunk; one more warp issues the chunk's 16 MMAs
//   Alo Blo + Alo Bhi + Ahi Blo + Ahi Bhi
// into one of two TMEM accumulators as soon as the tiles are staged.  The tensor core's
// float32 accumulation rounds toward zero at every step and C is ill-conditioned (its
// largest eigenvalue grows with n), so no TMEM accumulator runs longer than one chunk:
// the read-out adds it into double-float32 running sums (TwoSum) kept in two more TMEM
// regions, which frees the registers a per-thread sum would need.  lo x lo is kept: on
// the diagonal it is a sum of squares, and dropping it would shift every diagonal entry
// down by about 1e-7 of itself, which the eigenvalues of C near 1 do not tolerate.  The
// sums are written as float64 partials in the 64 x 64 pair layout that the float64 Gram
// kernel uses, so one reduction serves both.
#include "vif_internal.cuh"
#include "vif_tc.cuh"

namespace vif {

namespace {

constexpr int GC_T = 128;                       // tile edge (F columns per block)
constexpr int GC_K = 32;                        // rows of F per chunk
constexpr int GC_CW = 16;                       // compute warps: 8 read-out, then 8 staging
constexpr int GC_NC = GC_CW * 32;               // compute threads
constexpr int GC_NS = 256;                      // staging threads (warps 8..15)
constexpr int GC_ND = 256;                      // read-out threads (warps 0..7)
constexpr int GC_THREADS = GC_NC + 32;          // + the MMA warp
constexpr uint32_t GC_TILE = GC_T * 128;        // bytes of one swizzled operand tile
constexpr uint32_t GC_STAGE = 4 * GC_TILE;      // Ahi, Alo, Bhi, Blo
constexpr uint32_t GC_RAW = 2 * GC_K * GC_T * 4;  // raw rows of both blocks of one chunk
constexpr uint32_t GC_SMEM = 2 * GC_STAGE + 2 * GC_RAW + 1024;
constexpr uint32_t GC_TMEM_COLS = 4 * GC_T;     // accumulators 0, 1; running sums hi, lo
constexpr int GT64 = 64;                        // sub-tile edge of the partial layout

struct __align__(16) GcBars {
  uint64_t staged[2];   // tiles of the stage written (one arrival per staging thread)
  uint64_t done[2];     // MMAs of the stage's chunk finished (stage and accumulator free)
  uint64_t drained[2];  // accumulator read out (one arrival per read-out thread)
  uint64_t fin;         // every MMA of the CTA finished
  uint32_t tmem;
  int abort;            // the MMA warp gave up waiting
};

// 16-byte global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(tc::smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}

__global__ __launch_bounds__(GC_THREADS, 1) void gram_tc_kernel(const float* __restrict__ F, int64_t n, int fpad,
                                                                double* __restrict__ part, int nsplit,
                                                                int* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ GcBars sb;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* raw = reinterpret_cast<float*>(smem + 2 * GC_STAGE);   // [2][blk][GC_K][GC_T]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p = blockIdx.x;
  int ti = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= p) ++ti;
  while (ti * (ti + 1) / 2 > p) --ti;
  const int tj = p - ti * (ti + 1) / 2;
  const bool diag = ti == tj;
  const int nblk = diag ? 1 : 2;
  const int sidx = blockIdx.y;
  const int64_t per = (((n + nsplit - 1) / nsplit) + GC_K - 1) / GC_K * GC_K;
  const int64_t r0 = (int64_t)sidx * per;
  const int64_t r1 = (n < r0 + per) ? n : r0 + per;
  const int nchunk = r1 > r0 ? (int)((r1 - r0 + GC_K - 1) / GC_K) : 0;
  const uint32_t idesc = tc::idesc_tf32(GC_T, GC_T);

  if (warp == 0) tc::tmem_alloc(&sb.tmem, GC_TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&sb.staged[s], GC_NS);
      tc::mbar_init(&sb.done[s], 1);
      tc::mbar_init(&sb.drained[s], GC_ND);
    }
    tc::mbar_init(&sb.fin, 1);
    sb.abort = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sb.tmem;
  bool failed = false;

  if (warp == GC_CW) {
    // ------------------------------------------------ MMA warp (one lane)
    if (lane == 0) {
      for (int c = 0; c < nchunk; ++c) {
        const int s = c & 1;
        // the chunk's tiles are staged, and accumulator s was read out after chunk c-2
        if (!tc::mbar_wait(&sb.staged[s], (c >> 1) & 1) ||
            (c >= 2 && !tc::mbar_wait(&sb.drained[s], ((c - 2) >> 1) & 1))) {
          failed = true;
          sb.abort = 1;
          break;
        }
        tc::fence_after_sync();
        unsigned char* st = smem + s * GC_STAGE;
        const uint32_t dt = tmem + (uint32_t)(s * GC_T);
        const uint32_t ah = tc::smem_addr(st), al = ah + GC_TILE;
        const uint32_t bh = diag ? ah : ah + 2 * GC_TILE, bl = diag ? al : ah + 3 * GC_TILE;
        // the small terms first, the hi x hi products last
#pragma unroll
        for (int ks = 0; ks < GC_K / 8; ++ks) {
          const uint32_t o = ks * 32;
          tc::mma_tf32(dt, tc::desc_k_sw128(al + o), tc::desc_k_sw128(bl + o), idesc, ks > 0);
          tc::mma_tf32(dt, tc::desc_k_sw128(al + o), tc::desc_k_sw128(bh + o), idesc, 1u);
          tc::mma_tf32(dt, tc::desc_k_sw128(ah + o), tc::desc_k_sw128(bl + o), idesc, 1u);
        }
#pragma unroll
        for (int ks = 0; ks < GC_K / 8; ++ks) {
          const uint32_t o = ks * 32;
          tc::mma_tf32(dt, tc::desc_k_sw128(ah + o), tc::desc_k_sw128(bh + o), idesc, 1u);
        }
        tc::mma_commit(&sb.done[s]);
      }
      tc::mma_commit(&sb.fin);
    }
    __syncwarp();
  } else if (warp >= GC_CW / 2) {
    // ------------------------------------------------ staging warps
    const int stid = tid - GC_ND;
    // column (stid & 127) of both blocks, rows (stid >> 7) * 16 .. + 15 of the chunk
    const int scol = stid & (GC_T - 1), srow0 = (stid >> 7) * 16;
    // raw rows of chunk c into raw buffer c % 2: 16-byte segments, zeros past r1 / fpad
    auto fetch = [&](int c) {
      if (c < nchunk) {
        float* dst = raw + (size_t)(c & 1) * (2 * GC_K * GC_T);
        const int64_t rb = r0 + (int64_t)c * GC_K;
        for (int e = stid; e < nblk * GC_K * (GC_T / 4); e += GC_NS) {
          const int blk = e / (GC_K * (GC_T / 4));
          const int rr = (e / (GC_T / 4)) % GC_K, seg = e % (GC_T / 4);
          const int col = (blk == 0 ? ti : tj) * GC_T + seg * 4;
          const int64_t r = rb + rr;
          const bool ok = r < r1 && col < fpad;
          cp_async16z(dst + ((size_t)blk * GC_K + rr) * GC_T + seg * 4,
                      ok ? (const void*)(F + (size_t)r * fpad + col) : (const void*)F, ok ? 16u : 0u);
        }
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    fetch(0);
    for (int c = 0; c < nchunk; ++c) {
      const int s = c & 1;
      unsigned char* st = smem + s * GC_STAGE;
      unsigned char* a_hi = st;
      unsigned char* a_lo = st + GC_TILE;
      unsigned char* b_hi = diag ? a_hi : st + 2 * GC_TILE;
      unsigned char* b_lo = diag ? a_lo : st + 3 * GC_TILE;
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // raw rows of chunk c
      // stage s was last read by the MMAs of chunk c-2
      if (c >= 2 && !failed && !tc::mbar_wait(&sb.done[s], ((c - 2) >> 1) & 1)) failed = true;
      // everyone's rows of chunk c have landed and everyone is past chunk c-1's staging
      if (tc::bar_sync_or(1, GC_NS, failed || sb.abort)) {
        failed = true;
        break;
      }
      fetch(c + 1);
      const float* rw = raw + (size_t)s * (2 * GC_K * GC_T);
      for (int blk = 0; blk < nblk; ++blk) {
        unsigned char* th = blk == 0 ? a_hi : b_hi;
        unsigned char* tl = blk == 0 ? a_lo : b_lo;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float hv[4], lv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float v = rw[((size_t)blk * GC_K + srow0 + q * 4 + u) * GC_T + scol];
            hv[u] = tc::to_tf32(v);
            lv[u] = tc::to_tf32(v - hv[u]);
          }
          const uint32_t off = tc::sw128_off32(scol, srow0 + q * 4);
          *reinterpret_cast<float4*>(th + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<float4*>(tl + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(&sb.staged[s]);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  } else {
    // ------------------------------------------------ read-out warps
    // warp w: TMEM lanes 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63, in 16-column pieces
    const int dlane = 32 * (warp & 3), dcol = 64 * (warp >> 2);
    const uint32_t lane_base = tmem + ((uint32_t)dlane << 16);
    for (int j = 0; j < nchunk; ++j) {
      // warp-uniform outcome: the TMEM loads below are warp-collective
      if (failed || !__all_sync(0xffffffffu, tc::mbar_wait(&sb.done[j & 1], (j >> 1) & 1))) {
        failed = true;
        break;
      }
      tc::fence_after_sync();
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        const uint32_t col = (uint32_t)(dcol + g * 16);
        float v[16], hi[16], lo[16];
        // the partial and both running sums in flight together: one wait
        if (j == 0) {
          tc::tmem_ld16(lane_base + (uint32_t)((j & 1) * GC_T) + col, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            hi[i] = v[i];
            lo[i] = 0.f;
          }
        } else {
          uint32_t rv[16], rh[16], rl[16];
          tc::tmem_ld16_raw(lane_base + (uint32_t)((j & 1) * GC_T) + col, rv);
          tc::tmem_ld16_raw(lane_base + 2 * GC_T + col, rh);
          tc::tmem_ld16_raw(lane_base + 3 * GC_T + col, rl);
          tc::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            v[i] = __uint_as_float(rv[i]);
            hi[i] = __uint_as_float(rh[i]);
            lo[i] = __uint_as_float(rl[i]);
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float s2 = hi[i] + v[i];
            const float bb = s2 - hi[i];
            const float err = (hi[i] - (s2 - bb)) + (v[i] - bb);
            hi[i] = s2;
            lo[i] += err;
          }
        }
        tc::tmem_st16(lane_base + 2 * GC_T + col, hi);
        tc::tmem_st16(lane_base + 3 * GC_T + col, lo);
      }
      tc::tmem_st_wait();
      tc::fence_before_sync();
      tc::mbar_arrive(&sb.drained[j & 1]);
    }
    if (!failed) {
      const int np64 = (fpad / GT64) * (fpad / GT64 + 1) / 2;
      const int row = ti * GC_T + dlane + lane;
#pragma unroll 1
      for (int g = 0; g < 4; ++g) {
        float hi[16], lo[16];
        if (nchunk > 0) {
          tc::tmem_ld16(lane_base + 2 * GC_T + (uint32_t)(dcol + g * 16), hi);
          tc::tmem_ld16(lane_base + 3 * GC_T + (uint32_t)(dcol + g * 16), lo);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = tj * GC_T + dcol + g * 16 + i;
          if (row >= fpad || col >= fpad || col > row) continue;
          const int a64 = row / GT64, b64 = col / GT64;
          const int p64 = a64 * (a64 + 1) / 2 + b64;
          part[((size_t)sidx * np64 + p64) * GT64 * GT64 + (size_t)(row % GT64) * GT64 + (col % GT64)] =
              (double)hi[i] + (double)lo[i];
        }
      }
    }
  }
  // every MMA issued by this CTA completes on `fin` (committed by the MMA warp)
  // after a wait that gave up, MMAs may still be in flight: wait for them once more
  // (bounded) and release the TMEM only once they have finished (results of a call that
  // reports the timeout are discarded)
  bool fin_ok = tc::mbar_wait(&sb.fin, 0);
  if (!fin_ok) {
    failed = true;
    fin_ok = tc::mbar_wait(&sb.fin, 0);
  }
  tc::fence_after_sync();
  if (__syncthreads_or(failed) && tid == 0 && status) flag_status(status, ST_TIMEOUT, p);
  tc::fence_before_sync();
  const bool drained = __syncthreads_and(fin_ok);
  if (warp == 0 && drained) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, GC_TMEM_COLS);
  }
}

}  // namespace

cudaError_t gram_tc_init() {
  return cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GC_SMEM);
}

int gram_tc_nsplit(int64_t n, int fpad) {
  // at most one wave of one CTA per SM; slices of at least 64 chunks (2048 rows), so that a
  // small problem's few CTAs leave room for other problems' Grams on concurrent streams, but
  // no fewer than 8 CTAs while slices of 16 chunks allow it (the latency of a lone small call)
  const int nt = (fpad + GC_T - 1) / GC_T;
  const int npairs = nt * (nt + 1) / 2;
  int64_t want = 152 / npairs;
  const int64_t s64 = (n + 64 * GC_K - 1) / (64 * GC_K), s16 = (n + 16 * GC_K - 1) / (16 * GC_K);
  const int64_t low = (8 + npairs - 1) / npairs;
  const int64_t maxs = s64 > (s16 < low ? s16 : low) ? s64 : (s16 < low ? s16 : low);
  if (want > maxs) want = maxs;
  return (int)(want < 1 ? 1 : want);
}

cudaError_t gram_tc(const float* F, int64_t n, int fpad, double* part, int nsplit, int* status, cudaStream_t s) {
  if (fpad % GT64 != 0 || nsplit < 1) return cudaErrorInvalidValue;
  const int nt = (fpad + GC_T - 1) / GC_T;
  gram_tc_kernel<<<dim3(nt * (nt + 1) / 2, nsplit), GC_THREADS, GC_SMEM, s>>>(F, n, fpad, part, nsplit, status);
  return cudaGetLastError();
}

}  // namespace vif
