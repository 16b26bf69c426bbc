// The residual products A_N^T A_N of the Vecchia factors (Sec. 2.1, Eq. D_A_Vecchia) on
// the fifth-generation tensor cores, for the float32 (mixed) path.
//
// Point i needs the Gram of the rows [A_N(i); a_i] of A (q + 1 <= 32 rows of length m):
// its residual covariance is K([N,i],[N,i]) + tdiag I minus that Gram.  One such Gram is
// far too small for a tensor-core tile (M = 128), so points are packed into groups:
// consecutive points of the spatial processing order whose rows, taken together, number
// at most 128 (neighbouring points share neighbours, so a group holds more points than
// 128 / (q + 1)).  The CTA forms the full 128 x 128 Gram of a group's rows U and every
// point of the group reads its (q + 1)^2 block from it.
//
// Precision: each float32 value x of A, scaled by a power of two s that keeps |s x| <= 2^10
// (|x| <= sigma_1, as a row of A = L_m^{-1} K_mn has norm at most sigma_1), is split into two
// float16 values h = rn_f16(s x), l = rn_f16(s x - h): h carries 11 significant bits, and
// h + l represents s x to 2^-22 relative (l may be subnormal for |x| below 2^-13 / s, where
// its absolute error stays below 2^-25 / s).  The Gram is taken as P = H H^T + H (2L)^T
// (float16 inputs, float32 accumulation, products exact), whose symmetric part
//   (P + P^T) / 2 = H H^T + H L^T + L H^T = s^2 (x_a . x_b) up to 2^-21 relative
// is the two-term split product in two MMAs per K-step of 16 columns; 2L is exact.  What
// is left of the truncating accumulation after the per-chunk drains shifts every entry of
// a block alike (neighbouring rows are strongly correlated), so it is kept consistent
// between diagonal and off-diagonal entries; the D_i it leaves stay inside the spread of
// float32 rounding (measured against the float64 oracle, see the tests).  The
// tensor core's float32 accumulation rounds toward zero at every step, so no TMEM
// accumulator runs longer than one chunk of 64 columns (eight MMAs): each chunk's partial
// is added (round to nearest) into running sums held in the drain warps' registers.
//
// Roles (persistent CTAs, one per SM, each taking groups blockIdx.x, + gridDim.x, ...; the
// chunks of consecutive groups form one pipeline; chunk c's tiles are in operand stage
// c % UG_NS and its Gram partial in TMEM accumulator c % UG_NA):
//   warp 0       one lane issues the MMAs of chunk c once its tiles are staged and its
//                accumulator has been read out;
//   warps 1-4    (one per TMEM lane quarter) add the accumulator into running sums kept in a
//                further TMEM region (round to nearest); after a group's last chunk they write
//                the sums (times 1/s^2) to shared memory and copy each point's block,
//                symmetrised, to gsub;
//   warps 5-20   load the group's rows of A with 16-byte vector loads two chunks ahead (the
//                gathers keep many loads in flight), split them and store the float16 tiles.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "vif_internal.cuh"
#include "vif_tc.cuh"

namespace vif {

namespace {

constexpr int UG_R = 128;                          // rows per group (MMA M = N)
constexpr int UG_K = 64;                           // columns of A per chunk
constexpr int UG_NS = 3;                           // operand stages
constexpr int UG_NA = 3;                           // TMEM accumulators (+ one region of running sums)
constexpr int UG_DW = 4;                           // drain warps
constexpr int UG_SW = 16;                          // staging warps
constexpr int UG_NST = UG_SW * 32;                 // staging threads
constexpr int UG_ND = UG_DW * 32;                  // drain threads
constexpr int UG_THREADS = 32 + UG_ND + UG_NST;    // 672
constexpr int UG_LPT = UG_R * UG_K / 4 / UG_NST;   // 16-byte loads per staging thread per chunk (4)
constexpr uint32_t UG_TILE = UG_R * 128;           // one 128-byte-swizzled 128 x 64 tile of f16
constexpr uint32_t UG_STAGE = 2 * UG_TILE;         // hi, 2 lo
constexpr int UG_GLD = UG_R + 1;                   // row stride (floats) of the group Gram in smem
constexpr uint32_t UG_GS_BYTES = UG_R * UG_GLD * 4;
constexpr int UG_MAXPTS = UG_MAX_POINTS;           // points per group (the loc prefetch holds 32 each)
constexpr uint32_t UG_LOC_BYTES = UG_MAXPTS * 32;
constexpr uint32_t UG_SMEM = UG_NS * UG_STAGE + UG_GS_BYTES + UG_LOC_BYTES + 1024;
constexpr uint32_t UG_TMEM_COLS = 512;             // UG_NA accumulators and the running sums
constexpr uint32_t UG_SUM_COL = UG_NA * UG_R;
static_assert(UG_SUM_COL + UG_R <= UG_TMEM_COLS, "TMEM holds the accumulators and the sums");
static_assert(UG_LPT == 4, "staging: four 16-byte loads per thread and chunk");

struct __align__(16) UgBars {
  uint64_t staged[UG_NS];    // tiles of the stage stored (one arrival per staging thread)
  uint64_t sdone[UG_NS];     // MMAs reading the stage finished: stage free
  uint64_t adone[UG_NA];     // MMAs of the accumulator's chunk finished: accumulator ready
  uint64_t drained[UG_NA];   // accumulator added into the sums (one arrival per drain thread)
  uint64_t fin;              // every MMA of the CTA finished
  uint32_t tmem;
  int abort;
  unsigned char tri_a[528], tri_b[528];   // entry e of the packed lower triangle -> (a, b)
};

__device__ __forceinline__ void cp_async16z(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(tc::smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}

// two float32 -> packed float16x2 (round to nearest), a in the low half
__device__ __forceinline__ uint32_t f16x2_rn(float a, float b) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
__device__ __forceinline__ float2 f16x2_to_f32(uint32_t v) {
  return __half22float2(*reinterpret_cast<const __half2*>(&v));
}

// (hi, 2 lo) of two scaled values, packed float16x2
__device__ __forceinline__ void split2(float x0, float x1, float sc, uint32_t& h, uint32_t& l) {
  const float a0 = sc * x0, a1 = sc * x1;
  h = f16x2_rn(a0, a1);
  const float2 hf = f16x2_to_f32(h);
  const float d0 = a0 - hf.x, d1 = a1 - hf.y;   // exact
  l = f16x2_rn(d0 + d0, d1 + d1);
}

__global__ __launch_bounds__(UG_THREADS, 1) void union_gram_tc_kernel(
    const float* __restrict__ A, int mpad, const int32_t* __restrict__ grows, const int32_t* __restrict__ gptr,
    int64_t ngroups, const unsigned char* __restrict__ loc, int Q, float sc, float* __restrict__ gsub,
    int* status) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ UgBars sb;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* Gs = reinterpret_cast<float*>(smem + UG_NS * UG_STAGE);               // [UG_R][UG_GLD]
  unsigned char* locbuf = smem + UG_NS * UG_STAGE + UG_GS_BYTES;               // [UG_MAXPTS][32]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunk = (mpad + UG_K - 1) / UG_K;
  const int64_t ngc = ngroups > blockIdx.x ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t T = ngc * nchunk;   // chunks of this CTA
  const int SUB = Q * (Q + 1) / 2;
  const uint32_t idesc = tc::idesc_f16(UG_R, UG_R);

  if (warp == 0) tc::tmem_alloc(&sb.tmem, UG_TMEM_COLS);
  if (tid == 0) {
    for (int b = 0; b < UG_NS; ++b) {
      tc::mbar_init(&sb.staged[b], UG_NST);
      tc::mbar_init(&sb.sdone[b], 1);
    }
    for (int q = 0; q < UG_NA; ++q) {
      tc::mbar_init(&sb.adone[q], 1);
      tc::mbar_init(&sb.drained[q], UG_ND);
    }
    tc::mbar_init(&sb.fin, 1);
    sb.abort = 0;
    tc::fence_mbar_init();
  }
  for (int e = tid; e < SUB; e += UG_THREADS) {
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    sb.tri_a[e] = (unsigned char)a;
    sb.tri_b[e] = (unsigned char)(e - a * (a + 1) / 2);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sb.tmem;
  bool failed = false;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issue (one lane)
    if (lane == 0) {
      for (int64_t c = 0; c < T; ++c) {
        const int b = (int)(c % UG_NS), q = (int)(c % UG_NA);
        if (!tc::mbar_wait(&sb.staged[b], (uint32_t)(c / UG_NS) & 1u) ||
            (c >= UG_NA && !tc::mbar_wait(&sb.drained[q], (uint32_t)((c - UG_NA) / UG_NA) & 1u))) {
          failed = true;
          sb.abort = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t dt = tmem + (uint32_t)(q * UG_R);
        const uint32_t ah = tc::smem_addr(smem + b * UG_STAGE), al = ah + UG_TILE;
        // the small H (2L)^T terms first, the H H^T products last
#pragma unroll
        for (int ks = 0; ks < UG_K / 16; ++ks)
          tc::mma_f16(dt, tc::desc_k_sw128(ah + ks * 32), tc::desc_k_sw128(al + ks * 32), idesc, ks > 0);
#pragma unroll
        for (int ks = 0; ks < UG_K / 16; ++ks)
          tc::mma_f16(dt, tc::desc_k_sw128(ah + ks * 32), tc::desc_k_sw128(ah + ks * 32), idesc, 1u);
        tc::mma_commit(&sb.sdone[b]);
        tc::mma_commit(&sb.adone[q]);
      }
      tc::mma_commit(&sb.fin);
    }
    __syncwarp();
  } else if (warp <= UG_DW) {
    // ------------------------------------------------------------ drain and extraction
    const int dtid = tid - 32;
    const int qd = warp & 3;                       // TMEM lane quarter of this warp
    const int arow = 32 * qd + lane;
    const uint32_t lbase = tmem + ((uint32_t)(32 * qd) << 16);
    const float unscale = 1.0f / (sc * sc);        // a power of two: exact
    int p0 = 0, p1 = 0;
    int64_t jg = 0;
    int k = 0;
    for (int64_t c = 0; c < T; ++c, k = (k + 1 == nchunk) ? 0 : k + 1, jg += (k == 0)) {
      const int q = (int)(c % UG_NA);
      const bool first = k == 0, last = k == nchunk - 1;
      const int64_t g = blockIdx.x + jg * gridDim.x;
      if (first) {
        p0 = gptr[g];
        p1 = min(gptr[g + 1], p0 + UG_MAXPTS);   // groups are built with at most UG_MAXPTS points
      }
      if (last) {
        // the group's local-row table into shared memory, ahead of its extraction
        const int nb = (p1 - p0) * 32;
        for (int o = dtid * 16; o < nb; o += UG_ND * 16) cp_async16z(locbuf + o, loc + (size_t)p0 * 32 + o, 16u);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
      if (!failed && !__all_sync(0xffffffffu, tc::mbar_wait_sleep(&sb.adone[q], (uint32_t)(c / UG_NA) & 1u)))
        failed = true;
      if (!failed) {
        tc::fence_after_sync();
#pragma unroll 1
        for (int g4 = 0; g4 < UG_R / 32; ++g4) {
          float v[32];
          if (first) {
            tc::tmem_ld32(lbase + (uint32_t)(q * UG_R + 32 * g4), v);
          } else {
            float w[32];
            tc::tmem_ld32_pair(lbase + (uint32_t)(q * UG_R + 32 * g4), lbase + UG_SUM_COL + (uint32_t)(32 * g4), v,
                               w);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += w[i];
          }
          if (last) {
#pragma unroll
            for (int i = 0; i < 32; ++i) Gs[arow * UG_GLD + 32 * g4 + i] = v[i] * unscale;
          } else {
            tc::tmem_st32(lbase + UG_SUM_COL + (uint32_t)(32 * g4), v);
          }
        }
        if (!last) tc::tmem_st_wait();
        tc::fence_before_sync();
        tc::mbar_arrive(&sb.drained[q]);
      }
      if (last) {
        // the group's Gram is complete in Gs: copy each point's block, symmetrised
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        if (tc::bar_sync_or(2, UG_ND, failed)) failed = true;
        if (!failed) {
          // thread -> entries dtid, + 128, ... of every point of the group
          for (int ent = dtid; ent < SUB; ent += UG_ND) {
            const int ta = sb.tri_a[ent], tb = sb.tri_b[ent];
            for (int pl = 0; pl < p1 - p0; ++pl) {
              const int la = locbuf[pl * 32 + ta], lb = locbuf[pl * 32 + tb];
              if (la < UG_R && lb < UG_R)
                gsub[(size_t)(p0 + pl) * SUB + ent] = 0.5f * (Gs[la * UG_GLD + lb] + Gs[lb * UG_GLD + la]);
            }
          }
        }
        tc::bar_sync_or(2, UG_ND, false);
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  } else {
    // ------------------------------------------------------------ staging
    // Thread st loads 16-byte segment st % 16 of rows st / 16 + 32 j (j < 4) of each chunk
    // (a warp instruction reads two whole 256-byte row pieces), two chunks ahead of the one
    // it splits; the split stores 4 f16 hi and 4 f16 (2 lo) values per row and chunk at
    // columns 4 (st % 16) .. + 3 of the 128-byte-swizzled tiles.
    const int st = tid - 32 * (1 + UG_DW);
    const int seg = st & 15, row0 = st >> 4;
    int gcur[UG_LPT], gnxt[UG_LPT];   // global rows of the group being loaded, and of the next
#pragma unroll
    for (int j = 0; j < UG_LPT; ++j) {
      gcur[j] = ngc > 0 ? grows[(size_t)blockIdx.x * UG_R + row0 + 32 * j] : -1;
      gnxt[j] = ngc > 1 ? grows[(size_t)(blockIdx.x + gridDim.x) * UG_R + row0 + 32 * j] : -1;
    }
    int64_t fg = 0;
    int fk = 0;
    // the loads of chunk cl: zeros past mpad and for padding rows
    auto load = [&](int64_t cl, float4 (&x)[UG_LPT]) {
      const int col = fk * UG_K + seg * 4;
#pragma unroll
      for (int j = 0; j < UG_LPT; ++j)
        x[j] = (cl < T && gcur[j] >= 0 && col < mpad)
                   ? __ldg(reinterpret_cast<const float4*>(A + (size_t)gcur[j] * mpad + col))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      if (cl < T && ++fk == nchunk) {
        fk = 0;
        ++fg;
#pragma unroll
        for (int j = 0; j < UG_LPT; ++j) {
          gcur[j] = gnxt[j];
          gnxt[j] = fg + 1 < ngc ? grows[(size_t)(blockIdx.x + (fg + 1) * gridDim.x) * UG_R + row0 + 32 * j] : -1;
        }
      }
    };
    // the split and stores of chunk cs from its loaded values
    auto store = [&](int64_t cs, const float4 (&x)[UG_LPT]) {
      const int b = (int)(cs % UG_NS);
      // stage b was last read by the MMAs of chunk cs - UG_NS
      if (cs >= UG_NS && !tc::mbar_wait_sleep(&sb.sdone[b], (uint32_t)((cs - UG_NS) / UG_NS) & 1u)) {
        failed = true;
        return;
      }
      unsigned char* th = smem + b * UG_STAGE;
#pragma unroll
      for (int j = 0; j < UG_LPT; ++j) {
        const int r = row0 + 32 * j;
        uint2 hv, lv;
        split2(x[j].x, x[j].y, sc, hv.x, lv.x);
        split2(x[j].z, x[j].w, sc, hv.y, lv.y);
        const uint32_t off = r * 128 + ((((uint32_t)(seg >> 1)) ^ (uint32_t)(r & 7)) << 4) + 8 * (seg & 1);
        *reinterpret_cast<uint2*>(th + off) = hv;
        *reinterpret_cast<uint2*>(th + UG_TILE + off) = lv;
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(&sb.staged[b]);
    };
    float4 xa[UG_LPT], xb[UG_LPT], xc[UG_LPT];
    load(0, xa);
    load(1, xb);
    for (int64_t c = 0; c < T; c += 3) {
      if (failed || sb.abort) break;
      load(c + 2, xc);
      store(c, xa);
      if (c + 1 >= T || failed) break;
      load(c + 3, xa);
      store(c + 1, xb);
      if (c + 2 >= T || failed) break;
      load(c + 4, xb);
      store(c + 2, xc);
    }
  }
  // a wait that gave up may leave MMAs in flight: wait for them once more (bounded) and
  // release the TMEM only once they have finished (a call that reports the timeout
  // discards its results)
  bool fin_ok = tc::mbar_wait(&sb.fin, 0);
  if (!fin_ok) {
    failed = true;
    fin_ok = tc::mbar_wait(&sb.fin, 0);
  }
  tc::fence_after_sync();
  if (__syncthreads_or(failed) && tid == 0 && status) flag_status(status, ST_TIMEOUT, blockIdx.x);
  tc::fence_before_sync();
  const bool drained = __syncthreads_and(fin_ok);
  if (warp == 0 && drained) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, UG_TMEM_COLS);
  }
}

}  // namespace

cudaError_t union_gram_tc_init() {
  return cudaFuncSetAttribute(union_gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UG_SMEM);
}

cudaError_t union_gram_tc(const float* A, int mpad, const UnionGroups& ug, int Q, double var, float* gsub,
                          int* status, cudaStream_t s, int nsm) {
  if (mpad % 32 != 0 || Q < 1 || Q > 32 || ug.ngroups < 0 || !(var > 0.0)) return cudaErrorInvalidValue;
  if (ug.ngroups == 0) return cudaSuccess;
  // s = 2^(10 - e) with 2^e >= sigma_1 >= |A_ij|: s |A_ij| <= 2^10, far inside float16
  int e = 0;
  std::frexp(std::sqrt(var) * 1.0001, &e);
  const float sc = std::ldexp(1.0f, 10 - e);
  const unsigned grid = (unsigned)std::min<int64_t>(ug.ngroups, std::max(nsm, 1));
  union_gram_tc_kernel<<<grid, UG_THREADS, UG_SMEM, s>>>(A, mpad, ug.rows, ug.ptr, ug.ngroups, ug.loc, Q, sc,
                                                           gsub, status);
  return cudaGetLastError();
}

// Groups of consecutive points of `order` whose rows [N(i), i] together number at most
// UG_R (and at most max_pts points); false (and nothing built) if m_v + 1 > 32 or the
// neighbour table holds an index that is not a predecessor.  rows: ngroups x UG_R global row indices (-1 padded);
// ptr: ngroups + 1 offsets into the processing order; loc: per slot of the order, the
// group-local row of each of the point's rows (t < q: neighbour t, t = q: the point),
// 0xFF beyond.
bool build_union_groups(const int32_t* N, const int32_t* order, int64_t n, int mv, int max_pts,
                        std::vector<int32_t>& rows, std::vector<int32_t>& ptr, std::vector<unsigned char>& loc) {
  if (mv + 1 > 32 || n < 1) return false;
  for (int64_t i = 0; i < n; ++i) {
    if (order[i] < 0 || order[i] >= n) return false;
    const int q = (int)std::min<int64_t>(i, mv);
    for (int t = 0; t < q; ++t) {
      const int32_t j = N[(size_t)i * mv + t];
      if (j < 0 || j >= i) return false;   // not a predecessor: the SIMT kernel reports it
    }
  }
  rows.clear();
  ptr.clear();
  loc.assign((size_t)n * 32, 0xFF);
  std::vector<int16_t> pos((size_t)n, -1);
  std::vector<int32_t> cur;
  cur.reserve(UG_R);
  int npts = 0;
  auto close = [&](int64_t slot) {
    for (int32_t r : cur) pos[r] = -1;
    for (size_t k = cur.size(); k < (size_t)UG_R; ++k) cur.push_back(-1);
    rows.insert(rows.end(), cur.begin(), cur.end());
    ptr.push_back((int32_t)slot);
    cur.clear();
    npts = 0;
  };
  ptr.push_back(0);
  for (int64_t slot = 0; slot < n; ++slot) {
    const int32_t i = order[slot];
    const int q = (int)std::min<int64_t>(i, mv);
    int fresh = pos[i] < 0 ? 1 : 0;
    for (int t = 0; t < q; ++t) fresh += pos[N[(size_t)i * mv + t]] < 0 ? 1 : 0;
    if (npts > 0 && ((int)cur.size() + fresh > UG_R || npts >= max_pts)) close(slot);
    auto take = [&](int32_t r) -> unsigned char {
      if (pos[r] < 0) {
        pos[r] = (int16_t)cur.size();
        cur.push_back(r);
      }
      return (unsigned char)pos[r];
    };
    for (int t = 0; t < q; ++t) loc[(size_t)slot * 32 + t] = take(N[(size_t)i * mv + t]);
    loc[(size_t)slot * 32 + q] = take(i);
    ++npts;
  }
  if (npts > 0) close(n);
  return true;
}

}  // namespace vif
