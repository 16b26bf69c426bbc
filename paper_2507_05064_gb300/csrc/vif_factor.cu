// Residual Vecchia factors and the likelihood (Sec. 2.1-2.2).
//
// For point i with neighbours N = N(i) (q = |N| <= m_v) the kernel forms the
// (q+1) x (q+1) residual covariance of (s_N, s_i),
//     R = K([N,i],[N,i]) + tdiag I - [A_N; a_i] [A_N; a_i]^T,
// which holds Sigma~_N - Sigma_mN^T Sigma_m^{-1} Sigma_mN, its cross term with i
// and c~_r(i,i) of Eq. D_A_Vecchia (tdiag = sigma^2, or the latent jitter).  The
// Cholesky factor of R gives both outputs at once: with [l^T, l_ii] its last row,
// D_i = l_ii^2 and A_i = l^T L_NN^{-1}, i.e. the solution of L_NN^T A_i^T = l.
// It then emits the row  f_i = (a_i - sum_k A_i[k] a_{N_k}) / sqrt(D_i)  of
// F = D^{-1/2} B A^T and  z_i = (y_i - sum_k A_i[k] y_{N_k}) / sqrt(D_i)  of
// z = D^{-1/2} B y, stored as [F z] (n x fpad, z in column m).
//
// With Q = B^T D^{-1} B and C = I + A Q A^T = I + F^T F (= L_m^{-1} M L_m^{-T}, M
// of Eq. def_M), Woodbury and Sylvester (Sec. 2.2) give
//     log det Sigma~_dagger = log det C + sum_i log D_i,
//     y^T Sigma~_dagger^{-1} y = z^T z - u^T C^{-1} u,   u = F^T z.
// Both come from one Cholesky of the (m+1) x (m+1) matrix
//     G' = [F z]^T [F z] + diag(1,...,1,0) = [[C, u], [u^T, z^T z]]:
// its first m pivots give log det C and the square of its last pivot is
// z^T z - u^T C^{-1} u.
#include <algorithm>

#include "vif_internal.cuh"

namespace vif {

// ---------------------------------------------------------------------------
// Factor kernel: one warp per point.  The (q+1) rows [A_N; a_i] are padded to
// 7R rows and their Gram is split into the 28 R x R blocks (bi, bj), bj <= bi < 7,
// one per lane (28 of 32 lanes busy).  Rows stream through a double-buffered
// shared-memory window of 128 bytes per row, filled with cp.async while the
// previous window is being multiplied; each lane reads its operands as 16-byte
// vectors along k.  Points are visited in `order` (a spatial ordering chosen at
// build) so that neighbouring rows of A are still in L2 when they are gathered.
// ---------------------------------------------------------------------------
constexpr int FK_WARPS = 4;
constexpr int FK_MAXD = 16;
constexpr int FK_NB = 7;

__constant__ unsigned char c_blk_i[28] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4,
                                          4, 5, 5, 5, 5, 5, 5, 6, 6, 6, 6, 6, 6, 6};
__constant__ unsigned char c_blk_j[28] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3,
                                          4, 0, 1, 2, 3, 4, 5, 0, 1, 2, 3, 4, 5, 6};

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ void vget(const float4& v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
__device__ __forceinline__ void vget(const double2& v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
// 16 bytes, or 16 zero bytes when !valid (nothing is read from gmem then)
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool valid) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// 1/sqrt(p): the float32 hardware estimate plus one Newton step y <- y (3 - p y^2) / 2
// (float), or two steps in float64 (double); a division-free pivot for the warp Cholesky.
__device__ __forceinline__ float rsqrt_refined(float p) {
  const float y = rsqrtf(p);
  return y * fmaf(-0.5f * p * y, y, 1.5f);
}
__device__ __forceinline__ double rsqrt_refined(double p) {
  double y = (double)rsqrtf((float)p);
  y = y * (1.5 - 0.5 * p * y * y);
  y = y * (1.5 - 0.5 * p * y * y);
  return y;
}

template <typename T, int R, bool GS = false>
struct FactorSmem {
  // float32 with R = 3 (m_v = 14..20): seven-row blocks on 5 column groups of a
  // 40-column window (see the kernel); otherwise R x R blocks on 128-byte windows.
  // GS: the Gram comes from the tensor-core kernel, no windows are needed.
  static constexpr bool BIG = (sizeof(T) == 4 && R == 3 && !GS);
  static constexpr int QM = FK_NB * R;
  static constexpr int V = Vec16<T>::n;       // elements per 16 bytes
  static constexpr int GK = 5;                // BIG: column groups
  static constexpr int KC = BIG ? 8 * GK : 128 / (int)sizeof(T);   // window width
  static constexpr int LD = KC + V;           // row stride (16-byte aligned, bank shift)
  static constexpr int PL = BIG ? 6 * GK : 1, PE = BIG ? 49 : 1;   // BIG: partial Gram blocks
  // the windows are dead once the Gram is formed: the partial sums of the column
  // groups and the coordinates of the rows reuse their space
  struct Post {
    alignas(16) T xc[QM][FK_MAXD];
    T part[PL][PE];
  };
  union {
    alignas(16) T buf[2][GS ? 1 : QM][LD];
    Post post;
  };
  T G[QM][QM + 1];
  T coef[QM];
  int idx[QM];
};

// |x_a - x_b|^2 over d coordinates of two shared-memory rows (16-byte aligned)
template <typename T>
__device__ __forceinline__ T sqdist_rows(const T* __restrict__ xa, const T* __restrict__ xb, int d) {
  if constexpr (sizeof(T) == 4) {
    if ((d & 3) == 0) {
      float s = 0.f;
      for (int c = 0; c < d; c += 4) {
        const float4 a = *reinterpret_cast<const float4*>(xa + c), b = *reinterpret_cast<const float4*>(xb + c);
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        s = fmaf(d0, d0, s);
        s = fmaf(d1, d1, s);
        s = fmaf(d2, d2, s);
        s = fmaf(d3, d3, s);
      }
      return s;
    }
  }
  return sqdist(xa, xb, d);
}

// The factors and the row of [F z] of the point at position `slot` of the processing order,
// by one warp with its shared-memory block S.
template <typename T, int R, bool GS>
__device__ __forceinline__ void factor_point(
    const T* __restrict__ A, const T* __restrict__ Xs, const int32_t* __restrict__ N,
    const int32_t* __restrict__ order, const double* __restrict__ y, int64_t n, int d, int m, int mpad, int mv,
    int fpad, const CovParams& cp, T* __restrict__ F, double* __restrict__ Acoef, double* __restrict__ Dv,
    double* __restrict__ logD, int* status, const float* __restrict__ gsub, float* __restrict__ rho,
    const int64_t slot, FactorSmem<T, R, GS>& S) {
  using SM = FactorSmem<T, R, GS>;
  constexpr int QM = SM::QM, V = SM::V, KC = SM::KC;
  using VT = typename Vec16<T>::type;
  const int lane = threadIdx.x & 31;
  const int64_t i = order ? (int64_t)order[slot] : slot;
  const int q = (int)(i < (int64_t)mv ? i : (int64_t)mv);
  const int Q = q + 1;
  for (int t = lane; t < QM; t += 32) {
    int j = (t < q) ? N[(size_t)i * mv + t] : (t == q ? (int)i : -1);
    if (t < q && (j < 0 || (int64_t)j >= i)) {   // not a predecessor: report, read a valid row
      flag_status(status, ST_BAD_NEIGHBOR, i);
      j = 0;
    }
    S.idx[t] = j;
  }
  __syncwarp();
  if constexpr (!GS) {
  // rows Q..QM-1 of both windows stay zero (none once i >= m_v)
  for (int e = lane; e < 2 * (QM - Q) * SM::LD; e += 32) {
    const int b = e / ((QM - Q) * SM::LD), r = e % ((QM - Q) * SM::LD);
    S.buf[b][Q + r / SM::LD][r % SM::LD] = T(0);
  }
  __syncwarp();
  // ---- Gram of the gathered rows of A, double-buffered windows of KC columns
  // float32 with 15 <= Q <= 21 (the m_v = 20 workloads): seven-row blocks, 3 x 3 grid,
  // 6 lower block pairs x 5 column groups on 30 lanes, lane kg taking the window
  // columns kg + 5t, so each lane reads 14 values per column for 49 products; the 5
  // partial sums of a block pair are added through shared memory at the end.
  constexpr bool BIG = SM::BIG;
  if constexpr (BIG) {
    constexpr int BR = 7, GK = SM::GK;
    const bool own = lane < 6 * GK;
    const int bp = own ? lane / GK : 0, kg = lane % GK;
    const int bi = (bp == 0) ? 0 : (bp < 3 ? 1 : 2);
    const int bj = bp - (bi * (bi + 1) / 2);
    float acc[BR][BR];
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int c = 0; c < BR; ++c) acc[r][c] = 0.f;
    const int nwin = (m + KC - 1) / KC;
    constexpr int SEG = KC / V;
    auto issue = [&](int win, int b) {
      const int k0 = win * KC;
      for (int e = lane; e < Q * SEG; e += 32) {
        const int t = e / SEG, sg = e % SEG;
        const int k = k0 + sg * V;
        // columns past the row (the last window) are filled with zeros
        const bool in = k < mpad;
        cp_async16_zfill(&S.buf[b][t][sg * V], A + (size_t)S.idx[t] * mpad + (in ? k : 0), in);
      }
      cp_async_commit();
    };
    if (nwin > 0) issue(0, 0);
    for (int win = 0; win < nwin; ++win) {
      const int b = win & 1;
      if (win + 1 < nwin) {
        issue(win + 1, b ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
#pragma unroll 2
      for (int t = 0; t < KC / GK; ++t) {
        const int col = kg + GK * t;
        float u[BR], v[BR];
#pragma unroll
        for (int r = 0; r < BR; ++r) u[r] = (float)S.buf[b][bi * BR + r][col];
#pragma unroll
        for (int c = 0; c < BR; ++c) v[c] = (float)S.buf[b][bj * BR + c][col];
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int c = 0; c < BR; ++c) acc[r][c] = fmaf(u[r], v[c], acc[r][c]);
      }
      __syncwarp();
    }
    if (own) {
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int c = 0; c < BR; ++c) S.post.part[lane][r * BR + c] = acc[r][c];
    }
    __syncwarp();
    for (int e = lane; e < 6 * BR * BR; e += 32) {
      const int p = e / (BR * BR), rc = e % (BR * BR);
      const int pi = (p == 0) ? 0 : (p < 3 ? 1 : 2), pj = p - (pi * (pi + 1) / 2);
      float a = S.post.part[p * GK][rc];
#pragma unroll
      for (int k = 1; k < GK; ++k) a += S.post.part[p * GK + k][rc];
      S.G[pi * BR + rc / BR][pj * BR + rc % BR] = (T)a;
    }
    __syncwarp();
  } else {
  const bool owner = lane < 28;
  const int bi = owner ? c_blk_i[lane] : 0, bj = owner ? c_blk_j[lane] : 0;
  T acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = T(0);
  const int nwin = (m + KC - 1) / KC;
  constexpr int SEG = KC / V;                 // 16-byte segments per row window (8)
  auto issue = [&](int win, int b) {
    const int k0 = win * KC;
    for (int e = lane; e < Q * SEG; e += 32) {
      int t = e / SEG, sg = e % SEG;
      int k = k0 + sg * V;
      if (k < mpad) cp_async16(&S.buf[b][t][sg * V], A + (size_t)S.idx[t] * mpad + k);
    }
    cp_async_commit();
  };
  if (nwin > 0) issue(0, 0);
  for (int win = 0; win < nwin; ++win) {
    const int b = win & 1;
    if (win + 1 < nwin) {
      issue(win + 1, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    if (owner) {
#pragma unroll 2
      for (int kk = 0; kk < KC; kk += V) {
        T u[R][V], v[R][V];
#pragma unroll
        for (int r = 0; r < R; ++r) vget(*reinterpret_cast<const VT*>(&S.buf[b][bi * R + r][kk]), u[r]);
#pragma unroll
        for (int c = 0; c < R; ++c) vget(*reinterpret_cast<const VT*>(&S.buf[b][bj * R + c][kk]), v[c]);
#pragma unroll
        for (int e = 0; e < V; ++e)
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < R; ++c) acc[r][c] += u[r][e] * v[c][e];
      }
    }
    __syncwarp();
  }
  if (owner) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) S.G[bi * R + r][bj * R + c] = acc[r][c];
  }
  __syncwarp();
  }
  }  // !GS: the Gram of the gathered rows is in S.G
  // coordinates of the rows (their space was the windows')
  for (int e = lane; e < Q * d; e += 32) {
    const int t = e / d, c = e % d;
    S.post.xc[t][c] = Xs[(size_t)S.idx[t] * d + c];
  }
  __syncwarp();
  // ---- residual covariance R (lower triangle)
  const int npair = Q * (Q + 1) / 2;
  // lane walks the entries e = lane, lane + 32, ... of the triangle stored row by row
  // (e = a (a + 1) / 2 + b2): the first is decoded, the later ones stepped to
  int a = (int)((sqrtf(8.0f * lane + 1.0f) - 1.0f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= lane) ++a;
  while (a * (a + 1) / 2 > lane) --a;
  int b2 = lane - a * (a + 1) / 2;
  for (int e = lane; e < npair; e += 32, b2 += 32) {
    while (b2 > a) {
      b2 -= a + 1;
      ++a;
    }
    T kv = cov_r2<T>(sqdist_rows(&S.post.xc[a][0], &S.post.xc[b2][0], d), cp.kind, (T)cp.var);
    if (a == b2) kv += (T)cp.tdiag;
    if constexpr (GS)
      S.G[a][b2] = kv - (T)gsub[(size_t)slot * ((mv + 1) * (mv + 2) / 2) + e];
    else
      S.G[a][b2] = kv - S.G[a][b2];
  }
  __syncwarp();
  if (rho) {
    // residual correlations of i with its neighbours, R[q][k] / sqrt(R[q][q] R[k][k]): their
    // largest and mean absolute value (inputs of the learned preconditioner correction)
    float rmax = 0.f, rsum = 0.f;
    for (int k = lane; k < q; k += 32) {
      const float r = fabsf((float)((double)S.G[q][k] / sqrt((double)S.G[q][q] * (double)S.G[k][k])));
      rmax = fmaxf(rmax, r);
      rsum += r;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
      rsum += __shfl_xor_sync(0xffffffffu, rsum, off);
    }
    if (lane == 0) {
      rho[2 * i] = rmax;
      rho[2 * i + 1] = q > 0 ? rsum / (float)q : 0.f;
    }
  }
  T inv;   // 1 / sqrt(D_i)
  if constexpr (QM <= 32) {
    // ---- Cholesky of R in registers: lane r holds row r, columns broadcast by
    // shuffles; rows Q..QM-1 are identity so the unrolled sweep leaves them alone
    T row[QM];
#pragma unroll
    for (int c = 0; c < QM; ++c) {
      T v = (lane < Q && c <= lane) ? S.G[lane < QM ? lane : 0][c] : T(0);
      if (c == lane && lane >= Q) v = T(1);
      row[c] = v;
    }
    bool notpd = false;
    T my_rs = T(1);   // 1 / L[lane][lane]
#pragma unroll
    for (int c = 0; c < QM; ++c) {
      T piv = __shfl_sync(0xffffffffu, row[c], c);
      if (!(piv > T(0))) {
        notpd = true;
        piv = T(NAN);
      }
      const T rs = rsqrt_refined(piv);
      const T lc = (lane == c) ? piv * rs : row[c] * rs;
      if (lane == c) my_rs = rs;
      row[c] = lc;
      // lanes above s2 update entries above their diagonal, which are never read
#pragma unroll
      for (int s2 = c + 1; s2 < QM; ++s2) row[s2] = fma(-lc, __shfl_sync(0xffffffffu, lc, s2), row[s2]);
    }
    if (notpd && lane == 0) flag_status(status, ST_NOTPD_FACTOR, i);
    if (lane < Q) {
#pragma unroll
      for (int c = 0; c < QM; ++c)
        if (c <= lane) S.G[lane][c] = row[c];
    }
    __syncwarp();
    // ---- A_i: L_NN^T x = l (l = row q of the factor), column-oriented: once x_k
    // is known every t < k drops L[k][t] x_k from its right-hand side
    T b = (lane < q) ? S.G[q][lane] : T(0);
    T xk = T(0);
    for (int k = q - 1; k >= 0; --k) {
      const T x = __shfl_sync(0xffffffffu, b * my_rs, k);
      if (lane == k) xk = x;
      if (lane < k) b = fma(-S.G[k][lane], x, b);
    }
    if (lane < q) S.coef[lane] = xk;
    inv = __shfl_sync(0xffffffffu, my_rs, q);
    __syncwarp();
  } else if constexpr (QM <= 64 && sizeof(T) == 4) {
    // ---- float32: the same register sweep with two rows per lane, rows lane (ra) and
    // lane + 32 (rb); float64 rows of this length would not fit the register file
    T ra[QM], rb[QM];
    const int lb = lane + 32;
#pragma unroll
    for (int c = 0; c < QM; ++c) {
      T va = (lane < Q && c <= lane) ? S.G[lane][c] : T(0);
      if (c == lane && lane >= Q) va = T(1);
      T vb = (lb < Q && c <= lb) ? S.G[lb < QM ? lb : 0][c] : T(0);
      if (c == lb && lb >= Q) vb = T(1);
      ra[c] = va;
      rb[c] = vb;
    }
    bool notpd = false;
    T rsa = T(1), rsb = T(1);   // 1 / L[r][r] of the lane's two rows
#pragma unroll
    for (int c = 0; c < QM; ++c) {
      const bool hi = c >= 32;
      T piv = __shfl_sync(0xffffffffu, hi ? rb[c] : ra[c], c & 31);
      if (!(piv > T(0))) {
        notpd = true;
        piv = T(NAN);
      }
      const T rs = rsqrt_refined(piv);
      const T la = (!hi && lane == c) ? piv * rs : ra[c] * rs;
      const T lbv = (hi && lb == c) ? piv * rs : rb[c] * rs;
      if (!hi && lane == c) rsa = rs;
      if (hi && lb == c) rsb = rs;
      ra[c] = la;
      rb[c] = lbv;
#pragma unroll
      for (int s2 = c + 1; s2 < QM; ++s2) {
        const T ls = __shfl_sync(0xffffffffu, s2 < 32 ? la : lbv, s2 & 31);
        ra[s2] = fma(-la, ls, ra[s2]);
        rb[s2] = fma(-lbv, ls, rb[s2]);
      }
    }
    if (notpd && lane == 0) flag_status(status, ST_NOTPD_FACTOR, i);
#pragma unroll
    for (int c = 0; c < QM; ++c) {
      if (lane < Q && c <= lane) S.G[lane][c] = ra[c];
      if (lb < Q && c <= lb) S.G[lb][c] = rb[c];
    }
    __syncwarp();
    // ---- A_i: L_NN^T x = l column-oriented, rows t = lane and lane + 32 per lane
    T ba = (lane < q) ? S.G[q][lane] : T(0);
    T bb = (lb < q) ? S.G[q][lb] : T(0);
    T xa = T(0), xb = T(0);
    for (int k = q - 1; k >= 0; --k) {
      const T x = __shfl_sync(0xffffffffu, k >= 32 ? bb * rsb : ba * rsa, k & 31);
      if (lane == k) xa = x;
      if (lb == k) xb = x;
      if (lane < k) ba = fma(-S.G[k][lane], x, ba);
      if (lb < k) bb = fma(-S.G[k][lb], x, bb);
    }
    if (lane < q) S.coef[lane] = xa;
    if (lb < q) S.coef[lb] = xb;
    inv = __shfl_sync(0xffffffffu, q >= 32 ? rsb : rsa, q & 31);
    __syncwarp();
  } else {
    // ---- Cholesky of R (lower, in place)
    for (int c = 0; c < Q; ++c) {
      T piv = S.G[c][c];
      if (!(piv > T(0))) {
        if (lane == 0) flag_status(status, ST_NOTPD_FACTOR, i);
        piv = T(NAN);
      }
      T sp = dsqrt(piv);
      __syncwarp();
      if (lane == 0) S.G[c][c] = sp;
      for (int r = c + 1 + lane; r < Q; r += 32) S.G[r][c] /= sp;
      __syncwarp();
      for (int r = c + 1 + lane; r < Q; r += 32) {
        T grc = S.G[r][c];
        for (int s2 = c + 1; s2 <= r; ++s2) S.G[r][s2] -= grc * S.G[s2][c];
      }
      __syncwarp();
    }
    // ---- A_i: back substitution L_NN^T x = l, l = row q of the factor
    for (int t = lane; t < q; t += 32) S.coef[t] = S.G[q][t];
    __syncwarp();
    for (int k = q - 1; k >= 0; --k) {
      T x = S.coef[k] / S.G[k][k];
      __syncwarp();
      if (lane == 0) S.coef[k] = x;
      for (int t = lane; t < k; t += 32) S.coef[t] -= S.G[k][t] * x;
      __syncwarp();
    }
    inv = T(1) / S.G[q][q];
  }
  const T lii = S.G[q][q];
  for (int t = lane; t < mv; t += 32) Acoef[(size_t)i * mv + t] = (t < q) ? (double)S.coef[t] : 0.0;
  if (lane == 0) {
    if constexpr (sizeof(T) == 4) {
      // float64 instructions cost 64 cycles each on this part: D and log D of the
      // float32 factor are formed in float32 (they carry float32 information anyway)
      Dv[i] = (double)(lii * lii);
      logD[i] = (double)(2.f * logf(lii));
    } else {
      const double Dd = (double)lii * (double)lii;
      Dv[i] = Dd;
      logD[i] = log(Dd);
    }
  }
  // ---- row of [F z]: 16-byte vectors along k
  for (int k = lane * V; k < fpad; k += 32 * V) {
    T out[V];
    if (k < mpad) {
      T a[V];
      vget(*reinterpret_cast<const VT*>(A + (size_t)i * mpad + k), a);
#pragma unroll
      for (int e = 0; e < V; ++e) out[e] = a[e];
      if constexpr (QM <= 28) {
        // unrolled so that every neighbour row is requested before the first is used
#pragma unroll
        for (int t = 0; t < QM - 1; ++t) {
          if (t < q) {
            const T ct = S.coef[t];
            vget(*reinterpret_cast<const VT*>(A + (size_t)S.idx[t] * mpad + k), a);
#pragma unroll
            for (int e = 0; e < V; ++e) out[e] -= ct * a[e];
          }
        }
      } else {
        for (int t = 0; t < q; ++t) {
          const T ct = S.coef[t];
          vget(*reinterpret_cast<const VT*>(A + (size_t)S.idx[t] * mpad + k), a);
#pragma unroll
          for (int e = 0; e < V; ++e) out[e] -= ct * a[e];
        }
      }
#pragma unroll
      for (int e = 0; e < V; ++e) out[e] *= inv;
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) out[e] = T(0);
    }
    VT ov;
    if constexpr (V == 4) ov = make_float4(out[0], out[1], out[2], out[3]);
    else ov = make_double2(out[0], out[1]);
    *reinterpret_cast<VT*>(F + (size_t)i * fpad + k) = ov;
  }
  __syncwarp();
  // z_i = (y_i - sum_t A_i[t] y_{N_t}) / sqrt(D_i) in float64: one product per lane and a
  // shuffle tree (a few warp-wide float64 instructions instead of q serial ones)
  double zt = (lane < q) ? -(double)S.coef[lane] * y[S.idx[lane]] : 0.0;
  if (q > 32)
    for (int t = lane + 32; t < q; t += 32) zt -= (double)S.coef[t] * y[S.idx[t]];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) zt += __shfl_xor_sync(0xffffffffu, zt, off);
  if (lane == 0) F[(size_t)i * fpad + m] = (T)((y[i] + zt) * (double)inv);
}

// float32 m_v = 20 (R = 3): six CTAs of four warps per SM, as the shared memory allows
template <typename T, int R, bool GS>
__global__ __launch_bounds__(FK_WARPS * 32) void factor_kernel(
    const T* __restrict__ A, const T* __restrict__ Xs, const int32_t* __restrict__ N,
    const int32_t* __restrict__ order, const double* __restrict__ y, int64_t n, int d, int m, int mpad, int mv,
    int fpad, CovParams cp, T* __restrict__ F, double* __restrict__ Acoef, double* __restrict__ Dv,
    double* __restrict__ logD, int* status, const float* __restrict__ gsub, float* __restrict__ rho) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int w = threadIdx.x >> 5;
  const int64_t slot = (int64_t)blockIdx.x * FK_WARPS + w;
  if (slot >= n) return;
  factor_point<T, R, GS>(A, Xs, N, order, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, status, gsub, rho,
                         slot, reinterpret_cast<FactorSmem<T, R, GS>*>(smraw)[w]);
}

// Many problems' factors in one persistent launch (the batched likelihoods): the points of
// all jobs of one block size R form one list (job p owns positions off[p] .. off[p+1]); each
// warp takes the next 32 positions from a device work queue and factors them one by one.
// one point of a job, compiled on its own: inlined into the work loop, the float32 kernels
// for R >= 5 kept part of their register arrays in local memory
template <typename T, int R>
__device__ __noinline__ void factor_job_point(const FactorJob<T>* __restrict__ J, int64_t slot,
                                              FactorSmem<T, R, false>* S) {
  factor_point<T, R, false>(J->A, J->Xs, J->N, J->order, J->y, J->n, J->d, J->m, J->mpad, J->mv, J->fpad, J->cp,
                            J->F, J->Acoef, J->Dv, J->logD, J->status, nullptr, nullptr, slot, *S);
}

template <typename T, int R>
__global__ __launch_bounds__(FK_WARPS * 32) void factor_batched_kernel(const FactorJob<T>* __restrict__ jobs,
                                                                       const int64_t* __restrict__ off, int njobs,
                                                                       unsigned long long* __restrict__ queue) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto& S = reinterpret_cast<FactorSmem<T, R, false>*>(smraw)[w];
  const int64_t total = off[njobs];
  constexpr int CHUNK = 32;
  // one loop level: a fresh chunk whenever the warp's current one is used up
  int64_t g = 0, end = 0;
  int p = 0;
#pragma unroll 1
  for (;;) {
    if (g == end) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(queue, (unsigned long long)CHUNK);
      base = __shfl_sync(0xffffffffu, base, 0);
      if ((int64_t)base >= total) break;
      g = (int64_t)base;
      end = min(total, g + CHUNK);
      int hi = njobs;                                 // the job of the chunk's first position
      p = 0;
      while (hi - p > 1) {
        const int mid = (p + hi) >> 1;
        if (off[mid] <= g) p = mid;
        else hi = mid;
      }
    }
    while (p + 1 < njobs && off[p + 1] <= g) ++p;     // positions ascend: the job only moves forward
    factor_job_point<T, R>(jobs + p, g - off[p], &S);
    __syncwarp();
    ++g;
  }
}

static_assert(FK_WARPS == FT_BLOCK_POINTS, "table block offsets count blocks of FK_WARPS points");
static_assert(sizeof(FactorTable<float>) <= 32764 && sizeof(FactorTable<double>) <= 32764,
              "a factor table must fit the 32764-byte kernel parameter limit");
// the job records in the parameter bank: block b of the launch serves job p with
// boff[p] <= b < boff[p + 1], so p and the job's fields are the same for the whole block
template <typename T, int R>
__global__ __launch_bounds__(FK_WARPS * 32) void factor_table_kernel(const __grid_constant__ FactorTable<T> tab) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int w = threadIdx.x >> 5;
  auto& S = reinterpret_cast<FactorSmem<T, R, false>*>(smraw)[w];
  const int b = (int)blockIdx.x;
  int p = 0, hi = tab.njobs;
  while (hi - p > 1) {
    const int mid = (p + hi) >> 1;
    if (tab.boff[mid] <= b) p = mid;
    else hi = mid;
  }
  const FactorJob<T>& J = tab.job[p];
  const int64_t slot = (int64_t)(b - tab.boff[p]) * FK_WARPS + w;
  if (slot >= J.n) return;
  factor_point<T, R, false>(J.A, J.Xs, J.N, J.order, J.y, J.n, J.d, J.m, J.mpad, J.mv, J.fpad, J.cp, J.F, J.Acoef,
                            J.Dv, J.logD, J.status, nullptr, nullptr, slot, S);
}
template <typename T, int R>
static cudaError_t launch_factor_table(const FactorTable<T>& tab, cudaStream_t s) {
  const size_t smem = sizeof(FactorSmem<T, R, false>) * FK_WARPS;
  cudaError_t e = cudaFuncSetAttribute(factor_table_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  factor_table_kernel<T, R><<<(unsigned)tab.boff[tab.njobs], FK_WARPS * 32, smem, s>>>(tab);
  return cudaGetLastError();
}

template <typename T, int R, bool GS>
static cudaError_t launch_factor(const T* A, const T* Xs, const int32_t* N, const int32_t* order, const double* y,
                                 int64_t n, int d, int m, int mpad, int mv, int fpad, CovParams cp, T* F,
                                 double* Acoef, double* Dv, double* logD, int* status, cudaStream_t s,
                                 const float* gsub, float* rho) {
  size_t smem = sizeof(FactorSmem<T, R, GS>) * FK_WARPS;
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<T, R, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = (unsigned)((n + FK_WARPS - 1) / FK_WARPS);
  factor_kernel<T, R, GS><<<grid, FK_WARPS * 32, smem, s>>>(A, Xs, N, order, y, n, d, m, mpad, mv, fpad, cp, F,
                                                             Acoef, Dv, logD, status, gsub, rho);
  return cudaGetLastError();
}

template <typename T>
cudaError_t vecchia_factor_gs(const T* A, const T* Xs, const int32_t* N, const int32_t* order, const double* y,
                              int64_t n, int d, int m, int mpad, int mv, int fpad, CovParams cp, T* F,
                              double* Acoef, double* Dv, double* logD, int* status, cudaStream_t s,
                              const float* gsub, float* rho) {
  if (d > FK_MAXD) return cudaErrorInvalidValue;
  const int Q = mv + 1;
  if (gsub) {
    // the Gram of each point's rows comes from the tensor cores (float32, Q <= 32)
    if constexpr (sizeof(T) == 4) {
#define LG(RR) launch_factor<T, RR, true>(A, Xs, N, order, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, \
                                          status, s, gsub, rho)
      if (Q <= 14) return LG(2);
      if (Q <= 21) return LG(3);
      if (Q <= 28) return LG(4);
      if (Q <= 32) return LG(5);
#undef LG
    }
    return cudaErrorInvalidValue;
  }
#define LF(RR) launch_factor<T, RR, false>(A, Xs, N, order, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, \
                                           status, s, nullptr, rho)
  if (Q <= 14) return LF(2);
  if (Q <= 21) return LF(3);
  if (Q <= 28) return LF(4);
  if (Q <= 35) return LF(5);
  if (Q <= 42) return LF(6);
  if (Q <= 49) return LF(7);
#undef LF
  return cudaErrorInvalidValue;
}

template <typename T, int R>
static cudaError_t launch_factor_batched(const FactorJob<T>* jobs, const int64_t* off, int njobs,
                                         unsigned long long* queue, int nsm, cudaStream_t s) {
  const size_t smem = sizeof(FactorSmem<T, R, false>) * FK_WARPS;
  cudaError_t e = cudaFuncSetAttribute(factor_batched_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_batched_kernel<T, R>, FK_WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  factor_batched_kernel<T, R><<<(unsigned)(std::max(per_sm, 1) * std::max(nsm, 1)), FK_WARPS * 32, smem, s>>>(
      jobs, off, njobs, queue);
  return cudaGetLastError();
}

template <typename T>
cudaError_t vecchia_factor_batched(const FactorJob<T>* jobs, const int64_t* off, int njobs, int mv_max,
                                   unsigned long long* queue, int nsm, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  const int Q = mv_max + 1;
  if (Q <= 14) return launch_factor_batched<T, 2>(jobs, off, njobs, queue, nsm, s);
  if (Q <= 21) return launch_factor_batched<T, 3>(jobs, off, njobs, queue, nsm, s);
  if (Q <= 28) return launch_factor_batched<T, 4>(jobs, off, njobs, queue, nsm, s);
  if (Q <= 35) return launch_factor_batched<T, 5>(jobs, off, njobs, queue, nsm, s);
  if (Q <= 42) return launch_factor_batched<T, 6>(jobs, off, njobs, queue, nsm, s);
  if (Q <= 49) return launch_factor_batched<T, 7>(jobs, off, njobs, queue, nsm, s);
  return cudaErrorInvalidValue;
}
template cudaError_t vecchia_factor_batched<float>(const FactorJob<float>*, const int64_t*, int, int,
                                                   unsigned long long*, int, cudaStream_t);

template <typename T>
cudaError_t vecchia_factor_table(const FactorTable<T>& tab, int mv_max, cudaStream_t s) {
  if (tab.njobs <= 0 || tab.njobs > FT_MAXJ || tab.boff[tab.njobs] <= 0) return cudaSuccess;
  const int Q = mv_max + 1;
  if (Q <= 14) return launch_factor_table<T, 2>(tab, s);
  if (Q <= 21) return launch_factor_table<T, 3>(tab, s);
  if (Q <= 28) return launch_factor_table<T, 4>(tab, s);
  if (Q <= 35) return launch_factor_table<T, 5>(tab, s);
  if (Q <= 42) return launch_factor_table<T, 6>(tab, s);
  if (Q <= 49) return launch_factor_table<T, 7>(tab, s);
  return cudaErrorInvalidValue;
}
template cudaError_t vecchia_factor_table<float>(const FactorTable<float>&, int, cudaStream_t);
template cudaError_t vecchia_factor_table<double>(const FactorTable<double>&, int, cudaStream_t);
template cudaError_t vecchia_factor_batched<double>(const FactorJob<double>*, const int64_t*, int, int,
                                                    unsigned long long*, int, cudaStream_t);

template <typename T>
cudaError_t vecchia_factor(const T* A, const T* Xs, const int32_t* N, const int32_t* order, const double* y,
                           int64_t n, int d, int m, int mpad, int mv, int fpad, CovParams cp, T* F, double* Acoef,
                           double* Dv, double* logD, int* status, cudaStream_t s) {
  return vecchia_factor_gs<T>(A, Xs, N, order, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, status, s,
                              nullptr, nullptr);
}
template cudaError_t vecchia_factor_gs<float>(const float*, const float*, const int32_t*, const int32_t*,
                                              const double*, int64_t, int, int, int, int, int, CovParams, float*,
                                              double*, double*, double*, int*, cudaStream_t, const float*, float*);
template cudaError_t vecchia_factor_gs<double>(const double*, const double*, const int32_t*, const int32_t*,
                                               const double*, int64_t, int, int, int, int, int, CovParams,
                                               double*, double*, double*, double*, int*, cudaStream_t,
                                               const float*, float*);
template cudaError_t vecchia_factor<float>(const float*, const float*, const int32_t*, const int32_t*,
                                           const double*, int64_t, int, int, int, int, int, CovParams, float*,
                                           double*, double*, double*, int*, cudaStream_t);
template cudaError_t vecchia_factor<double>(const double*, const double*, const int32_t*, const int32_t*,
                                            const double*, int64_t, int, int, int, int, int, CovParams, double*,
                                            double*, double*, double*, int*, cudaStream_t);

// ---------------------------------------------------------------------------
// G' = [F z]^T [F z]: split-K SYRK.  CTA = one 64 x 64 tile pair (ti >= tj) and
// one contiguous slice of rows; float32 accumulation is flushed into float64
// every 256 rows; slices are summed in float64 in a fixed order.
// ---------------------------------------------------------------------------
constexpr int GT = 64;
constexpr int GR = 16;

template <typename T>
__global__ __launch_bounds__(256) void gram_kernel(const T* __restrict__ F, int64_t n, int fpad, double* part,
                                                   int nsplit, const double* __restrict__ wrow) {
  const int p = blockIdx.x;
  int ti = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= p) ++ti;
  while (ti * (ti + 1) / 2 > p) --ti;
  const int tj = p - ti * (ti + 1) / 2;
  const int npairs = gridDim.x;
  const int sidx = blockIdx.y;
  const int64_t chunk = (n + nsplit - 1) / nsplit;
  const int64_t r0 = (int64_t)sidx * chunk, r1 = (n < r0 + chunk) ? n : r0 + chunk;
  __shared__ __align__(16) T Fi[GR][GT + 4];
  __shared__ __align__(16) T Fj[GR][GT + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      acc[u][v] = T(0);
      dacc[u][v] = 0.0;
    }
  int flush = 0;
  for (int64_t r = r0; r < r1; r += GR) {
    __syncthreads();
    for (int e = threadIdx.x; e < GR * GT; e += 256) {
      int rr = e / GT, c = e % GT;
      int64_t row = r + rr;
      bool ok = row < r1;
      Fi[rr][c] = ok ? (wrow ? (T)wrow[row] : T(1)) * F[(size_t)row * fpad + ti * GT + c] : T(0);
      Fj[rr][c] = ok ? F[(size_t)row * fpad + tj * GT + c] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < GR; ++rr) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Fi[rr][ty * 4 + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Fj[rr][tx * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    if (++flush == 16) {
      flush = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          dacc[u][v] += (double)acc[u][v];
          acc[u][v] = T(0);
        }
    }
  }
  double* out = part + ((size_t)sidx * npairs + p) * GT * GT;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(ty * 4 + u) * GT + tx * 4 + v] = dacc[u][v] + (double)acc[u][v];
}

__global__ void gram_reduce_kernel(const double* part, int nsplit, int npairs, int m, double* G, int ldg) {
  const int M1 = m + 1;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M1 * M1) return;
  int a = (int)(e / M1), b = (int)(e % M1);
  if (b > a) return;
  int ti = a / GT, tj = b / GT;
  int p = ti * (ti + 1) / 2 + tj;
  size_t off = (size_t)p * GT * GT + (size_t)(a % GT) * GT + (b % GT);
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * npairs * GT * GT + off];
  if (a == b && a < m) s += 1.0;
  G[(size_t)a * ldg + b] = s;
}

int gram_nsplit(int64_t n, int fpad) {
  // row slices of the Gram: about four CTAs per SM counted in 128-wide tile pairs; the
  // float32 tensor-core Gram uses at most this many, the float64 one exactly this many
  int nt = (fpad + 127) / 128;
  int npairs = nt * (nt + 1) / 2;
  int64_t want = (4 * 152 + npairs - 1) / npairs;
  int64_t maxs = (n + 255) / 256;
  int64_t s = want < maxs ? want : maxs;
  return (int)(s < 1 ? 1 : s);
}

template <typename T>
cudaError_t gram_FtF(const T* F, int64_t n, int fpad, int m, double* part, int nsplit, double* G, int ldg,
                     cudaStream_t s, const double* wrow, int* status) {
  int nt = fpad / GT;
  int npairs = nt * (nt + 1) / 2;
  if (sizeof(T) == 4 && wrow) return cudaErrorInvalidValue;   // row weights: float64 path only
  if constexpr (sizeof(T) == 4) {
    // tensor cores; one wave of slices, never more than the partial buffer holds
    const int nst = std::min(nsplit, gram_tc_nsplit(n, fpad));
    cudaError_t e = gram_tc(F, n, fpad, part, nst, status, s);
    if (e != cudaSuccess) return e;
    nsplit = nst;
  } else {
    gram_kernel<T><<<dim3(npairs, nsplit), 256, 0, s>>>(F, n, fpad, part, nsplit, wrow);
  }
  int64_t tot = (int64_t)(m + 1) * (m + 1);
  gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, nsplit, npairs, m, G, ldg);
  return cudaGetLastError();
}
template cudaError_t gram_FtF<float>(const float*, int64_t, int, int, double*, int, double*, int, cudaStream_t,
                                     const double*, int*);
template cudaError_t gram_FtF<double>(const double*, int64_t, int, int, double*, int, double*, int, cudaStream_t,
                                      const double*, int*);

// NLL = 1/2 [ n log 2pi + sum_{k<m} 2 log L'_kk + sum_i log D_i + L'_mm^2 ],  L' = chol(G').
__global__ void nll_finish_kernel(const double* Lg, int ldg, int m, const double* logD_sum, int64_t n,
                                  double* out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) v += 2.0 * log(Lg[(size_t)k * ldg + k]);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w2 = 128; w2 > 0; w2 >>= 1) {
    if (threadIdx.x < w2) sh[threadIdx.x] += sh[threadIdx.x + w2];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double lmm = Lg[(size_t)m * ldg + m];
    const double log2pi = 1.8378770664093454836;
    out[0] = 0.5 * ((double)n * log2pi + sh[0] + *logD_sum + lmm * lmm);
    out[1] = sh[0];          // log det C
    out[2] = lmm * lmm;      // y^T Sigma~_dagger^{-1} y
  }
}

cudaError_t nll_finish(const double* Lg, int ldg, int m, const double* logD_sum, int64_t n, double* out,
                       cudaStream_t s) {
  nll_finish_kernel<<<1, 256, 0, s>>>(Lg, ldg, m, logD_sum, n, out);
  return cudaGetLastError();
}

}  // namespace vif
