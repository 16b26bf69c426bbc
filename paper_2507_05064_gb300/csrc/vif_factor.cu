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
#include "vif_internal.cuh"

namespace vif {

// ---------------------------------------------------------------------------
// Factor kernel: one warp per point.  Lane l < 21 owns the R x R block (bi, bj),
// bj <= bi < 6, of the (6R) x (6R) padded Gram [A_N; a_i][A_N; a_i]^T; the rows
// are staged through shared memory 32 columns at a time.
// ---------------------------------------------------------------------------
constexpr int FK_KC = 32;
constexpr int FK_WARPS = 4;
constexpr int FK_MAXD = 16;

__constant__ unsigned char c_blk_i[21] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5};
__constant__ unsigned char c_blk_j[21] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};

template <typename T, int R>
struct FactorSmem {
  static constexpr int QM = 6 * R;
  T buf[QM][FK_KC + 1];
  T G[QM][QM + 1];
  T coef[QM];
  T xc[QM][FK_MAXD];
  int idx[QM];
};

template <typename T, int R>
__global__ __launch_bounds__(FK_WARPS * 32) void factor_kernel(
    const T* __restrict__ A, const T* __restrict__ Xs, const int32_t* __restrict__ N,
    const double* __restrict__ y, int64_t n, int d, int m, int mpad, int mv, int fpad, CovParams cp,
    T* __restrict__ F, double* __restrict__ Acoef, double* __restrict__ Dv, double* __restrict__ logD,
    int* status) {
  constexpr int QM = 6 * R;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  FactorSmem<T, R>& S = reinterpret_cast<FactorSmem<T, R>*>(smraw)[w];
  const int64_t i = (int64_t)blockIdx.x * FK_WARPS + w;
  if (i >= n) return;
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
  for (int e = lane; e < QM * (FK_KC + 1); e += 32) (&S.buf[0][0])[e] = T(0);
  __syncwarp();
  for (int e = lane; e < Q * d; e += 32) {
    int t = e / d, c = e % d;
    S.xc[t][c] = Xs[(size_t)S.idx[t] * d + c];
  }
  // ---- Gram of the gathered rows of A
  const bool owner = lane < 21;
  const int bi = owner ? c_blk_i[lane] : 0, bj = owner ? c_blk_j[lane] : 0;
  T acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = T(0);
  for (int k0 = 0; k0 < m; k0 += FK_KC) {
    for (int t = 0; t < Q; ++t) {
      int k = k0 + lane;
      S.buf[t][lane] = (k < mpad) ? A[(size_t)S.idx[t] * mpad + k] : T(0);
    }
    __syncwarp();
    if (owner) {
#pragma unroll 4
      for (int kk = 0; kk < FK_KC; ++kk) {
        T u[R], v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = S.buf[bi * R + r][kk];
#pragma unroll
        for (int c = 0; c < R; ++c) v[c] = S.buf[bj * R + c][kk];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < R; ++c) acc[r][c] += u[r] * v[c];
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
  // ---- residual covariance R (lower triangle)
  const int npair = Q * (Q + 1) / 2;
  for (int e = lane; e < npair; e += 32) {
    int a = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    while (a * (a + 1) / 2 > e) --a;
    int b = e - a * (a + 1) / 2;
    T kv = cov_r2<T>(sqdist(&S.xc[a][0], &S.xc[b][0], d), cp.kind, (T)cp.var);
    if (a == b) kv += (T)cp.tdiag;
    S.G[a][b] = kv - S.G[a][b];
  }
  __syncwarp();
  // ---- Cholesky of R (lower, in place)
  for (int c = 0; c < Q; ++c) {
    T piv = S.G[c][c];
    bool bad = !(piv > T(0));
    if (bad) {
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
  const T lii = S.G[q][q];
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
  const double Dd = (double)lii * (double)lii;
  for (int t = lane; t < mv; t += 32) Acoef[(size_t)i * mv + t] = (t < q) ? (double)S.coef[t] : 0.0;
  if (lane == 0) {
    Dv[i] = Dd;
    logD[i] = log(Dd);
  }
  // ---- row of [F z]
  const T inv = T(1) / lii;
  for (int k = lane; k < fpad; k += 32) {
    T v;
    if (k < m) {
      v = A[(size_t)i * mpad + k];
      for (int t = 0; t < q; ++t) v -= S.coef[t] * A[(size_t)S.idx[t] * mpad + k];
      v *= inv;
    } else if (k == m) {
      double zz = y[i];
      for (int t = 0; t < q; ++t) zz -= (double)S.coef[t] * y[S.idx[t]];
      v = (T)(zz * (double)inv);
    } else {
      v = T(0);
    }
    F[(size_t)i * fpad + k] = v;
  }
}

template <typename T, int R>
static cudaError_t launch_factor(const T* A, const T* Xs, const int32_t* N, const double* y, int64_t n, int d,
                                 int m, int mpad, int mv, int fpad, CovParams cp, T* F, double* Acoef,
                                 double* Dv, double* logD, int* status, cudaStream_t s) {
  size_t smem = sizeof(FactorSmem<T, R>) * FK_WARPS;
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = (unsigned)((n + FK_WARPS - 1) / FK_WARPS);
  factor_kernel<T, R><<<grid, FK_WARPS * 32, smem, s>>>(A, Xs, N, y, n, d, m, mpad, mv, fpad, cp, F, Acoef,
                                                         Dv, logD, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t vecchia_factor(const T* A, const T* Xs, const int32_t* N, const double* y, int64_t n, int d, int m,
                           int mpad, int mv, int fpad, CovParams cp, T* F, double* Acoef, double* Dv,
                           double* logD, int* status, cudaStream_t s) {
  if (d > FK_MAXD) return cudaErrorInvalidValue;
  const int Q = mv + 1;
  if (Q <= 12) return launch_factor<T, 2>(A, Xs, N, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, status, s);
  if (Q <= 24) return launch_factor<T, 4>(A, Xs, N, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, status, s);
  if (Q <= 36) return launch_factor<T, 6>(A, Xs, N, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, status, s);
  if (Q <= 48) return launch_factor<T, 8>(A, Xs, N, y, n, d, m, mpad, mv, fpad, cp, F, Acoef, Dv, logD, status, s);
  return cudaErrorInvalidValue;
}
template cudaError_t vecchia_factor<float>(const float*, const float*, const int32_t*, const double*, int64_t, int,
                                           int, int, int, int, CovParams, float*, double*, double*, double*, int*,
                                           cudaStream_t);
template cudaError_t vecchia_factor<double>(const double*, const double*, const int32_t*, const double*, int64_t,
                                            int, int, int, int, int, CovParams, double*, double*, double*, double*,
                                            int*, cudaStream_t);

// ---------------------------------------------------------------------------
// G' = [F z]^T [F z]: split-K SYRK.  CTA = one 64 x 64 tile pair (ti >= tj) and
// one contiguous slice of rows; float32 accumulation is flushed into float64
// every 256 rows; slices are summed in float64 in a fixed order.
// ---------------------------------------------------------------------------
constexpr int GT = 64;
constexpr int GR = 16;

template <typename T>
__global__ __launch_bounds__(256) void gram_kernel(const T* __restrict__ F, int64_t n, int fpad, double* part,
                                                   int nsplit) {
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
      Fi[rr][c] = ok ? F[(size_t)row * fpad + ti * GT + c] : T(0);
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
  int nt = fpad / GT;
  int npairs = nt * (nt + 1) / 2;
  int64_t want = (4 * 152 + npairs - 1) / npairs;
  int64_t maxs = (n + 255) / 256;
  int64_t s = want < maxs ? want : maxs;
  return (int)(s < 1 ? 1 : s);
}

template <typename T>
cudaError_t gram_FtF(const T* F, int64_t n, int fpad, int m, double* part, int nsplit, double* G, int ldg,
                     cudaStream_t s) {
  int nt = fpad / GT;
  int npairs = nt * (nt + 1) / 2;
  gram_kernel<T><<<dim3(npairs, nsplit), 256, 0, s>>>(F, n, fpad, part, nsplit);
  int64_t tot = (int64_t)(m + 1) * (m + 1);
  gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, nsplit, npairs, m, G, ldg);
  return cudaGetLastError();
}
template cudaError_t gram_FtF<float>(const float*, int64_t, int, int, double*, int, double*, int, cudaStream_t);
template cudaError_t gram_FtF<double>(const double*, int64_t, int, int, double*, int, double*, int, cudaStream_t);

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
