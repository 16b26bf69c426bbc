// Low-rank part of the VIF approximation (Sec. 2.1, Eq. def_b_low):
//   Sigma_m (m x m, with jitter), L_m = chol(Sigma_m), A = L_m^{-1} Sigma_mn,
// so that Sigma^l = Sigma_mn^T Sigma_m^{-1} Sigma_mn = A^T A.
//
// A is stored point-major (n x mpad, row i = a_i), the layout every later step
// gathers from.  It is computed as A = K_nm L_m^{-T}: a GEMM whose left operand
// (the kernel matrix) is generated on the fly from the scaled coordinates and
// never stored, and whose right operand L_m^{-T} is upper triangular, so the
// k-loop of every output column stops at that column.
#include "vif_internal.cuh"

namespace vif {

__global__ void scale_coords_kernel(const double* X, int64_t n, int d, const double* inv_ls,
                                    const double* center, double* Xs, float* Xs32) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * d) return;
  int t = (int)(e % d);
  double v = (X[e] - center[t]) * inv_ls[t];
  if (Xs) Xs[e] = v;
  if (Xs32) Xs32[e] = (float)v;
}

cudaError_t scale_coords(const double* X, int64_t n, int d, const double* inv_ls, const double* center,
                         double* Xs, float* Xs32, cudaStream_t s) {
  int64_t tot = n * d;
  if (tot == 0) return cudaSuccess;
  scale_coords_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, d, inv_ls, center, Xs, Xs32);
  return cudaGetLastError();
}

__global__ void sigma_m_kernel(const double* Zs, int m, int d, CovParams cp, double* Sm, int lda) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  int a = (int)(e / m), b = (int)(e % m);
  double v = cov_r2<double>(sqdist(Zs + (size_t)a * d, Zs + (size_t)b * d, d), cp.kind, cp.var);
  if (a == b) v += cp.jitter;
  Sm[(size_t)a * lda + b] = v;
}

cudaError_t build_sigma_m(const double* Zs, int m, int d, CovParams cp, double* Sm, int lda,
                          cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  int64_t tot = (int64_t)m * m;
  sigma_m_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Zs, m, d, cp, Sm, lda);
  return cudaGetLastError();
}

template <typename T>
__global__ void linv_transpose_kernel(const double* Linv, int m, int lda, T* LinvT, int ldt) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ldt * ldt) return;
  int c = (int)(e / ldt), r = (int)(e % ldt);   // LinvT[c][r] = Linv[r][c]
  double v = (r < m && c < m && c <= r) ? Linv[(size_t)r * lda + c] : 0.0;
  LinvT[e] = (T)v;
}

template <typename T>
cudaError_t linv_transpose(const double* Linv, int m, int lda, T* LinvT, int ldt, cudaStream_t s) {
  int64_t tot = (int64_t)ldt * ldt;
  linv_transpose_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Linv, m, lda, LinvT, ldt);
  return cudaGetLastError();
}
template cudaError_t linv_transpose<float>(const double*, int, int, float*, int, cudaStream_t);
template cudaError_t linv_transpose<double>(const double*, int, int, double*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// A = K_nm L^{-T}.  CTA: 32 points x one pass of 512 output columns; thread
// (rg, cg) owns rows rg*8..rg*8+7 and columns cg + 64 j (j < 8), so every thread
// meets the triangular skip at the same rate.  K chunks are evaluated once per
// pass into shared memory.
// ---------------------------------------------------------------------------
constexpr int LR_BP = 32;      // points per CTA
constexpr int LR_PASS = 512;   // output columns per pass
constexpr int LR_MAXD = 16;

template <typename T>
__global__ __launch_bounds__(256) void lowrank_A_kernel(const T* __restrict__ Xs, const T* __restrict__ Zs,
                                                        const T* __restrict__ LinvT, int ldt, T* __restrict__ A,
                                                        int64_t n, int d, int m, int mpad, int kind, T var) {
  constexpr int BK = 64 / sizeof(T);  // 16 (float) or 8 (double): 32 KB of L^{-T} per chunk
  __shared__ T xs[LR_BP * LR_MAXD];
  __shared__ T zs[BK * LR_MAXD];
  __shared__ T Ks[LR_BP][BK + 1];
  __shared__ T Ls[BK][LR_PASS];
  const int64_t p0 = (int64_t)blockIdx.x * LR_BP;
  const int tid = threadIdx.x, cg = tid & 63, rg = tid >> 6;
  for (int e = tid; e < LR_BP * d; e += 256) {
    int64_t pi = p0 + e / d;
    xs[e] = (pi < n) ? Xs[(size_t)p0 * d + e] : T(0);
  }
  for (int base = 0; base < mpad; base += LR_PASS) {
    T acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[r][j] = T(0);
    const int cend = min(m, base + LR_PASS);
    for (int c0 = 0; c0 < cend; c0 += BK) {
      __syncthreads();
      for (int e = tid; e < BK * d; e += 256) {
        int c = c0 + e / d;
        zs[e] = (c < m) ? Zs[(size_t)c0 * d + e] : T(0);
      }
      for (int e = tid; e < BK * LR_PASS; e += 256) {
        int kk = e / LR_PASS, rr = e % LR_PASS;
        int c = c0 + kk, r = base + rr;
        Ls[kk][rr] = (c < m && r < ldt) ? LinvT[(size_t)c * ldt + r] : T(0);
      }
      __syncthreads();
      for (int e = tid; e < LR_BP * BK; e += 256) {
        int pi = e / BK, kk = e % BK;
        int c = c0 + kk;
        T v = T(0);
        if (c < m && p0 + pi < n) v = cov_r2<T>(sqdist(xs + pi * d, zs + kk * d, d), kind, var);
        Ks[pi][kk] = v;
      }
      __syncthreads();
#pragma unroll 2
      for (int kk = 0; kk < BK; ++kk) {
        T kv[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) kv[r] = Ks[rg * 8 + r][kk];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (base + 64 * j + 63 >= c0) {   // warp-uniform: L^{-T}[c][col] = 0 for c > col
            T lv = Ls[kk][cg + 64 * j];
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r][j] += kv[r] * lv;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      int64_t pi = p0 + rg * 8 + r;
      if (pi >= n) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int col = base + cg + 64 * j;
        if (col < mpad) A[(size_t)pi * mpad + col] = acc[r][j];
      }
    }
  }
}

template <typename T>
cudaError_t lowrank_A(const T* Xs, const T* Zs, const T* LinvT, int ldt, T* A, int64_t n, int d, int m,
                      int mpad, int kind, double var, cudaStream_t s) {
  if (m <= 0) return cudaMemsetAsync(A, 0, sizeof(T) * (size_t)n * mpad, s);
  if (d > LR_MAXD) return cudaErrorInvalidValue;
  unsigned grid = (unsigned)((n + LR_BP - 1) / LR_BP);
  lowrank_A_kernel<T><<<grid, 256, 0, s>>>(Xs, Zs, LinvT, ldt, A, n, d, m, mpad, kind, (T)var);
  return cudaGetLastError();
}
template cudaError_t lowrank_A<double>(const double*, const double*, const double*, int, double*, int64_t, int,
                                       int, int, int, double, cudaStream_t);

// ---------------------------------------------------------------------------
// Per-point quantities of the neighbour search (Sec. 6): residual variance
// c_r(i,i) = sigma1^2 - ||a_i||^2 in float64, the float32 copy of a_i, its norm
// rounded up, and 1/sqrt(c_r(i,i)) (0 when c_r(i,i) <= tau, where the
// correlation is taken as 0).
// ---------------------------------------------------------------------------
__global__ void residual_diag_kernel(const double* A, int64_t n, int m, int mpad, double var, double tau,
                                     float* A32, double* cii, float* rs32, float* nrm32) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s64 = 0.0, s32 = 0.0;
  for (int k = lane; k < mpad; k += 32) {
    double a = A[(size_t)i * mpad + k];
    float af = (float)a;
    A32[(size_t)i * mpad + k] = af;
    s64 += a * a;
    s32 += (double)af * (double)af;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s64 += __shfl_xor_sync(0xffffffffu, s64, o);
    s32 += __shfl_xor_sync(0xffffffffu, s32, o);
  }
  if (lane == 0) {
    double c = var - s64;
    cii[i] = c;
    rs32[i] = (c > tau) ? (float)(1.0 / sqrt(c)) : 0.0f;
    nrm32[i] = (float)(sqrt(s32) * (1.0 + 1e-6));
  }
}

cudaError_t residual_diag_stats(const double* A, int64_t n, int m, int mpad, double var, double tau,
                                float* A32, double* cii, float* rs32, float* nrm32, cudaStream_t s) {
  unsigned grid = (unsigned)((n + 7) / 8);
  residual_diag_kernel<<<grid, 256, 0, s>>>(A, n, m, mpad, var, tau, A32, cii, rs32, nrm32);
  return cudaGetLastError();
}

}  // namespace vif
