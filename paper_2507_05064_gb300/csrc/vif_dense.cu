// float64 dense linear algebra for the m x m matrices of the method: the Cholesky
// factor of Sigma_m (Sec. 2.1) and of the capacitance matrix C = L_m^{-1} M L_m^{-T}
// (M of Eq. def_M, Sec. 2.2), and the inverse of the lower factor L_m.
//
// GB300 executes float64 at ~1/60 of its float32 rate (about 2 DFMA per clock per
// SM), so a single-CTA factorisation of m = 500 would take ~10 ms.  The blocked
// right-looking algorithm below spreads every step over many CTAs: one launch
// factors the 32 x 32 diagonal tile (redundantly in every CTA) and solves the
// tiles below it, the next updates the trailing tiles, one CTA per tile.
#include "vif_internal.cuh"

namespace vif {

constexpr int NB = 32;

__device__ __forceinline__ double ld_lower(const double* A, int lda, int m, int r, int c) {
  if (r < m && c < m) return A[(size_t)r * lda + c];
  return (r == c) ? 1.0 : 0.0;
}

// In-shared-memory Cholesky of a 32 x 32 tile (lower triangle), all threads.  The
// pivot's reciprocal is formed once per column (one float64 division) and the
// column is scaled by multiplication; rinv[c] keeps 1/L_cc for the caller.
__device__ void tile_potrf(double (*T)[NB + 1], double* rinv, int* status, int code, int base) {
  for (int c = 0; c < NB; ++c) {
    if (threadIdx.x == 0) {
      double p = T[c][c];
      if (!(p > 0.0) || !isfinite(p)) {
        if (status) flag_status(status, code, base + c);
        p = nan("");
      }
      const double sp = sqrt(p);
      T[c][c] = sp;
      rinv[c] = 1.0 / sp;
    }
    __syncthreads();
    const double ip = rinv[c];
    for (int r = c + 1 + threadIdx.x; r < NB; r += blockDim.x) T[r][c] *= ip;
    __syncthreads();
    int w = NB - c - 1;
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
      int r = c + 1 + idx / w, s2 = c + 1 + idx % w;
      if (s2 <= r) T[r][s2] -= T[r][c] * T[s2][c];
    }
    __syncthreads();
  }
}

// Inverse of the lower-triangular tile L (in smem) into X (lower), one warp per
// column block of lanes: column c of X solves L x = e_c.
__device__ void tile_trtri(const double (*L)[NB + 1], const double* rinv, double (*X)[NB + 1]) {
  if (threadIdx.x < NB) {
    const int c = threadIdx.x;
    for (int r = 0; r < NB; ++r) {
      if (r < c) {
        X[r][c] = 0.0;
        continue;
      }
      double v = (r == c) ? 1.0 : 0.0;
      double a0 = 0.0, a1 = 0.0;
      int s2 = c;
      for (; s2 + 1 < r; s2 += 2) {
        a0 += L[r][s2] * X[s2][c];
        a1 += L[r][s2 + 1] * X[s2 + 1][c];
      }
      if (s2 < r) a0 += L[r][s2] * X[s2][c];
      X[r][c] = (v - a0 - a1) * rinv[r];
    }
  }
  __syncthreads();
}

__global__ void chol_panel_kernel(double* A, int m, int lda, int k, int* status, int code) {
  __shared__ double Lk[NB][NB + 1];
  __shared__ double Li[NB][NB + 1];
  __shared__ double Tt[NB][NB + 1];
  __shared__ double rinv[NB];
  const int k0 = k * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    Lk[r][c] = (c <= r) ? ld_lower(A, lda, m, k0 + r, k0 + c) : 0.0;
  }
  __syncthreads();
  tile_potrf(Lk, rinv, blockIdx.x == 0 ? status : nullptr, code, k0);
  if (blockIdx.x == 0) {
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
      int r = idx / NB, c = idx % NB;
      if (k0 + r < m && k0 + c < m) A[(size_t)(k0 + r) * lda + k0 + c] = (c <= r) ? Lk[r][c] : 0.0;
    }
    return;
  }
  tile_trtri(Lk, rinv, Li);
  const int r0 = (k + blockIdx.x) * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    Tt[r][c] = ld_lower(A, lda, m, r0 + r, k0 + c);
  }
  __syncthreads();
  // X = T L_kk^{-T}: independent dot products X[r][c] = sum_{s<=c} T[r][s] Linv[c][s]
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    double a0 = 0.0, a1 = 0.0;
    int s2 = 0;
    for (; s2 + 1 <= c; s2 += 2) {
      a0 += Tt[r][s2] * Li[c][s2];
      a1 += Tt[r][s2 + 1] * Li[c][s2 + 1];
    }
    if (s2 <= c) a0 += Tt[r][s2] * Li[c][s2];
    if (r0 + r < m && k0 + c < m) A[(size_t)(r0 + r) * lda + k0 + c] = a0 + a1;
  }
}

__global__ void chol_update_kernel(double* A, int m, int lda, int k, int T) {
  // tile (i, j), k < j <= i < k+1+T, enumerated over the lower triangle
  int b = blockIdx.x;
  int ii = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((ii + 1) * (ii + 2) / 2 <= b) ++ii;
  while (ii * (ii + 1) / 2 > b) --ii;
  int jj = b - ii * (ii + 1) / 2;
  const int i0 = (k + 1 + ii) * NB, j0 = (k + 1 + jj) * NB, k0 = k * NB;
  __shared__ double Li[NB][NB + 1];
  __shared__ double Lj[NB][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    Li[r][c] = (i0 + r < m && k0 + c < m) ? A[(size_t)(i0 + r) * lda + k0 + c] : 0.0;
    Lj[r][c] = (j0 + r < m && k0 + c < m) ? A[(size_t)(j0 + r) * lda + k0 + c] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2] = {{0, 0}, {0, 0}};
#pragma unroll 8
  for (int c = 0; c < NB; ++c) {
    double a0 = Li[ty][c], a1 = Li[ty + 16][c];
    double b0 = Lj[tx][c], b1 = Lj[tx + 16][c];
    acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
    acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
  }
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) {
      int r = i0 + ty + 16 * u, c = j0 + tx + 16 * v;
      if (r < m && c < m && c <= r) A[(size_t)r * lda + c] -= acc[u][v];
    }
}

cudaError_t dense_cholesky(double* A, int m, int lda, int* status, int code, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int nt = (m + NB - 1) / NB;
  for (int k = 0; k < nt; ++k) {
    chol_panel_kernel<<<nt - k, 256, 0, s>>>(A, m, lda, k, status, code);
    int T = nt - k - 1;
    if (T > 0) chol_update_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(A, m, lda, k, T);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inverse of a lower-triangular L (blocked):  Linv_tt = L_tt^{-1};
// Linv_ij = -Linv_ii * sum_{k=j}^{i-1} L_ik Linv_kj, one block diagonal s = i - j at
// a time.  Within a step every tile product L_ik Linv_kj is its own CTA and adds
// into a per-(i,j) float64 tile with atomics, so a step costs two tile products of
// latency instead of s + 1.
// ---------------------------------------------------------------------------
__global__ void trtri_diag_kernel(const double* L, double* Li, int m, int lda) {
  __shared__ double Lt[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  __shared__ double rinv[NB];
  const int t0 = blockIdx.x * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    Lt[r][c] = (c <= r) ? ld_lower(L, lda, m, t0 + r, t0 + c) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < NB) rinv[threadIdx.x] = 1.0 / Lt[threadIdx.x][threadIdx.x];
  __syncthreads();
  tile_trtri(Lt, rinv, X);
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    if (t0 + r < m && t0 + c < m) Li[(size_t)(t0 + r) * lda + t0 + c] = X[r][c];
  }
}

__device__ void tile_prod_acc(const double (*P)[NB + 1], const double (*Q)[NB + 1], double acc[2][2], int tx,
                              int ty) {
#pragma unroll 8
  for (int c = 0; c < NB; ++c) {
    double a0 = P[ty][c], a1 = P[ty + 16][c];
    double b0 = Q[c][tx], b1 = Q[c][tx + 16];
    acc[0][0] += a0 * b0;
    acc[0][1] += a0 * b1;
    acc[1][0] += a1 * b0;
    acc[1][1] += a1 * b1;
  }
}

// tmp[j] += L_{j+s,k} Linv_{k,j},  k = j + kk,  CTA b = j * s + kk
__global__ void trtri_prod_kernel(const double* L, const double* Li, int m, int lda, int sdiag, double* tmp) {
  const int j = blockIdx.x / sdiag, kk = blockIdx.x % sdiag;
  const int i0 = (j + sdiag) * NB, j0 = j * NB, k0 = (j + kk) * NB;
  __shared__ double P[NB][NB + 1];
  __shared__ double Q[NB][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    P[r][c] = (i0 + r < m && k0 + c < m) ? L[(size_t)(i0 + r) * lda + k0 + c] : 0.0;
    Q[r][c] = (k0 + r < m && j0 + c < m) ? Li[(size_t)(k0 + r) * lda + j0 + c] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2] = {{0, 0}, {0, 0}};
  tile_prod_acc(P, Q, acc, tx, ty);
  double* T = tmp + (size_t)j * NB * NB;
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) atomicAdd(&T[(ty + 16 * u) * NB + tx + 16 * v], acc[u][v]);
}

// Linv_{j+s,j} = -Linv_{j+s,j+s} tmp[j]; tmp[j] is cleared for the next step.
__global__ void trtri_fin_kernel(double* Li, int m, int lda, int sdiag, double* tmp) {
  const int j = blockIdx.x, i0 = (j + sdiag) * NB, j0 = j * NB;
  __shared__ double P[NB][NB + 1];
  __shared__ double Q[NB][NB + 1];
  double* T = tmp + (size_t)j * NB * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    int r = idx / NB, c = idx % NB;
    P[r][c] = (i0 + r < m && i0 + c < m) ? Li[(size_t)(i0 + r) * lda + i0 + c] : 0.0;
    Q[r][c] = T[idx];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) T[idx] = 0.0;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2] = {{0, 0}, {0, 0}};
  tile_prod_acc(P, Q, acc, tx, ty);
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) {
      int r = ty + 16 * u, c = tx + 16 * v;
      if (i0 + r < m && j0 + c < m) Li[(size_t)(i0 + r) * lda + j0 + c] = -acc[u][v];
    }
}

size_t trtri_work_doubles(int m) { return (size_t)((m + NB - 1) / NB) * NB * NB; }

cudaError_t dense_trtri_lower(const double* L, double* Linv, int m, int lda, double* work, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int nt = (m + NB - 1) / NB;
  // zero the strictly upper part so consumers may read full tiles
  cudaError_t e = cudaMemset2DAsync(Linv, lda * sizeof(double), 0, m * sizeof(double), m, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(work, 0, trtri_work_doubles(m) * sizeof(double), s);
  if (e != cudaSuccess) return e;
  trtri_diag_kernel<<<nt, 64, 0, s>>>(L, Linv, m, lda);
  for (int sd = 1; sd < nt; ++sd) {
    trtri_prod_kernel<<<(nt - sd) * sd, 256, 0, s>>>(L, Linv, m, lda, sd, work);
    trtri_fin_kernel<<<nt - sd, 256, 0, s>>>(Linv, m, lda, sd, work);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic two-stage sum of n doubles.
// ---------------------------------------------------------------------------
constexpr int RED_BLOCKS = 256;

__global__ void reduce_stage1(const double* x, int64_t n, double* partial) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v += x[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void reduce_stage2(const double* partial, int np, double* out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += partial[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t reduce_sum(const double* x, int64_t n, double* partial, double* out, cudaStream_t s) {
  reduce_stage1<<<RED_BLOCKS, 256, 0, s>>>(x, n, partial);
  reduce_stage2<<<1, 256, 0, s>>>(partial, RED_BLOCKS, out);
  return cudaGetLastError();
}

}  // namespace vif
