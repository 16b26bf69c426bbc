// float64 dense linear algebra for the m x m matrices of the method: the Cholesky
// factor of Sigma_m (Sec. 2.1) and of the capacitance matrix C = L_m^{-1} M L_m^{-T}
// (M of Eq. def_M, Sec. 2.2), and the inverse of the lower factor L_m.
//
// GB300 executes float64 at 1/64 of its float32 rate: a warp's float64 instruction
// occupies its SM sub-partition for 64 cycles whether 1 or 32 lanes are active, a
// square root ~680 cycles and a division ~430.  The blocked right-looking Cholesky
// below therefore keeps the serial chain short and spreads the rest over many SMs:
// one launch factors the 16 x 16 diagonal tile (redundantly in every CTA) together
// with the tile below it in one column sweep held in registers (pivots by a Newton-
// refined reciprocal square root, formed one column ahead), the next updates the
// trailing tiles, one CTA per tile.
#include <algorithm>

#include "vif_internal.cuh"

namespace vif {

constexpr int NB = 32;

__device__ __forceinline__ double ld_lower(const double* A, int lda, int m, int r, int c) {
  if (r < m && c < m) return A[(size_t)r * lda + c];
  return (r == c) ? 1.0 : 0.0;
}

// Inverse of the lower-triangular tile L (in smem) into X (lower): every column of X
// solves L x = e_c; the sweep goes row by row (x_r = b_r / L_rr, then every later row
// drops L[s][r] x_r), all 32 columns and all later rows at once.
__device__ void tile_trtri(const double (*L)[NB + 1], const double* rinv, double (*X)[NB + 1]) {
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int r = idx / NB, c = idx % NB;
    X[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int r = 0; r < NB; ++r) {
    if (threadIdx.x <= r) X[r][threadIdx.x] *= rinv[r];   // columns c <= r
    __syncthreads();
    const int w = NB - r - 1;
    for (int idx = threadIdx.x; idx < w * (r + 1); idx += blockDim.x) {
      const int s2 = r + 1 + idx / (r + 1), c = idx % (r + 1);
      X[s2][c] -= L[s2][r] * X[r][c];
    }
    __syncthreads();
  }
}

// 1/sqrt(p) for p > 0: a float32 estimate refined by two Newton steps
// y <- y (3 - p y^2) / 2 in float64 (quadratic convergence: ~1e-7 -> ~1e-14 -> rounding).
// Each float64 instruction costs tens of cycles on this part, and this takes fewer of
// them than a square root followed by a division.
__device__ __forceinline__ double rsqrt_newton(double p) {
  double y = (double)rsqrtf((float)p);
  y = y * (1.5 - 0.5 * p * y * y);
  y = y * (1.5 - 0.5 * p * y * y);
  return y;
}

// Blocked right-looking Cholesky with 16 x 16 tiles.  Step k: CTA b factors the diagonal
// tile L_kk and, for b > 0, the tile T_b below it (X L_kk^T = T_b) in one column sweep over
// the stacked 32 x 16 block [L_kk; T_b], which lives in registers: thread t holds row t / 4,
// columns t % 4 + 4j.  Per column: the owner of the pivot has already formed it (a
// look-ahead at the end of the previous column), the column below it is scaled and shared
// through shared memory, and every later column takes its rank-1 update; a thread whose
// columns are all done issues no float64 instruction.  CTA b writes X.  Every CTA reads the
// unfactored A_kk, and nothing orders the CTAs of a launch (a CTA may start only after
// another has finished, when the GPU is busy or the batched launch has more CTAs than fit),
// so CTA 0 must not overwrite A_kk while others may still read it: when the step has more
// than one CTA, CTA 0 parks L_kk in the upper triangle, which the factorisation never
// reads (its strictly lower part transposed into the tile's upper part, its diagonal in
// the column after the tile), and CTA 0 of the step's trailing update (the next launch)
// moves it into place.
constexpr int CH = 16;

__device__ __forceinline__ void chol_panel_body(double* A, int m, int lda, int k, int* status, int code,
                                                const int blk) {
  __shared__ double col[2 * CH];
  __shared__ double rs[CH];
  const int t = threadIdx.x, r = t >> 2, g = t & 3;
  const int k0 = k * CH;
  const bool has_t = blk > 0;
  const int r0 = (k + blk) * CH;   // first row of T_b
  const bool live = r < CH || has_t;
  const int nt = (m + CH - 1) / CH;
  double v[CH / 4];
#pragma unroll
  for (int j = 0; j < CH / 4; ++j) {
    const int sc = g + 4 * j;
    v[j] = !live ? 0.0
                 : (r < CH ? (sc <= r ? ld_lower(A, lda, m, k0 + r, k0 + sc) : 0.0)
                           : ld_lower(A, lda, m, r0 + r - CH, k0 + sc));
  }
  // pivot c from its owner's current value: M[c][c] <- sqrt(p), rs[c] <- 1/sqrt(p)
  auto pivot = [&](double& pv, int c) {
    double p = pv;
    if (!(p > 0.0)) {
      if (blk == 0 && status) flag_status(status, code, k0 + c);
      p = nan("");
    }
    const double y = rsqrt_newton(p);
    pv = p * y;
    rs[c] = y;
  };
  if (t == 0) pivot(v[0], 0);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int jc = c >> 2;
    // column c below the pivot, scaled and shared
    if (g == (c & 3) && r > c && live) {
      v[jc] *= rs[c];
      col[r] = v[jc];
    }
    __syncthreads();
    if (r > c && live) {
      const double lr = col[r];
#pragma unroll
      for (int j = 0; j < CH / 4; ++j) {
        if (j >= jc) {   // uniform: columns 4j .. 4j + 3 may still need column c
          const int sc = g + 4 * j;
          if (sc > c && (r >= CH || sc <= r)) v[j] = fma(-lr, col[sc], v[j]);
        }
      }
    }
    // look-ahead: the owner of pivot c + 1 has just updated it
    if (c + 1 < CH && t == 4 * (c + 1) + ((c + 1) & 3)) pivot(v[(c + 1) >> 2], c + 1);
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < CH / 4; ++j) {
    const int sc = g + 4 * j;
    if (!has_t) {
      if (r < CH && sc <= r && k0 + r < m && k0 + sc < m) {
        if (nt - k == 1) A[(size_t)(k0 + r) * lda + k0 + sc] = v[j];          // the only CTA
        else if (sc < r) A[(size_t)(k0 + sc) * lda + k0 + r] = v[j];          // parked, transposed
        else A[(size_t)(k0 + r) * lda + k0 + CH] = v[j];                      // parked diagonal
      }
    } else if (r >= CH) {
      const int rr = r0 + r - CH;
      if (rr < m && k0 + sc < m) A[(size_t)rr * lda + k0 + sc] = v[j];
    }
  }
}

// Trailing update A_ij -= L_ik L_jk^T of step k, one CTA per 16 x 16 tile (i, j), one
// output per thread, summed in a fixed order: the capacitance matrix is ill-conditioned
// enough (condition ~1e7-1e8) that a run-to-run change in the last bits of its factor shows
// in the likelihood.
__global__ __launch_bounds__(128) void chol_panel_kernel(double* A, int m, int lda, int k, int* status, int code) {
  chol_panel_body(A, m, lda, k, status, code, blockIdx.x);
}

__device__ __forceinline__ void chol_update_body(double* A, int m, int lda, int k, const int b) {
  if (b == 0) {
    // L_kk from where the panel launch parked it (the step had two or more CTAs, so its
    // tile is full and column k0 + 16 exists); no CTA of this launch touches tile k
    const int k0 = k * CH;
    for (int e = threadIdx.x; e < CH * CH; e += blockDim.x) {
      const int rr = e / CH, cc = e % CH;
      if (rr > cc) A[(size_t)(k0 + rr) * lda + k0 + cc] = A[(size_t)(k0 + cc) * lda + k0 + rr];
      else if (rr == cc) A[(size_t)(k0 + rr) * lda + k0 + rr] = A[(size_t)(k0 + rr) * lda + k0 + CH];
    }
  }
  // tile (i, j), k < j <= i < nt, enumerated over the lower triangle
  int ii = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((ii + 1) * (ii + 2) / 2 <= b) ++ii;
  while (ii * (ii + 1) / 2 > b) --ii;
  const int jj = b - ii * (ii + 1) / 2;
  const int i0 = (k + 1 + ii) * CH, j0 = (k + 1 + jj) * CH, k0 = k * CH;
  __shared__ double Li[CH][CH + 1];
  __shared__ double Lj[CH][CH + 1];
  const int t = threadIdx.x, r = t / CH, c = t % CH;
  Li[r][c] = (i0 + r < m && k0 + c < m) ? A[(size_t)(i0 + r) * lda + k0 + c] : 0.0;
  Lj[r][c] = (j0 + r < m && k0 + c < m) ? A[(size_t)(j0 + r) * lda + k0 + c] : 0.0;
  __syncthreads();
  if (i0 + r >= m || j0 + c >= m || (ii == jj && c > r)) return;
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < CH; ++q) acc = fma(Li[r][q], Lj[c][q], acc);
  A[(size_t)(i0 + r) * lda + j0 + c] -= acc;
}

__global__ __launch_bounds__(256) void chol_update_kernel(double* A, int m, int lda, int k) {
  chol_update_body(A, m, lda, k, blockIdx.x);
}

// k-slices of the triangular-inverse products (one CTA each, float64 atomics)
constexpr int KS = 4;
constexpr int KSW = NB / KS;

cudaError_t dense_cholesky(double* A, int m, int lda, int* status, int code, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int nt = (m + CH - 1) / CH;
  for (int k = 0; k < nt; ++k) {
    chol_panel_kernel<<<nt - k, 128, 0, s>>>(A, m, lda, k, status, code);
    const int T = nt - k - 1;
    if (T > 0) chol_update_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(A, m, lda, k);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inverse of a lower-triangular L (blocked):  Linv_tt = L_tt^{-1};
// Linv_ij = -Linv_ii * sum_{k=j}^{i-1} L_ik Linv_kj, one block diagonal s = i - j at
// a time.  Within a step every tile product L_ik Linv_kj is split into KS slices along
// k, each its own CTA adding into a per-(i,j) float64 tile with atomics, so a step costs
// two quarter tile products of latency instead of s + 1 whole ones.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void trtri_diag_body(const double* L, double* Li, int m, int lda, const int blk) {
  __shared__ double Lt[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  __shared__ double rinv[NB];
  const int t0 = blk * NB;
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

__global__ void trtri_diag_kernel(const double* L, double* Li, int m, int lda) {
  trtri_diag_body(L, Li, m, lda, blockIdx.x);
}

// acc += P[rows][kk0..kk0+KSW) Q[kk0..kk0+KSW)[cols] for the 2 x 2 outputs of thread (tx, ty)
__device__ void tile_prod_acc_k(const double (*P)[NB + 1], const double (*Q)[NB + 1], int kk0, double acc[2][2],
                                int tx, int ty) {
#pragma unroll
  for (int c = kk0; c < kk0 + KSW; ++c) {
    double a0 = P[ty][c], a1 = P[ty + 16][c];
    double b0 = Q[c][tx], b1 = Q[c][tx + 16];
    acc[0][0] += a0 * b0;
    acc[0][1] += a0 * b1;
    acc[1][0] += a1 * b0;
    acc[1][1] += a1 * b1;
  }
}

// tmp[j] += L_{j+s,k} Linv_{k,j},  k = j + kk; CTA b = (j * s + kk) * KS + slice
__device__ __forceinline__ void trtri_prod_body(const double* L, const double* Li, int m, int lda, int sdiag,
                                                double* tmp, const int blk) {
  const int pb = blk / KS, ks = blk % KS;
  const int j = pb / sdiag, kk = pb % sdiag;
  const int i0 = (j + sdiag) * NB, j0 = j * NB, k0 = (j + kk) * NB;
  __shared__ double P[NB][NB + 1];
  __shared__ double Q[NB][NB + 1];
  const int kk0 = ks * KSW;
  for (int idx = threadIdx.x; idx < NB * KSW; idx += blockDim.x) {
    const int r = idx / KSW, c = kk0 + idx % KSW;        // P columns / Q rows of this slice
    P[r][c] = (i0 + r < m && k0 + c < m) ? L[(size_t)(i0 + r) * lda + k0 + c] : 0.0;
    const int qr = kk0 + idx / NB, qc = idx % NB;
    Q[qr][qc] = (k0 + qr < m && j0 + qc < m) ? Li[(size_t)(k0 + qr) * lda + j0 + qc] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2] = {{0, 0}, {0, 0}};
  tile_prod_acc_k(P, Q, kk0, acc, tx, ty);
  double* Tm = tmp + (size_t)j * NB * NB;
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) atomicAdd(&Tm[(ty + 16 * u) * NB + tx + 16 * v], acc[u][v]);
}

__global__ void trtri_prod_kernel(const double* L, const double* Li, int m, int lda, int sdiag, double* tmp) {
  trtri_prod_body(L, Li, m, lda, sdiag, tmp, blockIdx.x);
}

// Linv_{j+s,j} = -Linv_{j+s,j+s} tmp[j] (added over KS slices into the zeroed Linv);
// each slice clears the rows of tmp[j] it read, for the next step.
__device__ __forceinline__ void trtri_fin_body(double* Li, int m, int lda, int sdiag, double* tmp, const int blk) {
  const int j = blk / KS, ks = blk % KS;
  const int i0 = (j + sdiag) * NB, j0 = j * NB;
  __shared__ double P[NB][NB + 1];
  __shared__ double Q[NB][NB + 1];
  double* Tm = tmp + (size_t)j * NB * NB;
  const int kk0 = ks * KSW;
  for (int idx = threadIdx.x; idx < NB * KSW; idx += blockDim.x) {
    const int r = idx / KSW, c = kk0 + idx % KSW;
    P[r][c] = (i0 + r < m && i0 + c < m) ? Li[(size_t)(i0 + r) * lda + i0 + c] : 0.0;
    const int qr = kk0 + idx / NB, qc = idx % NB;
    Q[qr][qc] = Tm[qr * NB + qc];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NB * KSW; idx += blockDim.x) Tm[(kk0 + idx / NB) * NB + idx % NB] = 0.0;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2] = {{0, 0}, {0, 0}};
  tile_prod_acc_k(P, Q, kk0, acc, tx, ty);
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) {
      int r = ty + 16 * u, c = tx + 16 * v;
      if (i0 + r < m && j0 + c < m) atomicAdd(&Li[(size_t)(i0 + r) * lda + j0 + c], -acc[u][v]);
    }
}

__global__ void trtri_fin_kernel(double* Li, int m, int lda, int sdiag, double* tmp) {
  trtri_fin_body(Li, m, lda, sdiag, tmp, blockIdx.x);
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
  trtri_diag_kernel<<<nt, 256, 0, s>>>(L, Linv, m, lda);
  for (int sd = 1; sd < nt; ++sd) {
    trtri_prod_kernel<<<(nt - sd) * sd * KS, 256, 0, s>>>(L, Linv, m, lda, sd, work);
    trtri_fin_kernel<<<(nt - sd) * KS, 256, 0, s>>>(Linv, m, lda, sd, work);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Many independent factorizations at once (the batched likelihoods): each launch runs the
// same step of every job, its blocks split among the jobs by a prefix of per-job block
// counts (block b belongs to the job p with off[p] <= b < off[p + 1]).  A job's blocks do
// exactly what the single-problem launch of that step does, so the results are the same.
// ---------------------------------------------------------------------------
namespace {

enum DenseOp { OP_PANEL = 0, OP_UPDATE = 1, OP_TDIAG = 2, OP_TPROD = 3, OP_TFIN = 4 };

__device__ __forceinline__ int job_of(const int* __restrict__ off, int njobs, int b) {
  int lo = 0, hi = njobs;   // largest p with off[p] <= b
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ __launch_bounds__(128) void chol_panel_batched(const DenseJob* __restrict__ jobs,
                                                          const int* __restrict__ off, int njobs, int k) {
  const int p = job_of(off, njobs, blockIdx.x);
  const DenseJob J = jobs[p];
  chol_panel_body(J.A, J.m, J.lda, k, J.status, J.code, blockIdx.x - off[p]);
}
__global__ __launch_bounds__(256) void chol_update_batched(const DenseJob* __restrict__ jobs,
                                                           const int* __restrict__ off, int njobs, int k) {
  const int p = job_of(off, njobs, blockIdx.x);
  const DenseJob J = jobs[p];
  chol_update_body(J.A, J.m, J.lda, k, blockIdx.x - off[p]);
}
__global__ void trtri_diag_batched(const DenseJob* __restrict__ jobs, const int* __restrict__ off, int njobs) {
  const int p = job_of(off, njobs, blockIdx.x);
  const DenseJob J = jobs[p];
  trtri_diag_body(J.A, J.Li, J.m, J.lda, blockIdx.x - off[p]);
}
__global__ void trtri_prod_batched(const DenseJob* __restrict__ jobs, const int* __restrict__ off, int njobs,
                                   int sd) {
  const int p = job_of(off, njobs, blockIdx.x);
  const DenseJob J = jobs[p];
  trtri_prod_body(J.A, J.Li, J.m, J.lda, sd, J.work, blockIdx.x - off[p]);
}
__global__ void trtri_fin_batched(const DenseJob* __restrict__ jobs, const int* __restrict__ off, int njobs, int sd) {
  const int p = job_of(off, njobs, blockIdx.x);
  const DenseJob J = jobs[p];
  trtri_fin_body(J.Li, J.m, J.lda, sd, J.work, blockIdx.x - off[p]);
}

// blocks of job J in launch (op, step)
int dense_blocks(const DenseJob& J, int op, int step) {
  if (J.m <= 0) return 0;
  const int nt = (J.m + CH - 1) / CH, ntt = (J.m + NB - 1) / NB;
  switch (op) {
    case OP_PANEL: return step < nt ? nt - step : 0;
    case OP_UPDATE: {
      const int T = nt - step - 1;
      return T > 0 ? T * (T + 1) / 2 : 0;
    }
    case OP_TDIAG: return ntt;
    case OP_TPROD: return step < ntt ? (ntt - step) * step * KS : 0;
    default: return step < ntt ? (ntt - step) * KS : 0;
  }
}

}  // namespace

void dense_batch_free(DenseBatch* b) {
  if (b->djobs) cudaFree(b->djobs);
  if (b->doff) cudaFree(b->doff);
  *b = DenseBatch();
}

cudaError_t dense_batch_init(const std::vector<DenseJob>& jobs, bool trtri, DenseBatch* b) {
  dense_batch_free(b);
  b->njobs = (int)jobs.size();
  b->trtri = trtri;
  if (b->njobs == 0) return cudaSuccess;
  int maxm = 0;
  for (const auto& J : jobs) maxm = std::max(maxm, J.m);
  std::vector<int> off;
  auto add = [&](int op, int step) {
    int tot = 0;
    std::vector<int> o(b->njobs + 1);
    for (int p = 0; p < b->njobs; ++p) {
      o[p] = tot;
      tot += dense_blocks(jobs[p], op, step);
    }
    o[b->njobs] = tot;
    if (tot == 0) return;
    b->launches.push_back({op, step, tot, (int)off.size()});
    off.insert(off.end(), o.begin(), o.end());
  };
  if (!trtri) {
    const int nt = (maxm + CH - 1) / CH;
    for (int k = 0; k < nt; ++k) {
      add(OP_PANEL, k);
      add(OP_UPDATE, k);
    }
  } else {
    const int ntt = (maxm + NB - 1) / NB;
    add(OP_TDIAG, 0);
    for (int sd = 1; sd < ntt; ++sd) {
      add(OP_TPROD, sd);
      add(OP_TFIN, sd);
    }
  }
  cudaError_t e = cudaMalloc((void**)&b->djobs, sizeof(DenseJob) * jobs.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->doff, sizeof(int) * std::max<size_t>(off.size(), 1));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->djobs, jobs.data(), sizeof(DenseJob) * jobs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !off.empty())
    e = cudaMemcpy(b->doff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) dense_batch_free(b);
  return e;
}

cudaError_t dense_batch_run(const DenseBatch& b, cudaStream_t s) {
  for (const auto& L : b.launches) {
    const int* off = b.doff + L.off;
    switch (L.op) {
      case OP_PANEL: chol_panel_batched<<<L.blocks, 128, 0, s>>>(b.djobs, off, b.njobs, L.step); break;
      case OP_UPDATE: chol_update_batched<<<L.blocks, 256, 0, s>>>(b.djobs, off, b.njobs, L.step); break;
      case OP_TDIAG: trtri_diag_batched<<<L.blocks, 256, 0, s>>>(b.djobs, off, b.njobs); break;
      case OP_TPROD: trtri_prod_batched<<<L.blocks, 256, 0, s>>>(b.djobs, off, b.njobs, L.step); break;
      default: trtri_fin_batched<<<L.blocks, 256, 0, s>>>(b.djobs, off, b.njobs, L.step); break;
    }
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
