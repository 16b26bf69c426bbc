// Prediction with the VIF approximation (Prop. 2.1; App. C.1), float64.
//
// Prediction points s^p condition on training points only (B_p = I): N_p(p) is
// the set of m_v training points with the smallest correlation distance d_c of
// Sec. 6, over all n training points.  With a_p = L_m^{-1} Sigma_{m,p},
// C = I + A Q A^T (Q = B^T D^{-1} B), u = A Q y and w = C^{-1} u, Prop. 2.1
// reduces to
//     mu_p = a_p . w + sum_k A_p[k] r_{N_k},     r = y - A^T w,
// and the nine terms of the App. C.1 variance collapse (using A Q A^T = C - I) to
//     var_p = D_p + || L_C^{-1} (a_p - sum_k A_p[k] a_{N_k}) ||^2,
// where A_p, D_p are the residual Vecchia coefficients and conditional variance
// of s^p given its neighbours (Eq. vecchia_pred), D_p including the nugget for
// the response y^p; the latent process b^p drops the nugget.
#include "vif_internal.cuh"

namespace vif {

// ---------------------------------------------------------------------------
// Non-causal float64 brute-force neighbours: one CTA per prediction point; each
// warp keeps a sorted top-64 list of (key, j) in registers, warp 0 merges.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool lexl(double ka, int ia, double kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

__device__ void list_insert64(double (&key)[2], int (&idx)[2], int& cnt, double nk, int ni) {
  const int lane = threadIdx.x & 31;
  int below = 0;
#pragma unroll
  for (int s = 0; s < 2; ++s) below += (idx[s] >= 0 && lexl(key[s], idx[s], nk, ni)) ? 1 : 0;
  const int pos = __reduce_add_sync(0xffffffffu, below);
  double pk = __shfl_up_sync(0xffffffffu, key[1], 1);
  int pi = __shfl_up_sync(0xffffffffu, idx[1], 1);
#pragma unroll
  for (int s = 1; s >= 0; --s) {
    const int g = lane * 2 + s;
    double ok = s ? key[0] : pk;
    int oi = s ? idx[0] : pi;
    if (g == pos) {
      key[s] = nk;
      idx[s] = ni;
    } else if (g > pos) {
      key[s] = ok;
      idx[s] = oi;
    }
  }
  if (cnt < 64) ++cnt;
}

__global__ __launch_bounds__(256) void pred_knn_kernel(const double* __restrict__ A, const double* __restrict__ Xs,
                                                       const double* __restrict__ cjj, const double* __restrict__ Ap,
                                                       const double* __restrict__ Xps, const double* __restrict__ cpp,
                                                       int64_t n, int d, int m, int mpad, int mv, int kind, double var,
                                                       double tau, int32_t* Np) {
  const int64_t p = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double mk[8][64];
  __shared__ int mi[8][64];
  double key[2] = {1e300, 1e300};
  int idx[2] = {-1, -1};
  int cnt = 0;
  const double cp = cpp[p];
  const double* ap = Ap + (size_t)p * mpad;
  const double* xp = Xps + (size_t)p * d;
  for (int64_t jb = (int64_t)w * 32; jb < n; jb += 256) {
    const int64_t j = jb + lane;
    double kj = 1e300;
    if (j < n) {
      double dot = 0.0;
      const double* aj = A + (size_t)j * mpad;
      for (int k = 0; k < m; ++k) dot += ap[k] * aj[k];
      const double cj = cjj[j];
      if (cp <= tau || cj <= tau) {
        kj = 1.0;
      } else {
        double K = cov_r2<double>(sqdist(xp, Xs + (size_t)j * d, d), kind, var);
        kj = 1.0 - fmin(fabs(K - dot) / sqrt(cp * cj), 1.0);
      }
    }
    double thr_k = __shfl_sync(0xffffffffu, key[1], 31);
    int thr_i = __shfl_sync(0xffffffffu, idx[1], 31);
    bool pass = (j < n) && (cnt < 64 || lexl(kj, (int)j, thr_k, thr_i));
    unsigned bal = __ballot_sync(0xffffffffu, pass);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      double nk = __shfl_sync(0xffffffffu, kj, src);
      int ni = __shfl_sync(0xffffffffu, (int)j, src);
      thr_k = __shfl_sync(0xffffffffu, key[1], 31);
      thr_i = __shfl_sync(0xffffffffu, idx[1], 31);
      if (cnt == 64 && !lexl(nk, ni, thr_k, thr_i)) continue;
      list_insert64(key, idx, cnt, nk, ni);
    }
  }
  mk[w][lane * 2] = key[0];
  mk[w][lane * 2 + 1] = key[1];
  mi[w][lane * 2] = idx[0];
  mi[w][lane * 2 + 1] = idx[1];
  __syncthreads();
  if (w != 0) return;
  for (int ww = 1; ww < 8; ++ww)
    for (int g = 0; g < 64; ++g) {
      double nk = mk[ww][g];
      int ni = mi[ww][g];
      if (ni < 0) continue;
      double thr_k = __shfl_sync(0xffffffffu, key[1], 31);
      int thr_i = __shfl_sync(0xffffffffu, idx[1], 31);
      if (cnt == 64 && !lexl(nk, ni, thr_k, thr_i)) continue;
      list_insert64(key, idx, cnt, nk, ni);
    }
  const int q = (int)(n < mv ? n : mv);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int gpos = lane * 2 + s;
    int rank = 0;
    for (int g = 0; g < 64; ++g) {
      int gid = __shfl_sync(0xffffffffu, idx[g & 1], g >> 1);
      if (g < q && gid >= 0 && gid < idx[s]) ++rank;
    }
    if (gpos < q && idx[s] >= 0) Np[(size_t)p * mv + rank] = idx[s];
  }
  for (int t = q + lane; t < mv; t += 32) Np[(size_t)p * mv + t] = -1;
}

// c_r(j,j) = sigma1^2 - ||a_j||^2 in float64, one warp per row.
__global__ void resid_var64_kernel(const double* A, int64_t n, int m, int mpad, double var, double* c) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int k = lane; k < m; k += 32) {
    double a = A[(size_t)i * mpad + k];
    s += a * a;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) c[i] = var - s;
}

// w = L_C^{-T} l_u, where row m of the augmented factor L' holds l_u = L_C^{-1} u.
// One CTA; column-oriented back substitution.
__global__ void solve_w_kernel(const double* Lg, int ldg, int m, double* w) {
  extern __shared__ double sw[];
  for (int k = threadIdx.x; k < m; k += blockDim.x) sw[k] = Lg[(size_t)m * ldg + k];
  __syncthreads();
  for (int k = m - 1; k >= 0; --k) {
    __shared__ double xk;
    if (threadIdx.x == 0) {
      xk = sw[k] / Lg[(size_t)k * ldg + k];
      sw[k] = xk;
    }
    __syncthreads();
    const double x = xk;
    for (int t = threadIdx.x; t < k; t += blockDim.x) sw[t] -= Lg[(size_t)k * ldg + t] * x;
    __syncthreads();
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) w[k] = sw[k];
}

// r_i = y_i - a_i . w, one warp per row.
__global__ void resid_r_kernel(const double* A, const double* w, const double* y, int64_t n, int m, int mpad,
                               double* r) {
  int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int k = lane; k < m; k += 32) s += A[(size_t)i * mpad + k] * w[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[i] = y[i] - s;
}

// ---------------------------------------------------------------------------
// One warp per prediction point: residual block of (s_{N_p}, s^p), Cholesky,
// coefficients A_p and D_p, mean and variance.  Shared memory per warp holds the
// (q+1) x (q+1) block and g_p = a_p - sum_k A_p[k] a_{N_k} (m values).
// ---------------------------------------------------------------------------
constexpr int PK_WARPS = 4;
constexpr int PK_QM = 49;

__global__ __launch_bounds__(PK_WARPS * 32) void predict_kernel(
    const double* __restrict__ A, const double* __restrict__ Xs, const double* __restrict__ Ap,
    const double* __restrict__ Xps, const int32_t* __restrict__ Np, const double* __restrict__ r,
    const double* __restrict__ w, const double* __restrict__ LinvC, int ldc, int64_t np, int d, int m, int mpad,
    int mv, CovParams cp, int latent, double nugget, double* mean, double* var, int* status) {
  extern __shared__ __align__(16) double psm[];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * PK_WARPS + wi;
  double* G = psm + (size_t)wi * (PK_QM * (PK_QM + 1) + PK_QM + mpad + 16 * PK_QM);
  double* coef = G + PK_QM * (PK_QM + 1);
  double* g = coef + PK_QM;
  double* xc = g + mpad;
  __shared__ int sidx[PK_WARPS][PK_QM];
  if (p >= np) return;
  int q = 0;
  for (int t = 0; t < mv; ++t)
    if (Np[(size_t)p * mv + t] >= 0) ++q;
  const int Q = q + 1;
  const int LD = PK_QM + 1;
  for (int t = lane; t < q; t += 32) sidx[wi][t] = Np[(size_t)p * mv + t];
  __syncwarp();
  // coordinates: neighbours, then the prediction point
  for (int e = lane; e < Q * d; e += 32) {
    int t = e / d, c = e % d;
    xc[t * 16 + c] = (t < q) ? Xs[(size_t)sidx[wi][t] * d + c] : Xps[(size_t)p * d + c];
  }
  __syncwarp();
  const double* ap = Ap + (size_t)p * mpad;
  // residual block (lower triangle): K + tdiag I - dot products
  const int npair = Q * (Q + 1) / 2;
  for (int e = lane; e < npair; e += 32) {
    int a = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    while (a * (a + 1) / 2 > e) --a;
    int b = e - a * (a + 1) / 2;
    const double* ra = (a < q) ? A + (size_t)sidx[wi][a] * mpad : ap;
    const double* rb = (b < q) ? A + (size_t)sidx[wi][b] * mpad : ap;
    double dot = 0.0;
    for (int k = 0; k < m; ++k) dot += ra[k] * rb[k];
    double kv = cov_r2<double>(sqdist(xc + a * 16, xc + b * 16, d), cp.kind, cp.var);
    if (a == b) kv += cp.tdiag;
    G[a * LD + b] = kv - dot;
  }
  __syncwarp();
  for (int c = 0; c < Q; ++c) {
    double piv = G[c * LD + c];
    if (!(piv > 0.0)) {
      if (lane == 0) flag_status(status, ST_NOTPD_FACTOR, p);
      piv = nan("");
    }
    double sp = sqrt(piv);
    __syncwarp();
    if (lane == 0) G[c * LD + c] = sp;
    for (int rr = c + 1 + lane; rr < Q; rr += 32) G[rr * LD + c] /= sp;
    __syncwarp();
    for (int rr = c + 1 + lane; rr < Q; rr += 32) {
      double grc = G[rr * LD + c];
      for (int s2 = c + 1; s2 <= rr; ++s2) G[rr * LD + s2] -= grc * G[s2 * LD + c];
    }
    __syncwarp();
  }
  const double lpp = G[q * LD + q];
  for (int t = lane; t < q; t += 32) coef[t] = G[q * LD + t];
  __syncwarp();
  for (int k = q - 1; k >= 0; --k) {
    double x = coef[k] / G[k * LD + k];
    __syncwarp();
    if (lane == 0) coef[k] = x;
    for (int t = lane; t < k; t += 32) coef[t] -= G[k * LD + t] * x;
    __syncwarp();
  }
  // g_p and the mean
  double mu = 0.0;
  for (int k = lane; k < m; k += 32) {
    double v = ap[k];
    mu += v * w[k];
    for (int t = 0; t < q; ++t) v -= coef[t] * A[(size_t)sidx[wi][t] * mpad + k];
    g[k] = v;
  }
  for (int t = lane; t < q; t += 32) mu += coef[t] * r[sidx[wi][t]];
  for (int o = 16; o > 0; o >>= 1) mu += __shfl_xor_sync(0xffffffffu, mu, o);
  __syncwarp();
  // || L_C^{-1} g ||^2 with the explicit inverse of L_C
  double ss = 0.0;
  for (int k = lane; k < m; k += 32) {
    double v = 0.0;
    const double* row = LinvC + (size_t)k * ldc;
    for (int c = 0; c <= k; ++c) v += row[c] * g[c];
    ss += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) {
    double v = lpp * lpp + ss;
    if (latent) v -= nugget;
    mean[p] = mu;
    if (var) var[p] = v;
  }
}

// Neighbour sets N_p and residual variances of the prediction points.
cudaError_t predict_setup(const double* A, const double* Xs, int64_t n, const double* Ap, const double* Xps,
                          int64_t np, int d, int m, int mpad, int mv, CovParams cp, double* cjj, double* cpp,
                          int32_t* Np, cudaStream_t s) {
  if (mv > PK_QM - 1 || d > 16) return cudaErrorInvalidValue;
  const double tau = 1e-6 * cp.var;
  resid_var64_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(A, n, m, mpad, cp.var, cjj);
  resid_var64_kernel<<<(unsigned)((np + 7) / 8), 256, 0, s>>>(Ap, np, m, mpad, cp.var, cpp);
  if (mv > 0)
    pred_knn_kernel<<<(unsigned)np, 256, 0, s>>>(A, Xs, cjj, Ap, Xps, cpp, n, d, m, mpad, mv, cp.kind, cp.var, tau,
                                                 Np);
  return cudaGetLastError();
}

// r = y - A^T w (one value per training point)
cudaError_t predict_resid(const double* A, const double* w, const double* y, int64_t n, int m, int mpad, double* r,
                          cudaStream_t s) {
  resid_r_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(A, w, y, n, m, mpad, r);
  return cudaGetLastError();
}

// Means (and, if var != NULL, variances) of the prediction points from w and r.
cudaError_t predict_eval(const double* A, const double* Xs, const double* Ap, const double* Xps, const int32_t* Np,
                         const double* r, const double* w, const double* LinvC, int ldg, int64_t np, int d, int m,
                         int mpad, int mv, CovParams cp, int latent, double nugget, double* mean, double* var,
                         int* status, cudaStream_t s) {
  const size_t per_warp = (size_t)(PK_QM * (PK_QM + 1) + PK_QM + mpad + 16 * PK_QM) * sizeof(double);
  const size_t smem = per_warp * PK_WARPS;
  cudaError_t e = cudaFuncSetAttribute(predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  predict_kernel<<<(unsigned)((np + PK_WARPS - 1) / PK_WARPS), PK_WARPS * 32, smem, s>>>(
      A, Xs, Ap, Xps, Np, r, w, LinvC, ldg, np, d, m, mpad, mv, cp, latent, nugget, mean, var, status);
  return cudaGetLastError();
}

cudaError_t predict_all(const double* A, const double* Xs, int64_t n, const double* Ap, const double* Xps,
                        int64_t np, int d, int m, int mpad, int mv, CovParams cp, const double* y, const double* Lg,
                        int ldg, double* LinvC, double* w, double* r, double* cjj, double* cpp, int32_t* Np,
                        int latent, double nugget, double* mean, double* var, int* status, double* trwork,
                        cudaStream_t s) {
  cudaError_t e = predict_setup(A, Xs, n, Ap, Xps, np, d, m, mpad, mv, cp, cjj, cpp, Np, s);
  if (e != cudaSuccess) return e;
  if (m > 0) {
    solve_w_kernel<<<1, 256, (size_t)m * sizeof(double), s>>>(Lg, ldg, m, w);
    e = dense_trtri_lower(Lg, LinvC, m, ldg, trwork, s);
    if (e != cudaSuccess) return e;
  }
  e = predict_resid(A, w, y, n, m, mpad, r, s);
  if (e != cudaSuccess) return e;
  return predict_eval(A, Xs, Ap, Xps, Np, r, w, LinvC, ldg, np, d, m, mpad, mv, cp, latent, nugget, mean, var,
                      status, s);
}

}  // namespace vif
