// Analytic gradient of the Gaussian VIF negative log-likelihood (Sec. 2.2, App. A) in
// (sigma1^2, lambda_1..lambda_k, sigma^2), float64, with N and Z fixed.
//
// The paper writes the gradient as 1/2 Tr(Sigma~_dagger^{-1} dSigma~_dagger) - 1/2 alpha^T
// dSigma~_dagger alpha with dB, dD from App. A, one pass per parameter.  This file computes
// the same numbers in reverse mode, so that the cost does not grow with the number of
// parameters: with the whitened rows a_j = L_m^{-1} Sigma_mj, the factor rows
// F_i = (a_i - sum_k A_ik a_{N_k}) / sqrt(D_i), z_i = (y_i - sum_k A_ik y_{N_k}) / sqrt(D_i),
// C = I + F^T F, v = C^{-1} F^T z, r_i = z_i - F_i . v and E_i = C^{-1} F_i - r_i v,
//   L = 1/2 [sum_i log D_i + log det C + z^T z - z^T F v]  (+ n/2 log 2 pi),
//   dL = sum_i [1/2 dD_i / D_i + <dF_i, E_i> + r_i dz_i].
// Point i's A_i, D_i come from its residual block R_i = K~([N,i],[N,i]) - a_[N,i] a_[N,i]^T
// (A_i = R_NN^{-1} r_Ni, D_i = r_ii - r_iN A_i), so the adjoints Abar_i = dL/dA_i,
// Dbar_i = dL/dD_i give Rbar_i = dL/dR_i with lambda = R_NN^{-1} Abar_i:
//   Rbar[i][i] = Dbar,  Rbar[k][i] = (lambda_k - 2 Dbar A_ik) / 2,
//   Rbar[k][l] = Dbar A_ik A_il - (lambda_k A_il + A_ik lambda_l) / 2.
// Every a_j then collects V_j = (B^T D^{-1/2} E)_j - 2 sum_i (Rbar_i a_[N,i])_j, and with
// da_j = L^{-1}(dSigma_mj - dL a_j), L^{-1} dL = lower(S) + diag(S)/2, S = L^{-1} dSigma_m L^{-T}:
//   dL/dtheta = sum_i <Rbar_i, dK~_i/dtheta> + sum_{j,l} dSigma(x_j, z_l)/dtheta (V L^{-1})_jl
//               - <dSigma_m/dtheta, L^{-T} Psi L^{-1}>,   Psi_ab = P_{min(a,b) max(a,b)} / 2,
// P = sum_j a_j V_j^T.  Each term is a sum over kernel derivatives with weights formed once.
#include "vif_internal.cuh"

namespace vif {

namespace {

constexpr int GR_MAXP = 18;   // parameters: sigma1^2, up to 16 length scales, sigma^2

struct GradPar {
  int kind, d, nls, q;        // q = nls + 2
  double var, tdiag, jitter;
  double ls[16];
};

unsigned nblocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// dK/d(r^2) of the kernel (var included); 0 at r = 0 for the exponential kernel (its
// length-scale derivative carries a factor r^2 there)
__device__ __forceinline__ double dk_dr2(double r2, int kind, double var) {
  if (kind == VIF_SE) return -0.5 * var * exp(-0.5 * r2);
  const double r = sqrt(r2);
  if (kind == VIF_MATERN12) return r > 0.0 ? -0.5 * var * exp(-r) / r : 0.0;
  if (kind == VIF_MATERN32) return -1.5 * var * exp(-sqrt(3.0) * r);
  return -(5.0 / 6.0) * var * (1.0 + sqrt(5.0) * r) * exp(-sqrt(5.0) * r);
}

// w * dK(a, b)/dtheta added into g[0..q) for scaled coordinates a, b (no nugget, no jitter)
__device__ __forceinline__ void add_dk(const double* a, const double* b, const GradPar& P, double w, double* g) {
  double s2[16];
  double r2 = 0.0;
  for (int t = 0; t < P.d; ++t) {
    const double u = a[t] - b[t];
    s2[t] = u * u;
    r2 += s2[t];
  }
  g[0] += w * cov_r2<double>(r2, P.kind, P.var) / P.var;
  const double dk = dk_dr2(r2, P.kind, P.var);
  if (P.nls == 1) {
    g[1] += w * dk * (-2.0 * r2 / P.ls[0]);
  } else {
    for (int t = 0; t < P.nls; ++t) g[1 + t] += w * dk * (-2.0 * s2[t] / P.ls[t]);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// v = LC^{-T} l (l: the last row of the augmented factor); Cinv = LC^{-T} LC^{-1}
__global__ void gr_cinv_kernel(const double* __restrict__ LinvC, int ld, int m, const double* __restrict__ G, int ldg,
                               double* __restrict__ Cinv, double* __restrict__ v) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)m * m) {
    const int a = (int)(e / m), b = (int)(e % m);
    double s = 0.0;
    for (int c = max(a, b); c < m; ++c) s += LinvC[(size_t)c * ld + a] * LinvC[(size_t)c * ld + b];
    Cinv[e] = s;
  } else if (e < (int64_t)m * m + m) {
    const int a = (int)(e - (int64_t)m * m);
    double s = 0.0;
    for (int c = a; c < m; ++c) s += LinvC[(size_t)c * ld + a] * G[(size_t)m * ldg + c];
    v[a] = s;
  }
}

// r_i = z_i - F_i . v and E_i = Cinv F_i - r_i v (one warp per point)
__global__ void gr_E_kernel(const double* __restrict__ F, int fpad, int64_t n, int m, const double* __restrict__ Cinv,
                            const double* __restrict__ v, double* __restrict__ E, double* __restrict__ r) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* f = F + (size_t)i * fpad;
  double s = 0.0;
  for (int a = lane; a < m; a += 32) s += f[a] * v[a];
  const double ri = f[m] - warp_sum(s);
  if (lane == 0) r[i] = ri;
  for (int b = lane; b < m; b += 32) {
    double e = 0.0;
    for (int a = 0; a < m; ++a) e += Cinv[(size_t)a * m + b] * f[a];
    E[(size_t)i * m + b] = e - ri * v[b];
  }
}

// Per point: the local residual block and its adjoint; the direct kernel-derivative terms
// into part[i][0..q), and V_a += -2 (Rbar a_[N,i])_a + c_a E_i / sqrt(D_i) (float64 atomics).
// One warp per point; shared memory R, Rbar ((Q) x (Q + 1)) and three Q-vectors.
__global__ void gr_local_kernel(const double* __restrict__ A, int mpad, const double* __restrict__ Xs,
                                const int32_t* __restrict__ N, int mv, const double* __restrict__ Acoef,
                                const double* __restrict__ Dv, const double* __restrict__ F, int fpad,
                                const double* __restrict__ y, const double* __restrict__ E,
                                const double* __restrict__ r, int64_t n, int m, GradPar P, double* __restrict__ V,
                                double* __restrict__ part) {
  extern __shared__ double sh[];
  const int64_t i = blockIdx.x;
  const int lane = threadIdx.x;
  const int q = (int)(i < mv ? i : mv), Q = q + 1, LD = mv + 2;
  double* R = sh;                       // [Q][LD]
  double* Rb = R + (size_t)(mv + 1) * LD;
  double* lam = Rb + (size_t)(mv + 1) * LD;
  __shared__ int idx[66];
  for (int k = lane; k < Q; k += 32) idx[k] = k < q ? N[(size_t)i * mv + k] : (int)i;
  __syncwarp();
  const int d = P.d;
  // residual block R = K~ - a a^T (lower triangle)
  for (int e = lane; e < Q * Q; e += 32) {
    const int a = e / Q, b = e % Q;
    if (b > a) continue;
    const double* xa = Xs + (size_t)idx[a] * d;
    const double* xb = Xs + (size_t)idx[b] * d;
    double r2 = 0.0;
    for (int t = 0; t < d; ++t) {
      const double u = xa[t] - xb[t];
      r2 += u * u;
    }
    double s = cov_r2<double>(r2, P.kind, P.var) + (a == b ? P.tdiag : 0.0);
    const double* pa = A + (size_t)idx[a] * mpad;
    const double* pb = A + (size_t)idx[b] * mpad;
    for (int c = 0; c < m; ++c) s -= pa[c] * pb[c];
    R[a * LD + b] = s;
  }
  __syncwarp();
  const double Di = Dv[i], sd = sqrt(Di), ri = r[i];
  const double* Ei = E + (size_t)i * m;
  const double* Fi = F + (size_t)i * fpad;
  // adjoints of A_i and D_i
  for (int k = 0; k < q; ++k) {
    const double* an = A + (size_t)idx[k] * mpad;
    double s = 0.0;
    for (int c = lane; c < m; c += 32) s += an[c] * Ei[c];
    s = warp_sum(s);
    if (lane == 0) lam[k] = -(s + ri * y[idx[k]]) / sd;
  }
  double sf = 0.0;
  for (int c = lane; c < m; c += 32) sf += Fi[c] * Ei[c];
  sf = warp_sum(sf);
  const double Dbar = 0.5 / Di - 0.5 * (sf + ri * Fi[m]) / Di;
  __syncwarp();
  // lambda = R_NN^{-1} Abar: Cholesky of R_NN in place (lower), then two triangular solves
  for (int c = 0; c < q; ++c) {
    const double p = sqrt(R[c * LD + c]);
    __syncwarp();
    if (lane == 0) R[c * LD + c] = p;
    for (int a = c + 1 + lane; a < q; a += 32) R[a * LD + c] /= p;
    __syncwarp();
    for (int a = c + 1 + lane; a < q; a += 32) {
      const double l = R[a * LD + c];
      for (int b = c + 1; b <= a; ++b) R[a * LD + b] -= l * R[b * LD + c];
    }
    __syncwarp();
  }
  for (int k = 0; k < q; ++k) {          // forward: L y = Abar
    const double yk = lam[k] / R[k * LD + k];
    __syncwarp();
    if (lane == 0) lam[k] = yk;
    for (int a = k + 1 + lane; a < q; a += 32) lam[a] -= R[a * LD + k] * yk;
    __syncwarp();
  }
  for (int k = q - 1; k >= 0; --k) {     // backward: L^T lambda = y
    const double xk = lam[k] / R[k * LD + k];
    __syncwarp();
    if (lane == 0) lam[k] = xk;
    for (int a = lane; a < k; a += 32) lam[a] -= R[k * LD + a] * xk;
    __syncwarp();
  }
  // Rbar (full symmetric)
  const double* Ai = Acoef + (size_t)i * mv;
  for (int e = lane; e < Q * Q; e += 32) {
    const int a = e / Q, b = e % Q;
    double w;
    if (a == q && b == q) w = Dbar;
    else if (a == q) w = 0.5 * (lam[b] - 2.0 * Dbar * Ai[b]);
    else if (b == q) w = 0.5 * (lam[a] - 2.0 * Dbar * Ai[a]);
    else w = Dbar * Ai[a] * Ai[b] - 0.5 * (lam[a] * Ai[b] + Ai[a] * lam[b]);
    Rb[a * LD + b] = w;
  }
  __syncwarp();
  // direct terms: sum_ab Rbar_ab dK~(x_a, x_b)/dtheta (the nugget on the diagonal)
  double g[GR_MAXP];
  for (int k = 0; k < P.q; ++k) g[k] = 0.0;
  for (int e = lane; e < Q * Q; e += 32) {
    const int a = e / Q, b = e % Q;
    const double w = Rb[a * LD + b];
    add_dk(Xs + (size_t)idx[a] * d, Xs + (size_t)idx[b] * d, P, w, g);
    if (a == b) g[P.q - 1] += w;
  }
  for (int k = 0; k < P.q; ++k) {
    const double s = warp_sum(g[k]);
    if (lane == 0) part[(size_t)i * P.q + k] = s;
  }
  // V scatter
  for (int a = 0; a < Q; ++a) {
    const double ca = (a == q ? 1.0 : -Ai[a]) / sd;
    double* va = V + (size_t)idx[a] * m;
    for (int c = lane; c < m; c += 32) {
      double s = ca * Ei[c];
      for (int b = 0; b < Q; ++b) s -= 2.0 * Rb[a * LD + b] * A[(size_t)idx[b] * mpad + c];
      atomicAdd(va + c, s);
    }
  }
}

// Cross terms: Vt_j = L^{-T} V_j, then sum_l dSigma(x_j, z_l)/dtheta Vt_jl (one warp per point)
__global__ void gr_cross_kernel(const double* __restrict__ V, const double* __restrict__ Linv, int ldl,
                                const double* __restrict__ Xs, const double* __restrict__ Zs, int64_t n, int m,
                                GradPar P, double* __restrict__ part) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  const double* vj = V + (size_t)j * m;
  double g[GR_MAXP];
  for (int k = 0; k < P.q; ++k) g[k] = 0.0;
  for (int l = lane; l < m; l += 32) {
    double t = 0.0;
    for (int a = l; a < m; ++a) t += Linv[(size_t)a * ldl + l] * vj[a];
    add_dk(Xs + (size_t)j * P.d, Zs + (size_t)l * P.d, P, t, g);
  }
  for (int k = 0; k < P.q; ++k) {
    const double s = warp_sum(g[k]);
    if (lane == 0) part[(size_t)j * P.q + k] = s;
  }
}

// P = sum_j a_j V_j^T: 32 x 32 tiles, rows j in slices, float64 atomics
__global__ void gr_P_kernel(const double* __restrict__ A, int mpad, const double* __restrict__ V, int64_t n, int m,
                            int64_t rows_per, double* __restrict__ Pm) {
  const int a = blockIdx.x * 32 + threadIdx.x;
  const int b0 = blockIdx.y * 32 + threadIdx.y * 4;
  const int64_t j0 = (int64_t)blockIdx.z * rows_per, j1 = min(n, j0 + rows_per);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (a < m)
    for (int64_t j = j0; j < j1; ++j) {
      const double aj = A[(size_t)j * mpad + a];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (b0 + u < m) acc[u] += aj * V[(size_t)j * m + b0 + u];
    }
  if (a < m)
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (b0 + u < m) atomicAdd(&Pm[(size_t)a * m + b0 + u], acc[u]);
}

// T = Psi L^{-1} with Psi_ab = P_{min(a,b), max(a,b)} / 2
__global__ void gr_T_kernel(const double* __restrict__ Pm, const double* __restrict__ Linv, int ldl, int m,
                            double* __restrict__ T) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int a = (int)(e / m), c = (int)(e % m);
  double s = 0.0;
  for (int b = c; b < m; ++b) s += 0.5 * Pm[(size_t)min(a, b) * m + max(a, b)] * Linv[(size_t)b * ldl + c];
  T[e] = s;
}

// Omega = L^{-T} T
__global__ void gr_omega_kernel(const double* __restrict__ T, const double* __restrict__ Linv, int ldl, int m,
                                double* __restrict__ Om) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int dd = (int)(e / m), c = (int)(e % m);
  double s = 0.0;
  for (int a = dd; a < m; ++a) s += Linv[(size_t)a * ldl + dd] * T[(size_t)a * m + c];
  Om[e] = s;
}

// -<dSigma_m/dtheta, Omega> per block of inducing pairs (Sigma_m carries the jitter, which
// scales with sigma1^2)
__global__ void gr_inducing_kernel(const double* __restrict__ Zs, const double* __restrict__ Om, int m, GradPar P,
                                   double* __restrict__ part) {
  __shared__ double red[GR_MAXP][8];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double g[GR_MAXP];
  for (int k = 0; k < P.q; ++k) g[k] = 0.0;
  if (e < (int64_t)m * m) {
    const int a = (int)(e / m), b = (int)(e % m);
    const double w = -Om[e];
    add_dk(Zs + (size_t)a * P.d, Zs + (size_t)b * P.d, P, w, g);
    if (a == b) g[0] += w * P.jitter / P.var;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < P.q; ++k) {
    const double s = warp_sum(g[k]);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < P.q) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    part[(size_t)blockIdx.x * P.q + threadIdx.x] = s;
  }
}

// grad[k] = sum of the partial rows (a fixed order: deterministic)
__global__ void gr_sum_kernel(const double* __restrict__ part, int64_t rows, int q, double* __restrict__ out) {
  __shared__ double sh[256];
  for (int k = 0; k < q; ++k) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) s += part[(size_t)i * q + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

}  // namespace

size_t grad_scratch_doubles(int64_t n, int m, int mv, int q) {
  const size_t mm = (size_t)std::max(m, 1) * std::max(m, 1);
  (void)mv;
  return 2 * (size_t)n * std::max(m, 1)      // E, V
         + (size_t)n                          // r
         + 5 * mm + (size_t)std::max(m, 1)    // Cinv, P, T, Omega, (spare), v
         + 2 * (size_t)n * q                  // direct and cross partials
         + (mm / 256 + 1) * q + 8 * (size_t)q + 64;   // inducing partials, sums
}

cudaError_t vif_grad_fp64(const GradInputs& in, double* scratch, double* LinvC, double* trw, double* grad_dev,
                          cudaStream_t s) {
  const int64_t n = in.n;
  const int m = in.m, mv = in.mv, q = in.nls + 2;
  if (q > GR_MAXP || in.d > 16 || mv > 64) return cudaErrorInvalidValue;
  GradPar P{};
  P.kind = in.cp.kind;
  P.d = in.d;
  P.nls = in.nls;
  P.q = q;
  P.var = in.cp.var;
  P.tdiag = in.cp.tdiag;
  P.jitter = in.cp.jitter;
  for (int t = 0; t < in.nls; ++t) P.ls[t] = in.ls[t];
  const int mm1 = std::max(m, 1);
  double* E = scratch;
  double* V = E + (size_t)n * mm1;
  double* r = V + (size_t)n * mm1;
  double* Cinv = r + n;
  double* Pm = Cinv + (size_t)mm1 * mm1;
  double* T = Pm + (size_t)mm1 * mm1;
  double* Om = T + (size_t)mm1 * mm1;
  double* v = Om + 2 * (size_t)mm1 * mm1;
  double* pdir = v + mm1;
  double* pcross = pdir + (size_t)n * q;
  double* pind = pcross + (size_t)n * q;
  const int64_t nind = m > 0 ? ((int64_t)m * m + 255) / 256 : 0;
  double* sums = pind + (size_t)std::max<int64_t>(nind, 1) * q;
  cudaError_t e = cudaSuccess;
  if (m > 0) {
    e = dense_trtri_lower(in.G, LinvC, m, in.fpad, trw, s);
    if (e != cudaSuccess) return e;
    const int64_t tot = (int64_t)m * m + m;
    gr_cinv_kernel<<<nblocks(tot, 256), 256, 0, s>>>(LinvC, in.fpad, m, in.G, in.fpad, Cinv, v);
    gr_E_kernel<<<nblocks(n * 32, 256), 256, 0, s>>>(in.F, in.fpad, n, m, Cinv, v, E, r);
    e = cudaMemsetAsync(V, 0, sizeof(double) * (size_t)n * m, s);
    if (e != cudaSuccess) return e;
  } else {
    // no low-rank part: r_i = z_i, E and V are empty
    e = cudaMemcpy2DAsync(r, sizeof(double), in.F, sizeof(double) * in.fpad, sizeof(double), n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  const size_t lsm = sizeof(double) * ((size_t)2 * (mv + 1) * (mv + 2) + (mv + 1));
  if (lsm > 48 * 1024) {
    e = cudaFuncSetAttribute(gr_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
    if (e != cudaSuccess) return e;
  }
  gr_local_kernel<<<(unsigned)n, 32, lsm, s>>>(in.A, in.mpad, in.Xs, in.N, mv, in.Acoef, in.Dv, in.F, in.fpad,
                                               in.y, E, r, n, m, P, V, pdir);
  gr_sum_kernel<<<1, 256, 0, s>>>(pdir, n, q, sums);
  if (m > 0) {
    gr_cross_kernel<<<nblocks(n * 32, 256), 256, 0, s>>>(V, in.Linv, in.ldl, in.Xs, in.Zs, n, m, P, pcross);
    const int64_t slices = std::min<int64_t>(std::max<int64_t>(1, n / 256), 1024);
    const int64_t rows_per = (n + slices - 1) / slices;
    e = cudaMemsetAsync(Pm, 0, sizeof(double) * (size_t)m * m, s);
    if (e != cudaSuccess) return e;
    dim3 grid((m + 31) / 32, (m + 31) / 32, (unsigned)slices);
    gr_P_kernel<<<grid, dim3(32, 8), 0, s>>>(in.A, in.mpad, V, n, m, rows_per, Pm);
    gr_T_kernel<<<nblocks((int64_t)m * m, 256), 256, 0, s>>>(Pm, in.Linv, in.ldl, m, T);
    gr_omega_kernel<<<nblocks((int64_t)m * m, 256), 256, 0, s>>>(T, in.Linv, in.ldl, m, Om);
    gr_inducing_kernel<<<(unsigned)nind, 256, 0, s>>>(in.Zs, Om, m, P, pind);
    gr_sum_kernel<<<1, 256, 0, s>>>(pcross, n, q, sums + q);
    gr_sum_kernel<<<1, 256, 0, s>>>(pind, nind, q, sums + 2 * q);
  } else {
    e = cudaMemsetAsync(sums + q, 0, sizeof(double) * 2 * q, s);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(grad_dev, sums, sizeof(double) * 3 * q, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace vif
