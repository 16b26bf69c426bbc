// Laplace approximation for a Bernoulli-logit likelihood with the VIF prior
// (Sec. 3, Eq. one_it_newton_mode), solved by preconditioned CG (Eq. pcls1) with
// the VIFDU preconditioner (Sec. 4.3, App. E.1).  float64 throughout.
//
// With Q = B^T D^{-1} B, F = D^{-1/2} B A^T (rows f_i) and C = I + F^T F:
//   (W + Sigma_dagger^{-1}) x = W x + B^T D^{-1/2} (t - F C^{-1} F^T t),  t = D^{-1/2} B x,
// and the VIFDU preconditioner P = B^T W B + Sigma_dagger^{-1} is applied as
//   P^{-1} w = B^{-1} G^{-1} (x + D^{-1/2} F C_3^{-1} F^T D^{-1/2} G^{-1} x),  x = B^{-T} w,
// with G = W + D^{-1} and C_3 = I + F^T diag(D_i W_i / (1 + D_i W_i)) F, which is
// L_m^{-1} M_3 L_m^{-T} for the M_3 of App. E.1.  A learned diagonal correction
// replaces W by W' = W exp(c) inside P only (the system keeps W).
//
// The triangular solves with B and B^T are sync-free: warps take rows from an
// atomic work queue in dependency order and wait for the rows they need through
// per-row epoch flags (release/acquire).  Every wait is bounded; a wait that runs
// out sets an abort flag that ends all waits, and the host reports
// VIF_ERR_TIMEOUT.
#include "vif_internal.cuh"

namespace vif {

constexpr int SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }

// Wait until flags[j] == epoch (or abort).  Returns false on abort/timeout.
__device__ __forceinline__ bool wait_ready(const int* flags, int64_t j, int epoch, int* abort_flag, int* status,
                                           int64_t row) {
  int it = 0;
  while (ld_acquire(flags + j) != epoch) {
    if (ld_volatile(abort_flag)) return false;
    if (++it > SPIN_LIMIT) {
      atomicExch(abort_flag, 1);
      flag_status(status, ST_TIMEOUT, row);
      return false;
    }
  }
  return true;
}

// out = B^{-1} rhs:  out_i = rhs_i + sum_k A_i[k] out_{N_k}  (rows in increasing order)
__global__ void sptrsv_B_kernel(const int32_t* __restrict__ N, const double* __restrict__ Acoef, int64_t n, int mv,
                                const double* __restrict__ rhs, double* out, int* flags, int epoch, int* counter,
                                int* abort_flag, int* status) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int64_t row = 0;
    if (lane == 0) row = atomicAdd(reinterpret_cast<unsigned long long*>(counter), 1ull);
    row = __shfl_sync(0xffffffffu, row, 0);
    if (row >= n) return;
    const int q = (int)(row < mv ? row : mv);
    double s = 0.0;
    bool ok = true;
    for (int t = lane; t < q; t += 32) {
      const int j = N[(size_t)row * mv + t];
      if (!wait_ready(flags, j, epoch, abort_flag, status, row)) {
        ok = false;
        break;
      }
      s += Acoef[(size_t)row * mv + t] * __ldcg(out + j);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    (void)__all_sync(0xffffffffu, ok);
    if (lane == 0) {
      out[row] = rhs[row] + s;
      __threadfence();
      st_release(flags + row, epoch);   // released even after an abort, so nobody waits on this row
    }
  }
}

// x = B^{-T} w:  x_j = w_j + sum_{(i,k): N_k(i) = j} A_i[k] x_i  (rows in decreasing order)
__global__ void sptrsv_Bt_kernel(const int32_t* __restrict__ ch_ptr, const int32_t* __restrict__ ch_row,
                                 const int32_t* __restrict__ ch_slot, const double* __restrict__ Acoef, int64_t n,
                                 int mv, const double* __restrict__ w, double* x, int* flags, int epoch, int* counter,
                                 int* abort_flag, int* status) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int64_t k = 0;
    if (lane == 0) k = atomicAdd(reinterpret_cast<unsigned long long*>(counter), 1ull);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= n) return;
    const int64_t row = n - 1 - k;
    const int b = ch_ptr[row], e = ch_ptr[row + 1];
    double s = 0.0;
    bool ok = true;
    for (int t = b + lane; t < e; t += 32) {
      const int i = ch_row[t];
      if (!wait_ready(flags, i, epoch, abort_flag, status, row)) {
        ok = false;
        break;
      }
      s += Acoef[(size_t)i * mv + ch_slot[t]] * __ldcg(x + i);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    (void)__all_sync(0xffffffffu, ok);
    if (lane == 0) {
      x[row] = w[row] + s;
      __threadfence();
      st_release(flags + row, epoch);
    }
  }
}

// t_i = (x_i - sum_k A_i[k] x_{N_k}) / sqrt(D_i)
__global__ void bx_scaled_kernel(const int32_t* __restrict__ N, const double* __restrict__ Acoef,
                                 const double* __restrict__ rsD, int64_t n, int mv, const double* __restrict__ x,
                                 double* t) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int q = (int)(i < mv ? i : mv);
  double s = x[i];
  for (int k = 0; k < q; ++k) s -= Acoef[(size_t)i * mv + k] * x[N[(size_t)i * mv + k]];
  t[i] = s * rsD[i];
}

// out_j = diagW_j x_j + rsD_j t_j - sum_{(i,k) in ch(j)} A_i[k] rsD_i t_i
__global__ void btx_kernel(const int32_t* __restrict__ ch_ptr, const int32_t* __restrict__ ch_row,
                           const int32_t* __restrict__ ch_slot, const double* __restrict__ Acoef,
                           const double* __restrict__ rsD, int64_t n, int mv, const double* __restrict__ t,
                           const double* __restrict__ diagW, const double* __restrict__ x, double* out) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = rsD[j] * t[j];
  for (int p = ch_ptr[j]; p < ch_ptr[j + 1]; ++p) {
    const int i = ch_row[p];
    s -= Acoef[(size_t)i * mv + ch_slot[p]] * rsD[i] * t[i];
  }
  if (diagW) s += diagW[j] * x[j];
  out[j] = s;
}

// partial[b][c] = sum over the rows of block b of F[i][c] * v[i]   (c < m)
constexpr int FT_ROWS = 256;
__global__ void ftv_kernel(const double* __restrict__ F, int fpad, int m, int64_t n, const double* __restrict__ v,
                           double* partial) {
  const int64_t r0 = (int64_t)blockIdx.x * FT_ROWS;
  const int64_t r1 = (n < r0 + FT_ROWS) ? n : r0 + FT_ROWS;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s += F[(size_t)r * fpad + c] * v[r];
    partial[(size_t)blockIdx.x * fpad + c] = s;
  }
}
__global__ void col_reduce_kernel(const double* partial, int nb, int fpad, int m, double* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(size_t)b * fpad + c];
  out[c] = s;
}

// y = L x (lower) or y = L^T x, L m x m with leading dimension ld; warp per output.
__global__ void lower_gemv_kernel(const double* __restrict__ L, int ld, int m, const double* __restrict__ x,
                                  double* y, int transpose) {
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= m) return;
  double s = 0.0;
  if (!transpose) {
    for (int c = lane; c <= r; c += 32) s += L[(size_t)r * ld + c] * x[c];
  } else {
    for (int c = r + lane; c < m; c += 32) s += L[(size_t)c * ld + r] * x[c];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[r] = s;
}

// out_i = scale_i * (base_i + sgn * rsD_i * (F_i . c)) ; warp per row
__global__ void f_dot_kernel(const double* __restrict__ F, int fpad, int m, int64_t n, const double* __restrict__ c,
                             const double* __restrict__ base, double sgn, const double* __restrict__ rsD,
                             const double* __restrict__ scale, double* out) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int k = lane; k < m; k += 32) s += F[(size_t)i * fpad + k] * c[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double v = base[i] + sgn * (rsD ? rsD[i] : 1.0) * s;
    out[i] = scale ? scale[i] * v : v;
  }
}

// Bernoulli-logit pieces at b (Eq. W_diag): W = p(1-p), v = W b + (y - p), and for the
// preconditioner Ginv = 1/(W' + 1/D), omega = D W' / (1 + D W'), W' = W exp(clip(corr, 4))
// (corr may be NULL), plus the log-likelihood terms y b - log(1 + e^b).
__global__ void lap_pointwise_kernel(const double* __restrict__ y, const double* __restrict__ b,
                                     const double* __restrict__ D, const double* __restrict__ corr, int64_t n,
                                     double* W, double* v, double* G, double* omega, double* rsD, double* ll) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double bi = b[i];
  const double p = 1.0 / (1.0 + exp(-bi));
  const double wi = p * (1.0 - p);
  W[i] = wi;
  v[i] = wi * bi + (y[i] - p);
  double wp = wi;
  if (corr) wp = wi * exp(fmin(fmax(corr[i], -4.0), 4.0));
  const double Di = D[i];
  G[i] = 1.0 / (wp + 1.0 / Di);
  omega[i] = Di * wp / (1.0 + Di * wp);
  rsD[i] = 1.0 / sqrt(Di);
  // log p(y|b) = y b - log(1 + e^b)
  ll[i] = y[i] * bi - (bi > 0 ? bi + log1p(exp(-bi)) : log1p(exp(bi)));
}

__global__ void axpby_kernel(int64_t n, const double* a, const double* x, const double* b, const double* y,
                             double* out, int mode) {
  // mode 0: out = x + a*y ; 1: out = x - a*y ; 2: out = x + (a)*out-prev  (p = z + beta p)
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = *a;
  if (mode == 0) out[i] = x[i] + s * y[i];
  else if (mode == 1) out[i] = x[i] - s * y[i];
  else out[i] = x[i] + s * out[i];
  (void)b;
}

__global__ void dot_stage1(const double* a, const double* b, int64_t n, double* partial) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += a[i] * (b ? b[i] : 1.0);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}
__global__ void dot_stage2(const double* partial, int np, double* out) {
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

// scalars: s[0]=rz, s[1]=pAp, s[2]=alpha, s[3]=rr, s[4]=rz_new, s[5]=beta
__global__ void pcg_alpha_kernel(double* s) { s[2] = s[0] / s[1]; }
__global__ void pcg_beta_kernel(double* s) {
  s[5] = s[4] / s[0];
  s[0] = s[4];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t lap_dot(const double* a, const double* b, int64_t n, double* partial, double* out, cudaStream_t s) {
  dot_stage1<<<256, 256, 0, s>>>(a, b, n, partial);
  dot_stage2<<<1, 256, 0, s>>>(partial, 256, out);
  return cudaGetLastError();
}

cudaError_t lap_ftv(const double* F, int fpad, int m, int64_t n, const double* v, double* partial, double* out,
                    cudaStream_t s) {
  const int nb = (int)((n + FT_ROWS - 1) / FT_ROWS);
  ftv_kernel<<<nb, 256, 0, s>>>(F, fpad, m, n, v, partial);
  col_reduce_kernel<<<blocks(m, 256), 256, 0, s>>>(partial, nb, fpad, m, out);
  return cudaGetLastError();
}

cudaError_t lap_spd_apply(const double* Linv, int ld, int m, const double* x, double* tmp, double* y, cudaStream_t s) {
  // y = (L L^T)^{-1} x = Linv^T (Linv x)
  lower_gemv_kernel<<<blocks(m, 8), 256, 0, s>>>(Linv, ld, m, x, tmp, 0);
  lower_gemv_kernel<<<blocks(m, 8), 256, 0, s>>>(Linv, ld, m, tmp, y, 1);
  return cudaGetLastError();
}

cudaError_t lap_matvec(const LapOps& o, const double* x, const double* diagW, double* out, cudaStream_t s) {
  bx_scaled_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.N, o.Acoef, o.rsD, o.n, o.mv, x, o.t);
  if (o.m > 0) {
    lap_ftv(o.F, o.fpad, o.m, o.n, o.t, o.partial, o.sm, s);
    lap_spd_apply(o.LinvC, o.ldl, o.m, o.sm, o.tmpm, o.cm, s);
    f_dot_kernel<<<blocks(o.n, 8), 256, 0, s>>>(o.F, o.fpad, o.m, o.n, o.cm, o.t, -1.0, nullptr, nullptr, o.t2);
  } else {
    cudaMemcpyAsync(o.t2, o.t, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  btx_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.ch_ptr, o.ch_row, o.ch_slot, o.Acoef, o.rsD, o.n, o.mv, o.t2, diagW,
                                              x, out);
  return cudaGetLastError();
}

cudaError_t lap_precond(const LapOps& o, const double* w, double* out, int* epoch, cudaStream_t s) {
  const unsigned grid = 152 * 4;
  // x = B^{-T} w
  cudaMemsetAsync(o.counter, 0, 2 * sizeof(unsigned long long), s);
  ++*epoch;
  if (o.mv > 0) {
    sptrsv_Bt_kernel<<<grid, 256, 0, s>>>(o.ch_ptr, o.ch_row, o.ch_slot, o.Acoef, o.n, o.mv, w, o.x1, o.flags,
                                          *epoch, o.counter, o.abort_flag, o.status);
  } else {
    cudaMemcpyAsync(o.x1, w, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  // e = G^{-1} (x + D^{-1/2} F C3^{-1} F^T D^{-1/2} G^{-1} x)
  if (o.m > 0) {
    f_dot_kernel<<<blocks(o.n, 8), 256, 0, s>>>(o.F, o.fpad, 0, o.n, o.cm, o.x1, 0.0, nullptr, o.Ginv, o.t);
    // t = x / G ; then t <- rsD * t for the F^T product
    f_dot_kernel<<<blocks(o.n, 8), 256, 0, s>>>(o.F, o.fpad, 0, o.n, o.cm, o.t, 0.0, nullptr, o.rsD, o.t2);
    lap_ftv(o.F, o.fpad, o.m, o.n, o.t2, o.partial, o.sm, s);
    lap_spd_apply(o.LinvC3, o.ldl, o.m, o.sm, o.tmpm, o.cm, s);
    f_dot_kernel<<<blocks(o.n, 8), 256, 0, s>>>(o.F, o.fpad, o.m, o.n, o.cm, o.x1, 1.0, o.rsD, o.Ginv, o.t);
  } else {
    f_dot_kernel<<<blocks(o.n, 8), 256, 0, s>>>(o.F, o.fpad, 0, o.n, o.cm, o.x1, 0.0, nullptr, o.Ginv, o.t);
  }
  // out = B^{-1} e
  ++*epoch;
  if (o.mv > 0) {
    sptrsv_B_kernel<<<grid, 256, 0, s>>>(o.N, o.Acoef, o.n, o.mv, o.t, out, o.flags, *epoch, o.counter + 2,
                                         o.abort_flag, o.status);
  } else {
    cudaMemcpyAsync(out, o.t, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

cudaError_t lap_pointwise(const double* y, const double* b, const double* D, const double* corr, int64_t n, double* W,
                          double* v, double* Gd, double* omega, double* rsD, double* ll, cudaStream_t s) {
  lap_pointwise_kernel<<<blocks(n, 256), 256, 0, s>>>(y, b, D, corr, n, W, v, Gd, omega, rsD, ll);
  return cudaGetLastError();
}

__global__ void recip_kernel(const double* a, int64_t n, double* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = 1.0 / a[i];
}
cudaError_t lap_recip(const double* a, int64_t n, double* out, cudaStream_t s) {
  recip_kernel<<<blocks(n, 256), 256, 0, s>>>(a, n, out);
  return cudaGetLastError();
}

cudaError_t lap_axpy(int64_t n, const double* scal, const double* x, const double* y, double* out, int mode,
                     cudaStream_t s) {
  axpby_kernel<<<blocks(n, 256), 256, 0, s>>>(n, scal, x, nullptr, y, out, mode);
  return cudaGetLastError();
}

cudaError_t lap_alpha(double* sc, cudaStream_t s) {
  pcg_alpha_kernel<<<1, 1, 0, s>>>(sc);
  return cudaGetLastError();
}
cudaError_t lap_beta(double* sc, cudaStream_t s) {
  pcg_beta_kernel<<<1, 1, 0, s>>>(sc);
  return cudaGetLastError();
}

}  // namespace vif
