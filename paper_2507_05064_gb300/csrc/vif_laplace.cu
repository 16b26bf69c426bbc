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
// The triangular solves with B and B^T are sync-free: rows are ordered by level (a
// row's level is one more than the deepest row it reads), grouped in steps of four
// rows of one level (eight lanes per row; one row with many terms gets the whole
// warp), and the steps are dealt round-robin to the warps of a cooperative launch.
// The output vector is filled with an all-ones bit pattern (a NaN that no arithmetic
// result takes) before the solve; a row reads its inputs by polling their values
// until they differ from that pattern, so the value is its own ready flag and no
// separate flag or fence is needed.  Every wait is bounded; a wait that runs out sets
// an abort flag that ends all waits, and the host reports VIF_ERR_TIMEOUT.
#include "vif_internal.cuh"

namespace vif {

constexpr int SPIN_LIMIT = 1 << 22;
constexpr unsigned long long TR_PENDING = ~0ull;

__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if (b == TR_PENDING) b = 0x7FF8000000000000ull;   // never publish the pending pattern
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}

// Value of *p once it has been written (NaN after an abort or a timeout).  Polls are
// back to back: a row's inputs land one L2 round trip apart at best, and backing off
// only lengthens the chain of levels (measured: 1.37 us per level of a pure chain with
// back-to-back polls, 2.06 us with a 64-512 ns backoff).  abort_flag[0] is the abort
// flag, abort_flag[1] the poll bound (0: SPIN_LIMIT); the flag is read every 64 polls,
// the bound at every poll once it is below that.
__device__ __noinline__ double wait_value(const double* p, int* abort_flag, int* status, int64_t row) {
  const int lim0 = ld_volatile(abort_flag + 1);
  const int lim = lim0 > 0 ? lim0 : SPIN_LIMIT;
  for (int it = 1;; ++it) {
    const unsigned long long b = ld_relaxed_u64(p);
    if (b != TR_PENDING) return __longlong_as_double((long long)b);
    if ((it & 63) == 0 || it >= lim) {
      if (ld_volatile(abort_flag)) return NAN;
      if (it >= lim) {
        atomicExch(abort_flag, 1);
        flag_status(status, ST_TIMEOUT, row);
        return NAN;
      }
    }
  }
}

// A step is four rows of one level, eight lanes per row, or (a "solo" step) one row
// with many terms and all 32 lanes; a schedule slot is {row, first term, end of
// terms, solo}, the four slots of a solo step all naming its row, padding slots
// {-1, 0, 0, 0}.  Lane `sub` of a row owns the terms sub, sub + lanes, ... of the
// row's sum  sum_t coef[t] * out[idx[t]].
constexpr int TR_LPR = 8;                  // lanes per row
constexpr int TR_RPS = 32 / TR_LPR;        // rows per warp step
static_assert(TR_RPS == LAP_TRSV_RPS, "schedule padding and rows per step differ");
constexpr int TR_MAXV = 6;                 // terms in flight per lane

struct TrsvTerms {
  int row, b, e, lanes, sub;
  bool solo;
  double rhs;
  int j[TR_MAXV];
  double c[TR_MAXV];
};

// issue the loads of a step's first TR_MAXV terms per lane and of its right-hand side
__device__ __forceinline__ void trsv_issue(TrsvTerms& T, int4 sl, int lane, const int32_t* __restrict__ idx,
                                           const double* __restrict__ coef, const double* __restrict__ rhs) {
  T.row = sl.x;
  T.b = sl.y;
  T.e = sl.z;
  T.solo = sl.w != 0;
  T.lanes = T.solo ? 32 : TR_LPR;
  T.sub = T.solo ? lane : lane % TR_LPR;
  T.rhs = (T.row >= 0 && T.sub == 0) ? rhs[T.row] : 0.0;
#pragma unroll
  for (int u = 0; u < TR_MAXV; ++u) {
    const int t = T.b + T.sub + u * T.lanes;
    T.j[u] = -1;
    T.c[u] = 0.0;
    if (t < T.e) {
      T.j[u] = idx[t];
      T.c[u] = coef[t];
    }
  }
}

// the row sum of a step whose first terms were issued by trsv_issue (all lanes of the
// warp take part: the partial sums are added by shuffles)
__device__ __forceinline__ double trsv_finish(const TrsvTerms& T, const int32_t* __restrict__ idx,
                                              const double* __restrict__ coef, const double* out, int* abort_flag,
                                              int* status) {
  double s = 0.0;
  unsigned long long v[TR_MAXV];
#pragma unroll
  for (int u = 0; u < TR_MAXV; ++u)
    if (T.j[u] >= 0) v[u] = ld_relaxed_u64(out + T.j[u]);
#pragma unroll
  for (int u = 0; u < TR_MAXV; ++u) {
    if (T.j[u] >= 0) {
      double x = __longlong_as_double((long long)v[u]);
      if (v[u] == TR_PENDING) x = wait_value(out + T.j[u], abort_flag, status, T.row);
      s = fma(T.c[u], x, s);
    }
  }
  // rows with more than lanes * TR_MAXV terms: further passes, one term per lane at a time
  for (int t = T.b + T.sub + TR_MAXV * T.lanes; t < T.e; t += T.lanes) {
    const int j = idx[t];
    const unsigned long long b = ld_relaxed_u64(out + j);
    const double x = b == TR_PENDING ? wait_value(out + j, abort_flag, status, T.row)
                                     : __longlong_as_double((long long)b);
    s = fma(coef[t], x, s);
  }
  if (T.solo) {
    s += __shfl_xor_sync(0xffffffffu, s, 16);
    s += __shfl_xor_sync(0xffffffffu, s, 8);
  }
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

// Both solves: out_r = rhs_r + sum over the terms t of row r of coef[t] * out[idx[t]],
// rows in level order.
//   B^{-1}: terms of row i are its neighbours (t = i m_v + k, idx = N, coef = A);
//   B^{-T}: terms of row j are its children (CSR), idx = child rows, coef = the
//           children's coefficients of j.
// Steps are dealt round-robin to the warps of a cooperative launch (all resident), each
// warp taking its steps in schedule order: a step only reads rows of earlier levels,
// i.e. of earlier steps, so the earliest unfinished step can always proceed.  While a
// step waits, the loads of the warp's next step are already in flight and the slots
// of the one after are being read.
__global__ __launch_bounds__(128) void sptrsv_kernel(const int4* __restrict__ sched, int64_t nsteps,
                                                     const int32_t* __restrict__ idx, const double* __restrict__ coef,
                                                     const double* __restrict__ rhs, double* out, int* abort_flag,
                                                     int* status) {
  const int lane = threadIdx.x & 31, g = lane / TR_LPR;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t step = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int4 pad = make_int4(-1, 0, 0, 0);
  TrsvTerms cur, nxt;
  trsv_issue(cur, step < nsteps ? sched[step * TR_RPS + g] : pad, lane, idx, coef, rhs);
  int4 sl1 = step + W < nsteps ? sched[(step + W) * TR_RPS + g] : pad;
  for (; step < nsteps; step += W) {
    trsv_issue(nxt, sl1, lane, idx, coef, rhs);
    sl1 = step + 2 * W < nsteps ? sched[(step + 2 * W) * TR_RPS + g] : pad;
    const double s = trsv_finish(cur, idx, coef, out, abort_flag, status);
    if (cur.sub == 0 && cur.row >= 0) st_relaxed_f64(out + cur.row, cur.rhs + s);
    cur = nxt;
  }
}

// ch_coef[p] = A_{ch_row[p]}[ch_slot[p]]: the coefficient of each child term, in CSR order
__global__ void child_coef_kernel(const int32_t* __restrict__ ch_row, const int32_t* __restrict__ ch_slot,
                                  const double* __restrict__ Acoef, int64_t nnz, int mv, double* ch_coef) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) ch_coef[p] = Acoef[(size_t)ch_row[p] * mv + ch_slot[p]];
}

__global__ void set_i32_kernel(int* p, int v) { *p = v; }

cudaError_t lap_set_wait_polls(int* abort_flag, int polls, cudaStream_t s) {
  set_i32_kernel<<<1, 1, 0, s>>>(abort_flag + 1, polls);
  return cudaGetLastError();
}

// t_i = (x_i - sum_k A_i[k] x_{N_k}) / sqrt(D_i); thread per row, four gathers in flight
__global__ void bx_scaled_kernel(const int32_t* __restrict__ N, const double* __restrict__ Acoef,
                                 const double* __restrict__ rsD, int64_t n, int mv, const double* __restrict__ x,
                                 double* t) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int q = (int)(i < mv ? i : mv);
  const int32_t* Ni = N + (size_t)i * mv;
  const double* Ai = Acoef + (size_t)i * mv;
  double s = x[i], s2 = 0.0;
  int k = 0;
  for (; k + 3 < q; k += 4) {
    const int j0 = Ni[k], j1 = Ni[k + 1], j2 = Ni[k + 2], j3 = Ni[k + 3];
    const double x0 = x[j0], x1 = x[j1], x2 = x[j2], x3 = x[j3];
    s = fma(-Ai[k], x0, s);
    s2 = fma(-Ai[k + 1], x1, s2);
    s = fma(-Ai[k + 2], x2, s);
    s2 = fma(-Ai[k + 3], x3, s2);
  }
  for (; k < q; ++k) s = fma(-Ai[k], x[Ni[k]], s);
  t[i] = (s + s2) * rsD[i];
}

// out_j = diagW_j x_j + u_j - sum_{(i,k) in ch(j)} A_i[k] u_i   (u = D^{-1/2} t2), over
// the steps of the B^T schedule (four rows of eight lanes, or one row with many
// children on the whole warp), so that rows with hundreds of children do not hold a
// single thread; nothing here waits, the level order is simply reused.
__global__ __launch_bounds__(256) void btx_kernel(const int4* __restrict__ sched, int64_t nsteps,
                                                  const int32_t* __restrict__ ch_row,
                                                  const double* __restrict__ ch_coef, const double* __restrict__ u,
                                                  const double* __restrict__ diagW, const double* __restrict__ x,
                                                  double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t step = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (step >= nsteps) return;
  const int4 sl = sched[step * TR_RPS + lane / TR_LPR];
  const bool solo = sl.w != 0;
  const int lanes = solo ? 32 : TR_LPR, sub = solo ? lane : lane % TR_LPR;
  double s = 0.0, s2 = 0.0;
  int t = sl.y + sub;
  for (; t + lanes < sl.z; t += 2 * lanes) {
    s = fma(ch_coef[t], u[ch_row[t]], s);
    s2 = fma(ch_coef[t + lanes], u[ch_row[t + lanes]], s2);
  }
  if (t < sl.z) s = fma(ch_coef[t], u[ch_row[t]], s);
  s += s2;
  if (solo) {
    s += __shfl_xor_sync(0xffffffffu, s, 16);
    s += __shfl_xor_sync(0xffffffffu, s, 8);
  }
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  const int j = sl.x;
  if (sub == 0 && j >= 0) out[j] = u[j] - s + (diagW ? diagW[j] * x[j] : 0.0);
}

// partial[b][c] = sum over the rows of block b of F[i][c] * v[i]   (c < m); one block
// per SM-sized slice of rows, one thread per column
__global__ void ftv_kernel(const double* __restrict__ F, int fpad, int m, int64_t n, int64_t rows_per_block,
                           const double* __restrict__ v, double* partial) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = (n < r0 + rows_per_block) ? n : r0 + rows_per_block;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    int64_t r = r0;
    for (; r + 1 < r1; r += 2) {
      s0 = fma(F[(size_t)r * fpad + c], v[r], s0);
      s1 = fma(F[(size_t)(r + 1) * fpad + c], v[r + 1], s1);
    }
    if (r < r1) s0 = fma(F[(size_t)r * fpad + c], v[r], s0);
    partial[(size_t)blockIdx.x * fpad + c] = s0 + s1;
  }
}
// out[c] = sum_b partial[b][c]: 32 columns per block, the 8 warps take every 8th partial
// and their sums are added in a fixed order
__global__ void col_reduce_kernel(const double* partial, int nb, int fpad, int m, double* out) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (c < m)
    for (int b = w; b < nb; b += 8) s += partial[(size_t)b * fpad + c];
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0 && c < m) {
    double t = sh[0][lane];
#pragma unroll
    for (int k = 1; k < 8; ++k) t += sh[k][lane];
    out[c] = t;
  }
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

// out_i = scale_i * (base_i + sgn * rsD_i * (F_i . c)), m > 0; thread per row, each
// thread reading its row in 32-byte pieces (c staged in shared memory)
constexpr int FD_THREADS = 128;
__global__ __launch_bounds__(FD_THREADS) void f_dot_kernel(const double* __restrict__ F, int fpad, int m, int64_t n,
                                                           const double* __restrict__ c,
                                                           const double* __restrict__ base, double sgn,
                                                           const double* __restrict__ rsD,
                                                           const double* __restrict__ scale, double* out) {
  extern __shared__ double cs[];
  const int m4 = (m + 3) & ~3;
  for (int k = threadIdx.x; k < m4; k += blockDim.x) cs[k] = k < m ? c[k] : 0.0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* row = F + (size_t)i * fpad;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int k = 0; k < m4; k += 4) {
    const double2 a = *reinterpret_cast<const double2*>(row + k);
    const double2 b = *reinterpret_cast<const double2*>(row + k + 2);
    s0 = fma(a.x, cs[k], s0);
    s1 = fma(a.y, cs[k + 1], s1);
    s2 = fma(b.x, cs[k + 2], s2);
    s3 = fma(b.y, cs[k + 3], s3);
  }
  const double s = (s0 + s1) + (s2 + s3);
  const double v = base[i] + sgn * (rsD ? rsD[i] : 1.0) * s;
  out[i] = scale ? scale[i] * v : v;
}

// out_i = a_i * b_i * x_i (b may be NULL)
__global__ void scale2_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              const double* __restrict__ x, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] * (b ? b[i] : 1.0) * x[i];
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
  const int64_t rpb = (n + LAP_FT_BLOCKS - 1) / LAP_FT_BLOCKS;
  const int nb = (int)((n + rpb - 1) / rpb);
  ftv_kernel<<<nb, 256, 0, s>>>(F, fpad, m, n, rpb, v, partial);
  col_reduce_kernel<<<blocks(m, 32), 256, 0, s>>>(partial, nb, fpad, m, out);
  return cudaGetLastError();
}

cudaError_t lap_spd_apply(const double* Linv, int ld, int m, const double* x, double* tmp, double* y, cudaStream_t s) {
  // y = (L L^T)^{-1} x = Linv^T (Linv x)
  lower_gemv_kernel<<<blocks(m, 8), 256, 0, s>>>(Linv, ld, m, x, tmp, 0);
  lower_gemv_kernel<<<blocks(m, 8), 256, 0, s>>>(Linv, ld, m, tmp, y, 1);
  return cudaGetLastError();
}

static void f_dot(const LapOps& o, const double* c, const double* base, double sgn, const double* rsD,
                  const double* scale, double* out, cudaStream_t s) {
  const size_t smem = (size_t)((o.m + 3) & ~3) * sizeof(double);
  f_dot_kernel<<<blocks(o.n, FD_THREADS), FD_THREADS, smem, s>>>(o.F, o.fpad, o.m, o.n, c, base, sgn, rsD, scale,
                                                                  out);
}

cudaError_t lap_matvec(const LapOps& o, const double* x, const double* diagW, double* out, cudaStream_t s) {
  // t = D^{-1/2} B x ; u = D^{-1/2} (t - F C^{-1} F^T t) ; out = W x + B^T u
  bx_scaled_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.N, o.Acoef, o.rsD, o.n, o.mv, x, o.t);
  if (o.m > 0) {
    lap_ftv(o.F, o.fpad, o.m, o.n, o.t, o.partial, o.sm, s);
    lap_spd_apply(o.LinvC, o.ldl, o.m, o.sm, o.tmpm, o.cm, s);
    f_dot(o, o.cm, o.t, -1.0, nullptr, o.rsD, o.t2, s);
  } else {
    scale2_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.rsD, nullptr, o.t, o.t2);
  }
  btx_kernel<<<blocks(o.nsteps_rev, 8), 256, 0, s>>>(o.sched_rev, o.nsteps_rev, o.ch_row, o.ch_coef, o.t2, diagW,
                                                        x, out);
  return cudaGetLastError();
}

cudaError_t lap_child_coef(const LapOps& o, double* ch_coef, cudaStream_t s) {
  if (o.nnz > 0)
    child_coef_kernel<<<blocks(o.nnz, 256), 256, 0, s>>>(o.ch_row, o.ch_slot, o.Acoef, o.nnz, o.mv, ch_coef);
  return cudaGetLastError();
}

// CTAs per SM of a triangular solve (1, 2 and 4 measured within 5% of one another at
// n = 2e5).  The launch is cooperative (every CTA resident at once), which the
// round-robin step assignment needs.
constexpr int TRSV_CTAS_PER_SM = 2;

static cudaError_t launch_trsv(const int4* sched, int64_t nsteps, const int32_t* idx, const double* coef,
                               const double* rhs, double* out, int* abort_flag, int* status, cudaStream_t s) {
  static int grid_of_dev[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int& grid = grid_of_dev[dev & 63];
  if (grid == 0) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sptrsv_kernel, 128, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    grid = sms * (per_sm < TRSV_CTAS_PER_SM ? per_sm : TRSV_CTAS_PER_SM);
  }
  void* args[] = {(void*)&sched, (void*)&nsteps, (void*)&idx, (void*)&coef, (void*)&rhs, (void*)&out,
                  (void*)&abort_flag, (void*)&status};
  return cudaLaunchCooperativeKernel((const void*)sptrsv_kernel, dim3(grid), dim3(128), args, 0, s);
}

cudaError_t lap_precond(const LapOps& o, const double* w, double* out, cudaStream_t s) {
  // x = B^{-T} w
  if (o.mv > 0) {
    cudaMemsetAsync(o.x1, 0xFF, (size_t)o.n * sizeof(double), s);
    cudaError_t e = launch_trsv(o.sched_rev, o.nsteps_rev, o.ch_row, o.ch_coef, w, o.x1, o.abort_flag, o.status, s);
    if (e != cudaSuccess) return e;
  } else {
    cudaMemcpyAsync(o.x1, w, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  // e = G^{-1} (x + D^{-1/2} F C3^{-1} F^T D^{-1/2} G^{-1} x)
  if (o.m > 0) {
    scale2_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.rsD, o.Ginv, o.x1, o.t2);
    lap_ftv(o.F, o.fpad, o.m, o.n, o.t2, o.partial, o.sm, s);
    lap_spd_apply(o.LinvC3, o.ldl, o.m, o.sm, o.tmpm, o.cm, s);
    f_dot(o, o.cm, o.x1, 1.0, o.rsD, o.Ginv, o.t, s);
  } else {
    scale2_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.Ginv, nullptr, o.x1, o.t);
  }
  // out = B^{-1} e
  if (o.mv > 0) {
    cudaMemsetAsync(out, 0xFF, (size_t)o.n * sizeof(double), s);
    cudaError_t e = launch_trsv(o.sched_fwd, o.nsteps_fwd, o.N, o.Acoef, o.t, out, o.abort_flag, o.status, s);
    if (e != cudaSuccess) return e;
  } else {
    cudaMemcpyAsync(out, o.t, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pieces of the VIF-Laplace likelihood with the preconditioned SLQ log-determinant
// (Eq. log_det_VIFLA, Eq. slq_v1): probe draws z ~ N(0, P) by the recipe of Sec. 4.3
// and the log-determinants of App. E.1.
// ---------------------------------------------------------------------------

// u_i = sqrt(D_i) eps2_i ;  v_i = sqrt(W'_i) eps3_i with W' = W exp(clip(corr, 4)) (corr may be NULL)
__global__ void probe_prep_kernel(int64_t n, const double* __restrict__ D, const double* __restrict__ W,
                                  const double* __restrict__ corr, const double* __restrict__ eps2,
                                  const double* __restrict__ eps3, double* u, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double wp = W[i];
  if (corr) wp *= exp(fmin(fmax(corr[i], -4.0), 4.0));
  u[i] = sqrt(D[i]) * eps2[i];
  v[i] = sqrt(wp) * eps3[i];
}

__global__ void vec_add_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}

// partial[b] = sum over this block's share of sgn * log(x[i * stride])
__global__ void logsum_stage1(const double* x, int64_t n, int64_t stride, double sgn, double* partial) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += log(x[i * stride]);
  sh[threadIdx.x] = sgn * v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

cudaError_t lap_log_sum(const double* x, int64_t n, int64_t stride, double sgn, double* partial, double* out,
                        cudaStream_t s) {
  logsum_stage1<<<256, 256, 0, s>>>(x, n, stride, sgn, partial);
  dot_stage2<<<1, 256, 0, s>>>(partial, 256, out);
  return cudaGetLastError();
}

cudaError_t lap_probe_prep(int64_t n, const double* D, const double* W, const double* corr, const double* eps2,
                           const double* eps3, double* u, double* v, cudaStream_t s) {
  probe_prep_kernel<<<blocks(n, 256), 256, 0, s>>>(n, D, W, corr, eps2, eps3, u, v);
  return cudaGetLastError();
}

cudaError_t lap_vec_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  vec_add_kernel<<<blocks(n, 256), 256, 0, s>>>(n, a, b, out);
  return cudaGetLastError();
}

// out = B^{-1} rhs (level-scheduled solve)
cudaError_t lap_solve_B(const LapOps& o, const double* rhs, double* out, cudaStream_t s) {
  if (o.mv == 0) return cudaMemcpyAsync(out, rhs, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaMemsetAsync(out, 0xFF, (size_t)o.n * sizeof(double), s);
  if (e != cudaSuccess) return e;
  return launch_trsv(o.sched_fwd, o.nsteps_fwd, o.N, o.Acoef, rhs, out, o.abort_flag, o.status, s);
}

// out = B^T u
cudaError_t lap_apply_Bt(const LapOps& o, const double* u, double* out, cudaStream_t s) {
  btx_kernel<<<blocks(o.nsteps_rev, 8), 256, 0, s>>>(o.sched_rev, o.nsteps_rev, o.ch_row, o.ch_coef, u, nullptr,
                                                      nullptr, out);
  return cudaGetLastError();
}

// out_i = base_i + rows_i . c  (rows: n x m, leading dimension ld, 16-byte aligned rows)
cudaError_t lap_rows_dot_add(const double* rows, int ld, int m, int64_t n, const double* c, const double* base,
                             double* out, cudaStream_t s) {
  const size_t smem = (size_t)((m + 3) & ~3) * sizeof(double);
  f_dot_kernel<<<blocks(n, FD_THREADS), FD_THREADS, smem, s>>>(rows, ld, m, n, c, base, 1.0, nullptr, nullptr, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FITC preconditioner (Sec. 4.3, App. E.2) with the system form of Eq. pcls2,
//   (W^{-1} + Sigma_dagger) x = v,   Sigma_dagger x = B^{-1} D B^{-T} x + A^T A x,
//   P = D_V + A^T A,   D_V = diag(sigma_1^2 - |a_i|^2) + W^{-1},
// its inducing points being those of the VIF (A^T A = Sigma_mn^T Sigma_m^{-1} Sigma_mn).
// Solves by Woodbury with the whitened M_V = I + A D_V^{-1} A^T (m x m), draws by
// D_V^{1/2} eps2 + A^T eps1.
// ---------------------------------------------------------------------------

// Apad = A with rows zero-padded from mpad to fpad columns (columns >= m zero); anorm2_i = |a_i|^2
__global__ void fitc_prepare_kernel(const double* __restrict__ A, int mpad, int m, int64_t n, int fpad, double* Apad,
                                    double* anorm2) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int k = lane; k < fpad; k += 32) {
    const double v = k < m ? A[(size_t)i * mpad + k] : 0.0;
    Apad[(size_t)i * fpad + k] = v;
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) anorm2[i] = s;
}

__global__ void fitc_dv_kernel(int64_t n, double var, const double* __restrict__ anorm2, const double* __restrict__ W,
                               double* dvinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dvinv[i] = 1.0 / (var - anorm2[i] + 1.0 / W[i]);
}

// out_i = a_i + x_i / d_i   (d may be NULL: out = a + 0)
__global__ void add_div_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ x,
                               const double* __restrict__ d, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + (d ? x[i] / d[i] : 0.0);
}

__global__ void div_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ d, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] / d[i];
}

// z_i = sqrt(D_V,i) eps2_i
__global__ void fitc_probe_kernel(int64_t n, const double* __restrict__ dvinv, const double* __restrict__ eps2,
                                  double* z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = eps2[i] / sqrt(dvinv[i]);
}

cudaError_t lap_fitc_prepare_A(const double* A, int mpad, int m, int64_t n, int fpad, double* Apad, double* anorm2,
                               cudaStream_t s) {
  fitc_prepare_kernel<<<blocks(n, 8), 256, 0, s>>>(A, mpad, m, n, fpad, Apad, anorm2);
  return cudaGetLastError();
}

cudaError_t lap_fitc_dv(int64_t n, double var, const double* anorm2, const double* W, double* dvinv, cudaStream_t s) {
  fitc_dv_kernel<<<blocks(n, 256), 256, 0, s>>>(n, var, anorm2, W, dvinv);
  return cudaGetLastError();
}

cudaError_t lap_div(int64_t n, const double* x, const double* d, double* out, cudaStream_t s) {
  div_kernel<<<blocks(n, 256), 256, 0, s>>>(n, x, d, out);
  return cudaGetLastError();
}

// out = Sigma_dagger x (+ x / Wd when Wd is given) = B^{-1}(D o B^{-T} x) + A^T A x (+ W^{-1} x)
cudaError_t lap_sigma_matvec(const LapOps& o, const double* x, const double* Wd, double* out, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (o.mv > 0) {
    if ((e = cudaMemsetAsync(o.t, 0xFF, (size_t)o.n * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = launch_trsv(o.sched_rev, o.nsteps_rev, o.ch_row, o.ch_coef, x, o.t, o.abort_flag, o.status, s)) !=
        cudaSuccess)
      return e;
    scale2_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.D, nullptr, o.t, o.t2);
    if ((e = lap_solve_B(o, o.t2, o.x1, s)) != cudaSuccess) return e;
  } else {
    scale2_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.D, nullptr, x, o.x1);
  }
  add_div_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.x1, x, Wd, o.t);
  if (o.m > 0) {
    lap_ftv(o.A, o.mpad, o.m, o.n, x, o.partial, o.cm, s);
    return lap_rows_dot_add(o.A, o.mpad, o.m, o.n, o.cm, o.t, out, s);
  }
  return cudaMemcpyAsync(out, o.t, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// out = P^{-1} w = D_V^{-1} (w - A^T M_V^{-1} A D_V^{-1} w)
cudaError_t lap_precond_fitc(const LapOps& o, const double* w, double* out, cudaStream_t s) {
  scale2_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.dvinv, nullptr, w, o.t2);
  if (o.m == 0) return cudaMemcpyAsync(out, o.t2, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  lap_ftv(o.A, o.mpad, o.m, o.n, o.t2, o.partial, o.sm, s);
  lap_spd_apply(o.LinvMV, o.ldl, o.m, o.sm, o.tmpm, o.cm, s);
  const size_t smem = (size_t)((o.m + 3) & ~3) * sizeof(double);
  f_dot_kernel<<<blocks(o.n, FD_THREADS), FD_THREADS, smem, s>>>(o.A, o.mpad, o.m, o.n, o.cm, w, -1.0, nullptr,
                                                                  o.dvinv, out);
  return cudaGetLastError();
}

cudaError_t lap_system_matvec(const LapOps& o, const double* x, double* out, cudaStream_t s) {
  return o.kind == LAP_FITC ? lap_sigma_matvec(o, x, o.W, out, s) : lap_matvec(o, x, o.W, out, s);
}

cudaError_t lap_system_precond(const LapOps& o, const double* w, double* out, cudaStream_t s) {
  return o.kind == LAP_FITC ? lap_precond_fitc(o, w, out, s) : lap_precond(o, w, out, s);
}

// z = D_V^{1/2} eps2 + A^T eps1  ~ N(0, P) for the FITC preconditioner
cudaError_t lap_fitc_probe(const LapOps& o, const double* eps1, const double* eps2, double* z, cudaStream_t s) {
  fitc_probe_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.n, o.dvinv, eps2, o.t);
  if (o.m == 0) return cudaMemcpyAsync(z, o.t, o.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  return lap_rows_dot_add(o.A, o.mpad, o.m, o.n, eps1, o.t, z, s);
}

// acc_i += x_i^2 ;  out_i = x_i + a y_i
__global__ void sq_acc_kernel(int64_t n, const double* __restrict__ x, double* acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] = fma(x[i], x[i], acc[i]);
}
__global__ void axpy_host_kernel(int64_t n, double a, const double* __restrict__ x, const double* __restrict__ y,
                                 double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fma(a, y[i], x[i]);
}

cudaError_t lap_sq_accumulate(int64_t n, const double* x, double* acc, cudaStream_t s) {
  sq_acc_kernel<<<blocks(n, 256), 256, 0, s>>>(n, x, acc);
  return cudaGetLastError();
}

cudaError_t lap_axpy_host(int64_t n, double a, const double* x, const double* y, double* out, cudaStream_t s) {
  axpy_host_kernel<<<blocks(n, 256), 256, 0, s>>>(n, a, x, y, out);
  return cudaGetLastError();
}

// t = D^{-1/2} B x
cudaError_t lap_bx_scaled(const LapOps& o, const double* x, double* t, cudaStream_t s) {
  bx_scaled_kernel<<<blocks(o.n, 256), 256, 0, s>>>(o.N, o.Acoef, o.rsD, o.n, o.mv, x, t);
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

// ---------------------------------------------------------------------------
// Gradient of the VIF-Laplace likelihood by stochastic trace estimation (Sec. 4.1,
// App. B, App. D): the probe estimate of dL/db~ and the bilinear forms whose central
// differences in theta give the traces.
// ---------------------------------------------------------------------------

// With dhat_i = (1/l) sum_j U[j][i] Y[j][i] (U, Y: l x n, probe-major) and the Bernoulli-logit
// W = p (1 - p), dW/db = p (1 - p)(1 - 2p), p = sigmoid(b_i):
//   form 0 (VIFDU, dhat ~ (W + Sigma_dagger^{-1})^{-1}_ii):  g_i = 1/2 dW/db dhat_i
//   form 1 (FITC, dhat ~ (W^{-1} + Sigma_dagger)^{-1}_ii):   g_i = 1/2 dW/db (1 - dhat_i / W) / W
__global__ void ste_diag_kernel(int64_t n, int l, const double* __restrict__ U, const double* __restrict__ Y,
                                const double* __restrict__ b, int form, double* g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s0 = 0.0, s1 = 0.0;
  int j = 0;
  for (; j + 1 < l; j += 2) {
    s0 = fma(U[(size_t)j * n + i], Y[(size_t)j * n + i], s0);
    s1 = fma(U[(size_t)(j + 1) * n + i], Y[(size_t)(j + 1) * n + i], s1);
  }
  if (j < l) s0 = fma(U[(size_t)j * n + i], Y[(size_t)j * n + i], s0);
  const double p = 1.0 / (1.0 + exp(-b[i]));
  const double w = p * (1.0 - p), dw = w * (1.0 - 2.0 * p), dhat = (s0 + s1) / l;
  g[i] = form == 0 ? 0.5 * dw * dhat : 0.5 * dw * (1.0 - dhat / w) / w;
}

// per block: sum a_i x_i, sum c_i x_i and (t != NULL) sum t_i^2 w_i d_i, into partial[k * 256 + block]
__global__ __launch_bounds__(256) void forms_stage1(const double* __restrict__ a, const double* __restrict__ c,
                                                    const double* __restrict__ x, const double* __restrict__ t,
                                                    const double* __restrict__ w, const double* __restrict__ d,
                                                    int64_t n, double* partial) {
  __shared__ double sh[3][256];
  double v0 = 0.0, v1 = 0.0, v2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = x[i];
    v0 = fma(a[i], xi, v0);
    v1 = fma(c[i], xi, v1);
    if (t) {
      const double ti = t[i];
      v2 = fma(ti * ti, w[i] * d[i], v2);
    }
  }
  sh[0][threadIdx.x] = v0;
  sh[1][threadIdx.x] = v1;
  sh[2][threadIdx.x] = v2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sh[0][0];
    partial[256 + blockIdx.x] = sh[1][0];
    partial[512 + blockIdx.x] = sh[2][0];
  }
}

// block k sums partial[k * 256 .. k * 256 + 255] into *out_k (out_k may be NULL)
__global__ void forms_stage2(const double* partial, double* out0, double* out1, double* out2) {
  double* out = blockIdx.x == 0 ? out0 : (blockIdx.x == 1 ? out1 : out2);
  if (!out) return;
  __shared__ double sh[256];
  sh[threadIdx.x] = partial[blockIdx.x * 256 + threadIdx.x];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t lap_ste_diag(int64_t n, int l, const double* U, const double* Y, const double* b, int form, double* g,
                         cudaStream_t s) {
  ste_diag_kernel<<<blocks(n, 256), 256, 0, s>>>(n, l, U, Y, b, form, g);
  return cudaGetLastError();
}

cudaError_t lap_grad_forms(int64_t n, const double* a, const double* c, const double* x, const double* t,
                           const double* w, const double* d, double* partial, double* out0, double* out1,
                           double* out2, cudaStream_t s) {
  forms_stage1<<<256, 256, 0, s>>>(a, c, x, t, w, d, n, partial);
  forms_stage2<<<3, 256, 0, s>>>(partial, out0, out1, out2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Many right-hand sides at once: the L probes of the SLQ (Sec. 4.1) share every operator
// application of their CG.  Block vectors are n x L, row-major (value j of row i at
// i L + j, L <= LAP_MR_MAXL); each kernel acts on every column as the single-vector kernel
// above acts on its vector, and nothing mixes columns.  The triangular solves keep the
// value-as-flag protocol over the rows in level order; their work is split so that few
// float64 instructions (64 cycles each per warp on this part) lie on the chain of levels.
// ---------------------------------------------------------------------------
constexpr int MR_CW = 8;              // columns of one solve task
constexpr int MR_TS = 32 / MR_CW;     // lanes sharing one column's terms
constexpr int MR_TG = 8;              // terms per lane with loads in flight

// A task is one row and one chunk of MR_CW columns: lane (u, h) = (lane % MR_CW, lane / MR_CW)
// sums the terms h, h + MR_TS, ... of column c MR_CW + u, and the MR_TS partial sums are added
// by two shuffles.  Tasks are numbered (position of the row in level order) * nch + chunk and
// dealt round-robin to the warps of a cooperative launch; a task reads only its own chunk of
// rows of earlier levels, i.e. of earlier tasks, so the earliest unfinished task can always
// proceed.  Each chunk is a solve of its own, and chunks of consecutive levels overlap.
__global__ __launch_bounds__(128) void mr_sptrsv_kernel(const int4* __restrict__ ord, int64_t nrows,
                                                        const int32_t* __restrict__ idx,
                                                        const double* __restrict__ coef,
                                                        const double* __restrict__ rhs, double* out, int L, int nch,
                                                        int* abort_flag, int* status) {
  const int lane = threadIdx.x & 31, u = lane % MR_CW, h = lane / MR_CW;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t ntask = nrows * nch;
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < ntask; task += W) {
    const int64_t k = task / nch;
    const int c = (int)(task - k * nch);
    const int4 sl = ord[k];
    const int col = c * MR_CW + u;
    const bool on = col < L;
    double acc = 0.0;
    for (int t0 = sl.y + h; t0 < sl.z; t0 += MR_TG * MR_TS) {
      int jj[MR_TG];
      double cf[MR_TG];
      unsigned long long v[MR_TG];
#pragma unroll
      for (int q = 0; q < MR_TG; ++q) {
        const int t = t0 + q * MR_TS;
        jj[q] = t < sl.z ? idx[t] : -1;
        cf[q] = t < sl.z ? coef[t] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < MR_TG; ++q)
        if (on && jj[q] >= 0) v[q] = ld_relaxed_u64(out + (size_t)jj[q] * L + col);
#pragma unroll
      for (int q = 0; q < MR_TG; ++q)
        if (on && jj[q] >= 0) {
          const double* src = out + (size_t)jj[q] * L + col;
          const double x = v[q] == TR_PENDING ? wait_value(src, abort_flag, status, sl.x)
                                               : __longlong_as_double((long long)v[q]);
          acc = fma(cf[q], x, acc);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, MR_CW);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2 * MR_CW);
    if (h == 0 && on) {
      const size_t e = (size_t)sl.x * L + col;
      st_relaxed_f64(out + e, rhs[e] + acc);
    }
  }
}

// t[i][j] = (x[i][j] - sum_k A_i[k] x[N_k][j]) / sqrt(D_i)
__global__ void mr_bx_scaled_kernel(const int32_t* __restrict__ N, const double* __restrict__ Acoef,
                                    const double* __restrict__ rsD, int64_t n, int mv, int L,
                                    const double* __restrict__ x, double* t) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * L) return;
  const int64_t i = e / L;
  const int j = (int)(e - i * L);
  const int q = (int)(i < mv ? i : mv);
  const int32_t* Ni = N + (size_t)i * mv;
  const double* Ai = Acoef + (size_t)i * mv;
  double s = x[e], s2 = 0.0;
  int k = 0;
  for (; k + 1 < q; k += 2) {
    s = fma(-Ai[k], x[(size_t)Ni[k] * L + j], s);
    s2 = fma(-Ai[k + 1], x[(size_t)Ni[k + 1] * L + j], s2);
  }
  if (k < q) s = fma(-Ai[k], x[(size_t)Ni[k] * L + j], s);
  t[e] = (s + s2) * rsD[i];
}

// out[r][j] = diagW_r x[r][j] + u[r][j] - sum over the children c of r of A_c[slot] u[c][j]  (CSR)
__global__ void mr_btx_kernel(const int32_t* __restrict__ ch_ptr, const int32_t* __restrict__ ch_row,
                              const double* __restrict__ ch_coef, int64_t n, int L, const double* __restrict__ u,
                              const double* __restrict__ diagW, const double* __restrict__ x, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * L) return;
  const int64_t r = e / L;
  const int j = (int)(e - r * L);
  double s = 0.0, s2 = 0.0;
  int p = ch_ptr[r];
  const int pe = ch_ptr[r + 1];
  for (; p + 1 < pe; p += 2) {
    s = fma(ch_coef[p], u[(size_t)ch_row[p] * L + j], s);
    s2 = fma(ch_coef[p + 1], u[(size_t)ch_row[p + 1] * L + j], s2);
  }
  if (p < pe) s = fma(ch_coef[p], u[(size_t)ch_row[p] * L + j], s);
  out[e] = u[e] - (s + s2) + (diagW ? diagW[r] * x[e] : 0.0);
}

// partial[b][c][j] = sum over the rows r of slice b of F[r][c] T[r][j]: shared-memory chunks of
// 16 rows, 128 columns c per pass, each thread 8 c x 4 j products (j fastest across threads)
constexpr int MR_FT_ROWS = 16;
constexpr int MR_FT_CB = 128;
__global__ __launch_bounds__(256) void mr_ftv_kernel(const double* __restrict__ F, int fpad, int m, int64_t n,
                                                     int64_t rows_per_block, const double* __restrict__ T, int L,
                                                     double* partial) {
  __shared__ double Fs[MR_FT_ROWS][MR_FT_CB];
  __shared__ double Ts[MR_FT_ROWS][LAP_MR_MAXL];
  const int tj = threadIdx.x & 15, tc = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = (n < r0 + rows_per_block) ? n : r0 + rows_per_block;
  for (int cb = 0; cb < m; cb += MR_FT_CB) {
    double acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t rr = r0; rr < r1; rr += MR_FT_ROWS) {
      for (int e = threadIdx.x; e < MR_FT_ROWS * MR_FT_CB; e += blockDim.x) {
        const int rl = e / MR_FT_CB, cl = e % MR_FT_CB;
        const int64_t r = rr + rl;
        const int c = cb + cl;
        Fs[rl][cl] = (r < r1 && c < m) ? F[(size_t)r * fpad + c] : 0.0;
      }
      for (int e = threadIdx.x; e < MR_FT_ROWS * LAP_MR_MAXL; e += blockDim.x) {
        const int rl = e / LAP_MR_MAXL, jl = e % LAP_MR_MAXL;
        const int64_t r = rr + rl;
        Ts[rl][jl] = (r < r1 && jl < L) ? T[(size_t)r * L + jl] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int rl = 0; rl < MR_FT_ROWS; ++rl) {
        double f[8], tv[4];
#pragma unroll
        for (int a = 0; a < 8; ++a) f[a] = Fs[rl][tc + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) tv[b] = Ts[rl][tj + 16 * b];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(f[a], tv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = cb + tc + 16 * a, j = tj + 16 * b;
        if (c < m && j < L) partial[((size_t)blockIdx.x * fpad + c) * L + j] = acc[a][b];
      }
  }
}

// out[c][j] = sum_b partial[b][c][j], the slices added in a fixed order
__global__ void mr_col_reduce_kernel(const double* __restrict__ partial, int nb, int fpad, int m, int L,
                                     double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * L) return;
  const int c = e / L, j = e % L;
  double s0 = 0.0, s1 = 0.0;
  int b = 0;
  for (; b + 1 < nb; b += 2) {
    s0 += partial[((size_t)b * fpad + c) * L + j];
    s1 += partial[((size_t)(b + 1) * fpad + c) * L + j];
  }
  if (b < nb) s0 += partial[((size_t)b * fpad + c) * L + j];
  out[e] = s0 + s1;
}

// Y = Lm X (lower, m x m, leading dimension ld) or Y = Lm^T X; X, Y: m x L
__global__ void mr_lower_gemm_kernel(const double* __restrict__ Lm, int ld, int m, int L, const double* __restrict__ X,
                                     double* Y, int transpose) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * L) return;
  const int r = e / L, j = e % L;
  double s0 = 0.0, s1 = 0.0;
  if (!transpose) {
    int c = 0;
    for (; c + 1 <= r; c += 2) {
      s0 = fma(Lm[(size_t)r * ld + c], X[(size_t)c * L + j], s0);
      s1 = fma(Lm[(size_t)r * ld + c + 1], X[(size_t)(c + 1) * L + j], s1);
    }
    if (c <= r) s0 = fma(Lm[(size_t)r * ld + c], X[(size_t)c * L + j], s0);
  } else {
    int c = r;
    for (; c + 1 < m; c += 2) {
      s0 = fma(Lm[(size_t)c * ld + r], X[(size_t)c * L + j], s0);
      s1 = fma(Lm[(size_t)(c + 1) * ld + r], X[(size_t)(c + 1) * L + j], s1);
    }
    if (c < m) s0 = fma(Lm[(size_t)c * ld + r], X[(size_t)c * L + j], s0);
  }
  Y[e] = s0 + s1;
}

// out[i][j] = scale_i (base[i][j] + sgn rsD_i sum_c F[i][c] Y[c][j]); 64 rows x 64 columns per
// block in chunks of 32 c, each thread 4 rows x 4 columns (j fastest across threads)
__global__ __launch_bounds__(256) void mr_f_dot_kernel(const double* __restrict__ F, int fpad, int m, int64_t n, int L,
                                                       const double* __restrict__ Y, const double* __restrict__ base,
                                                       double sgn, const double* __restrict__ rsD,
                                                       const double* __restrict__ scale, double* out) {
  __shared__ double Fs[32][65];
  __shared__ double Ys[32][LAP_MR_MAXL];
  const int tj = threadIdx.x & 15, tr = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < m; k0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
      const int rl = e / 32, kk = e % 32;
      const int64_t i = i0 + rl;
      const int k = k0 + kk;
      Fs[kk][rl] = (i < n && k < m) ? F[(size_t)i * fpad + k] : 0.0;
    }
    for (int e = threadIdx.x; e < 32 * LAP_MR_MAXL; e += blockDim.x) {
      const int kk = e / LAP_MR_MAXL, jl = e % LAP_MR_MAXL;
      const int k = k0 + kk;
      Ys[kk][jl] = (k < m && jl < L) ? Y[(size_t)k * L + jl] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      double f[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) f[a] = Fs[kk][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) y[b] = Ys[kk][tj + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(f[a], y[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + tr + 16 * a;
    if (i >= n) continue;
    const double rs = rsD ? rsD[i] : 1.0;
    const double sc = scale ? scale[i] : 1.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = tj + 16 * b;
      if (j < L) {
        const size_t e = (size_t)i * L + j;
        out[e] = sc * (base[e] + sgn * rs * acc[a][b]);
      }
    }
  }
}

// out[i][j] = a_i (b_i) x[i][j]  (b may be NULL)
__global__ void mr_scale2_kernel(int64_t n, int L, const double* __restrict__ a, const double* __restrict__ b,
                                 const double* __restrict__ x, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * L) return;
  const int64_t i = e / L;
  out[e] = a[i] * (b ? b[i] : 1.0) * x[e];
}

// partial[blk][j] = sum over this block's rows of a[i][j] b[i][j] (b may be NULL: a alone)
__global__ __launch_bounds__(256) void mr_dot_stage1(const double* __restrict__ a, const double* __restrict__ b,
                                                     int64_t n, int L, double* partial) {
  __shared__ double sh[256];
  const int rpb = 256 / L;
  const int j = threadIdx.x % L, r0 = threadIdx.x / L;
  double v = 0.0;
  if (r0 < rpb)
    for (int64_t i = (int64_t)blockIdx.x * rpb + r0; i < n; i += (int64_t)gridDim.x * rpb) {
      const size_t e = (size_t)i * L + j;
      v = b ? fma(a[e], b[e], v) : v + a[e];
    }
  sh[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < L) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += sh[r * L + threadIdx.x];
    partial[(size_t)blockIdx.x * L + threadIdx.x] = s;
  }
}
__global__ void mr_dot_stage2(const double* __restrict__ partial, int nb, int L, double* out) {
  const int j = threadIdx.x;
  if (j >= L) return;
  double s0 = 0.0, s1 = 0.0;
  int b = 0;
  for (; b + 1 < nb; b += 2) {
    s0 += partial[(size_t)b * L + j];
    s1 += partial[(size_t)(b + 1) * L + j];
  }
  if (b < nb) s0 += partial[(size_t)b * L + j];
  out[j] = s0 + s1;
}

// per column: alpha_j = rz_j / pAp_j (0 for a finished column)
__global__ void mr_alpha_kernel(int L, const int* __restrict__ active, const double* __restrict__ rz,
                                const double* __restrict__ pAp, double* alpha) {
  const int j = threadIdx.x;
  if (j < L) alpha[j] = active[j] ? rz[j] / pAp[j] : 0.0;
}
// per column: beta_j = rz_new_j / rz_j and rz_j = rz_new_j (0 and unchanged for a finished column)
__global__ void mr_beta_kernel(int L, const int* __restrict__ active, double* rz, const double* __restrict__ rznew,
                               double* beta) {
  const int j = threadIdx.x;
  if (j >= L) return;
  if (active[j]) {
    beta[j] = rznew[j] / rz[j];
    rz[j] = rznew[j];
  } else {
    beta[j] = 0.0;
  }
}
// x += alpha_j p ;  r -= alpha_j Ap
__global__ void mr_update_xr_kernel(int64_t n, int L, const double* __restrict__ alpha, const double* __restrict__ p,
                                    const double* __restrict__ Ap, double* x, double* r) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * L) return;
  const double a = alpha[e % L];
  x[e] = fma(a, p[e], x[e]);
  r[e] = fma(-a, Ap[e], r[e]);
}
// p = z + beta_j p
__global__ void mr_update_p_kernel(int64_t n, int L, const double* __restrict__ beta, const double* __restrict__ z,
                                   double* p) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * L) return;
  p[e] = fma(beta[e % L], p[e], z[e]);
}
// X[i][j] = v[i] (put) or v[i] = X[i][j] (get)
__global__ void mr_column_kernel(int64_t n, int L, int j, double* X, double* v, int get) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (get) v[i] = X[(size_t)i * L + j];
  else X[(size_t)i * L + j] = v[i];
}

// CTAs per SM of a block solve: its tasks are many and short, so more resident warps keep more
// loads in flight (all resident at once: the launch is cooperative)
constexpr int MR_TRSV_CTAS_PER_SM = 6;

static cudaError_t launch_mr_trsv(const int4* ord, int64_t nrows, const int32_t* idx, const double* coef,
                                  const double* rhs, double* out, int L, int* abort_flag, int* status,
                                  cudaStream_t s) {
  static int grid_of_dev[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int& grid = grid_of_dev[dev & 63];
  if (grid == 0) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mr_sptrsv_kernel, 128, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    grid = sms * (per_sm < MR_TRSV_CTAS_PER_SM ? per_sm : MR_TRSV_CTAS_PER_SM);
  }
  int nch = (L + MR_CW - 1) / MR_CW;
  void* args[] = {(void*)&ord, (void*)&nrows, (void*)&idx, (void*)&coef, (void*)&rhs, (void*)&out, (void*)&L,
                  (void*)&nch, (void*)&abort_flag, (void*)&status};
  return cudaLaunchCooperativeKernel((const void*)mr_sptrsv_kernel, dim3(grid), dim3(128), args, 0, s);
}

static unsigned mr_blocks(int64_t n, int L) { return blocks(n * L, 256); }

// out (m x L) = F^T T for the n x m rows F (leading dimension o.fpad: F itself or A zero-padded)
static void mr_ftv(const LapOps& o, const LapMulti& w, const double* F, const double* T, double* out,
                   cudaStream_t s) {
  const int64_t rpb = (o.n + LAP_MR_FT_BLOCKS - 1) / LAP_MR_FT_BLOCKS;
  const int nb = (int)((o.n + rpb - 1) / rpb);
  mr_ftv_kernel<<<nb, 256, 0, s>>>(F, o.fpad, o.m, o.n, rpb, T, w.L, w.partial);
  mr_col_reduce_kernel<<<blocks((int64_t)o.m * w.L, 256), 256, 0, s>>>(w.partial, nb, o.fpad, o.m, w.L, out);
}

static void mr_spd_apply(const LapMulti& w, const double* Linv, int ld, int m, const double* X, double* Y,
                         cudaStream_t s) {
  mr_lower_gemm_kernel<<<blocks((int64_t)m * w.L, 256), 256, 0, s>>>(Linv, ld, m, w.L, X, w.tmpm, 0);
  mr_lower_gemm_kernel<<<blocks((int64_t)m * w.L, 256), 256, 0, s>>>(Linv, ld, m, w.L, w.tmpm, Y, 1);
}

static void mr_f_dot(const LapOps& o, const LapMulti& w, const double* F, const double* Y, const double* base,
                     double sgn, const double* rsD, const double* scale, double* out, cudaStream_t s) {
  mr_f_dot_kernel<<<blocks(o.n, 64), 256, 0, s>>>(F, o.fpad, o.m, o.n, w.L, Y, base, sgn, rsD, scale, out);
}

cudaError_t lap_mr_matvec(const LapOps& o, const LapMulti& w, const double* X, double* out, cudaStream_t s) {
  // t = D^{-1/2} B X ; t2 = D^{-1/2} (t - F C^{-1} F^T t) ; out = W X + B^T t2
  mr_bx_scaled_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.N, o.Acoef, o.rsD, o.n, o.mv, w.L, X, w.t);
  if (o.m > 0) {
    mr_ftv(o, w, o.F, w.t, w.sm, s);
    mr_spd_apply(w, o.LinvC, o.ldl, o.m, w.sm, w.cm, s);
    mr_f_dot(o, w, o.F, w.cm, w.t, -1.0, nullptr, o.rsD, w.t2, s);
  } else {
    mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.rsD, nullptr, w.t, w.t2);
  }
  mr_btx_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.ch_ptr, o.ch_row, o.ch_coef, o.n, w.L, w.t2, o.W, X, out);
  return cudaGetLastError();
}

cudaError_t lap_mr_precond(const LapOps& o, const LapMulti& w, const double* R, double* out, cudaStream_t s) {
  const size_t bytes = (size_t)o.n * w.L * sizeof(double);
  cudaError_t e = cudaSuccess;
  // x1 = B^{-T} R
  if (o.mv > 0) {
    if ((e = cudaMemsetAsync(w.x1, 0xFF, bytes, s)) != cudaSuccess) return e;
    if ((e = launch_mr_trsv(o.ord_rev, o.n, o.ch_row, o.ch_coef, R, w.x1, w.L, o.abort_flag, o.status, s)) !=
        cudaSuccess)
      return e;
  } else if ((e = cudaMemcpyAsync(w.x1, R, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
    return e;
  }
  // t = G^{-1} (x1 + D^{-1/2} F C3^{-1} F^T D^{-1/2} G^{-1} x1)
  if (o.m > 0) {
    mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.rsD, o.Ginv, w.x1, w.t2);
    mr_ftv(o, w, o.F, w.t2, w.sm, s);
    mr_spd_apply(w, o.LinvC3, o.ldl, o.m, w.sm, w.cm, s);
    mr_f_dot(o, w, o.F, w.cm, w.x1, 1.0, o.rsD, o.Ginv, w.t, s);
  } else {
    mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.Ginv, nullptr, w.x1, w.t);
  }
  // out = B^{-1} t
  if (o.mv > 0) {
    if ((e = cudaMemsetAsync(out, 0xFF, bytes, s)) != cudaSuccess) return e;
    if ((e = launch_mr_trsv(o.ord_fwd, o.n, o.N, o.Acoef, w.t, out, w.L, o.abort_flag, o.status, s)) !=
        cudaSuccess)
      return e;
  } else if ((e = cudaMemcpyAsync(out, w.t, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
    return e;
  }
  return cudaGetLastError();
}

// out[i][j] = t[i][j] + x[i][j] / d_i
__global__ void mr_add_div_kernel(int64_t n, int L, const double* __restrict__ t, const double* __restrict__ x,
                                  const double* __restrict__ d, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * L) return;
  out[e] = t[e] + x[e] / d[e / L];
}

// FITC form (Eq. pcls2): out = (W^{-1} + Sigma_dagger) X = B^{-1} (D o B^{-T} X) + A^T (A X) + X / W, or
// Sigma_dagger X alone (add_winv = false)
cudaError_t lap_mr_sigma_matvec(const LapOps& o, const LapMulti& w, const double* X, double* out, cudaStream_t s,
                                bool add_winv) {
  const size_t bytes = (size_t)o.n * w.L * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (o.mv > 0) {
    if ((e = cudaMemsetAsync(w.x1, 0xFF, bytes, s)) != cudaSuccess) return e;
    if ((e = launch_mr_trsv(o.ord_rev, o.n, o.ch_row, o.ch_coef, X, w.x1, w.L, o.abort_flag, o.status, s)) !=
        cudaSuccess)
      return e;
    mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.D, nullptr, w.x1, w.t2);
    if ((e = cudaMemsetAsync(w.t, 0xFF, bytes, s)) != cudaSuccess) return e;
    if ((e = launch_mr_trsv(o.ord_fwd, o.n, o.N, o.Acoef, w.t2, w.t, w.L, o.abort_flag, o.status, s)) !=
        cudaSuccess)
      return e;
  } else {
    mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.D, nullptr, X, w.t);
  }
  if (add_winv) {
    mr_add_div_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, w.t, X, o.W, w.t2);
  } else if ((e = cudaMemcpyAsync(w.t2, w.t, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
    return e;
  }
  if (o.m > 0) {
    mr_ftv(o, w, o.Apad, X, w.sm, s);
    mr_f_dot(o, w, o.Apad, w.sm, w.t2, 1.0, nullptr, nullptr, out, s);
  } else if ((e = cudaMemcpyAsync(out, w.t2, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
    return e;
  }
  return cudaGetLastError();
}

// FITC preconditioner (App. E.2): out = D_V^{-1} (R - A^T M_V^{-1} A D_V^{-1} R)
cudaError_t lap_mr_precond_fitc(const LapOps& o, const LapMulti& w, const double* R, double* out, cudaStream_t s) {
  if (o.m == 0) {
    mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.dvinv, nullptr, R, out);
    return cudaGetLastError();
  }
  mr_scale2_kernel<<<mr_blocks(o.n, w.L), 256, 0, s>>>(o.n, w.L, o.dvinv, nullptr, R, w.t2);
  mr_ftv(o, w, o.Apad, w.t2, w.sm, s);
  mr_spd_apply(w, o.LinvMV, o.ldl, o.m, w.sm, w.cm, s);
  mr_f_dot(o, w, o.Apad, w.cm, R, -1.0, nullptr, o.dvinv, out, s);
  return cudaGetLastError();
}

cudaError_t lap_mr_system_matvec(const LapOps& o, const LapMulti& w, const double* X, double* out, cudaStream_t s) {
  return o.kind == LAP_FITC ? lap_mr_sigma_matvec(o, w, X, out, s, true) : lap_mr_matvec(o, w, X, out, s);
}

cudaError_t lap_mr_system_precond(const LapOps& o, const LapMulti& w, const double* R, double* out, cudaStream_t s) {
  return o.kind == LAP_FITC ? lap_mr_precond_fitc(o, w, R, out, s) : lap_mr_precond(o, w, R, out, s);
}

cudaError_t lap_mr_scale2(const LapMulti& w, int64_t n, const double* a, const double* b, const double* x,
                          double* out, cudaStream_t s) {
  mr_scale2_kernel<<<mr_blocks(n, w.L), 256, 0, s>>>(n, w.L, a, b, x, out);
  return cudaGetLastError();
}

cudaError_t lap_mr_ftv(const LapOps& o, const LapMulti& w, const double* F, const double* T, double* out,
                       cudaStream_t s) {
  mr_ftv(o, w, F, T, out, s);
  return cudaGetLastError();
}

cudaError_t lap_mr_dot(const LapMulti& w, int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  mr_dot_stage1<<<LAP_MR_DOT_BLOCKS, 256, 0, s>>>(a, b, n, w.L, w.dpart);
  mr_dot_stage2<<<1, LAP_MR_MAXL, 0, s>>>(w.dpart, LAP_MR_DOT_BLOCKS, w.L, out);
  return cudaGetLastError();
}

cudaError_t lap_mr_alpha(const LapMulti& w, const int* active, const double* rz, const double* pAp, double* alpha,
                         cudaStream_t s) {
  mr_alpha_kernel<<<1, LAP_MR_MAXL, 0, s>>>(w.L, active, rz, pAp, alpha);
  return cudaGetLastError();
}

cudaError_t lap_mr_beta(const LapMulti& w, const int* active, double* rz, const double* rznew, double* beta,
                        cudaStream_t s) {
  mr_beta_kernel<<<1, LAP_MR_MAXL, 0, s>>>(w.L, active, rz, rznew, beta);
  return cudaGetLastError();
}

cudaError_t lap_mr_update_xr(const LapMulti& w, int64_t n, const double* alpha, const double* p, const double* Ap,
                             double* x, double* r, cudaStream_t s) {
  mr_update_xr_kernel<<<mr_blocks(n, w.L), 256, 0, s>>>(n, w.L, alpha, p, Ap, x, r);
  return cudaGetLastError();
}

cudaError_t lap_mr_update_p(const LapMulti& w, int64_t n, const double* beta, const double* z, double* p,
                            cudaStream_t s) {
  mr_update_p_kernel<<<mr_blocks(n, w.L), 256, 0, s>>>(n, w.L, beta, z, p);
  return cudaGetLastError();
}

// dst[i][j] = src[i][map[j]]  (src n x Ls, dst n x Ld)
__global__ void mr_gather_kernel(int64_t n, int Ls, int Ld, const int* __restrict__ map,
                                 const double* __restrict__ src, double* dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * Ld) return;
  const int64_t i = e / Ld;
  const int j = (int)(e - i * Ld);
  dst[e] = src[(size_t)i * Ls + map[j]];
}
// dst[i][jd] = src[i][js]
__global__ void mr_copy_col_kernel(int64_t n, const double* __restrict__ src, int Ls, int js, double* dst, int Ld,
                                   int jd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[(size_t)i * Ld + jd] = src[(size_t)i * Ls + js];
}

cudaError_t lap_mr_gather(int64_t n, int Ls, int Ld, const int* map, const double* src, double* dst,
                          cudaStream_t s) {
  mr_gather_kernel<<<mr_blocks(n, Ld), 256, 0, s>>>(n, Ls, Ld, map, src, dst);
  return cudaGetLastError();
}

cudaError_t lap_mr_copy_col(int64_t n, const double* src, int Ls, int js, double* dst, int Ld, int jd,
                            cudaStream_t s) {
  mr_copy_col_kernel<<<blocks(n, 256), 256, 0, s>>>(n, src, Ls, js, dst, Ld, jd);
  return cudaGetLastError();
}

cudaError_t lap_mr_column(int64_t n, int L, int j, double* X, double* v, bool get, cudaStream_t s) {
  mr_column_kernel<<<blocks(n, 256), 256, 0, s>>>(n, L, j, X, v, get ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace vif
