// Internal declarations of libvif (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/vif.h"

namespace vif {

// ---------------------------------------------------------------------------
// Covariance functions (Sec. 2; Eq. cov_trans_iso of Sec. 6), written on the
// squared scaled distance r2 = ||(s-s')/lambda||^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }

template <typename T>
__device__ __forceinline__ T cov_r2(T r2, int kind, T var) {
  if (kind == VIF_SE) return var * dexp(T(-0.5) * r2);
  if (kind == VIF_MATERN12) return var * dexp(-dsqrt(r2));
  if (kind == VIF_MATERN32) {
    T t = dsqrt(T(3) * r2);
    return var * (T(1) + t) * dexp(-t);
  }
  T t = dsqrt(T(5) * r2);  // Matern-5/2
  return var * (T(1) + t + t * t * T(1.0 / 3.0)) * dexp(-t);
}

template <typename T>
__device__ __forceinline__ T sqdist(const T* __restrict__ a, const T* __restrict__ b, int d) {
  T s = 0;
  for (int t = 0; t < d; ++t) {
    T u = a[t] - b[t];
    s += u * u;
  }
  return s;
}

// Packed float32 pairs for the f32x2 instructions of the sm_100 family (two IEEE
// operations per instruction, same rounding as the scalar ones).
__device__ __forceinline__ unsigned long long pack_f2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack_f2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// float32 covariance for the tensor-core A kernel: the exponential through exp2 of a
// rescaled argument (2-ulp exp2 plus the rounding of the product; the absolute error
// stays far below the tf32 split error of the operand)
__device__ __forceinline__ float cov_r2_fast(float r2, int kind, float var) {
  constexpr float L2E = 1.4426950408889634f;
  if (kind == VIF_SE) return var * exp2f(-0.5f * L2E * r2);
  if (kind == VIF_MATERN12) return var * exp2f(-L2E * sqrtf(r2));
  if (kind == VIF_MATERN32) {
    const float t = sqrtf(3.f * r2);
    return var * (1.f + t) * exp2f(-L2E * t);
  }
  const float t = sqrtf(5.f * r2);
  return var * (1.f + t + t * t * (1.f / 3.f)) * exp2f(-L2E * t);
}

// Device status words (int32): [0] error code, [1] failing index, [2..] counters.
enum StatusCode { ST_OK = 0, ST_NOTPD_SIGMAM = 1, ST_NOTPD_FACTOR = 2, ST_NOTPD_CAP = 3,
                  ST_NOTPD_PRECOND = 4, ST_TIMEOUT = 5, ST_BAD_NEIGHBOR = 6 };

__device__ __forceinline__ void flag_status(int* status, int code, long long idx) {
  if (atomicCAS(status, 0, code) == 0) status[1] = (int)idx;
}

// Per-call hyperparameters, in the form the kernels use.
struct CovParams {
  int kind;
  double var;
  double tdiag;   // diagonal added to residual Vecchia blocks (nugget, or latent jitter)
  double jitter;  // diagonal added to Sigma_m
};

// Host-side checks and conversions shared by the context API (vif_api.cu) and the
// allocation-free entry point (vif_noalloc.cu), so that both accept, reject and
// report alike.
bool is_device_ptr(const void* p);                              // device or managed memory
bool cov_valid(const vif_cov* cv, int d, char* why, size_t cap);  // false: reason in why
CovParams cov_params(const vif_cov* cv);                        // kernel form, with the R6 jitters
vif_status status_error(const int* st, char* why, size_t cap);  // device status words -> vif_status

// ---------------------------------------------------------------------------
// Launchers (host side), grouped by translation unit.
// ---------------------------------------------------------------------------
// vif_dense.cu: float64 dense m x m linear algebra for Sigma_m and capacitance matrices.
cudaError_t dense_cholesky(double* A, int m, int lda, int* status, int code, cudaStream_t s);
// work: trtri_work_doubles(m) float64 scratch
size_t trtri_work_doubles(int m);
cudaError_t dense_trtri_lower(const double* L, double* Linv, int m, int lda, double* work, cudaStream_t s);
cudaError_t reduce_sum(const double* x, int64_t n, double* partial, double* out, cudaStream_t s);

// Batched form for many independent problems: one launch per step for all jobs.  A job
// is a Cholesky of A (m x m, leading dimension lda, non-PD pivots flagged with `code` in
// status) or, with trtri, the inverse of the lower factor A into Li (zeroed beforehand,
// work: trtri_work_doubles(m) zeroed doubles).
struct DenseJob {
  double* A;
  double* Li;
  double* work;
  int* status;
  int m, lda, code;
};
struct DenseLaunch {
  int op, step, blocks, off;
};
struct DenseBatch {
  DenseJob* djobs = nullptr;   // device copy of the jobs
  int* doff = nullptr;         // device block offsets, njobs + 1 per launch
  int njobs = 0;
  bool trtri = false;
  std::vector<DenseLaunch> launches;
};
cudaError_t dense_batch_init(const std::vector<DenseJob>& jobs, bool trtri, DenseBatch* b);   // allocates
cudaError_t dense_batch_run(const DenseBatch& b, cudaStream_t s);
void dense_batch_free(DenseBatch* b);

// vif_grad.cu: analytic gradient of the Gaussian likelihood (float64) from the buffers a
// float64 evaluation leaves: A (whitened rows, n x mpad), [F z] (n x fpad), A_i (n x mv),
// D_i, the augmented capacitance factor G (lda fpad), L_m^{-1} (ldl), scaled coordinates.
struct GradInputs {
  const double *A, *F, *Xs, *Zs, *Acoef, *Dv, *y, *G, *Linv, *ls;
  const int32_t* N;
  int64_t n;
  int d, m, mpad, fpad, mv, ldl, nls;
  CovParams cp;
};
size_t grad_scratch_doubles(int64_t n, int m, int mv, int q);
// grad_dev receives 3 q doubles (direct, cross and inducing-point sums; the gradient is their
// sum); LinvC: fpad x fpad doubles; trw: trtri_work_doubles(m) doubles.
cudaError_t vif_grad_fp64(const GradInputs& in, double* scratch, double* LinvC, double* trw, double* grad_dev,
                          cudaStream_t s);

// vif_lowrank_tc.cu: A = K_nm L_m^{-T} on the tensor cores for the float32 path.  init
// (once per device, outside stream capture) raises the kernel's shared-memory limit;
// pack holds lowrank_A_tc_pack_floats(mpad) floats; mpad = 32 ceil(m / 32).
cudaError_t lowrank_A_tc_init();
size_t lowrank_A_tc_pack_floats(int mpad);
cudaError_t lowrank_A_tc(const float* Xs, const float* Zs, const double* Linv, int ldl, float* pack, float* A,
                         int64_t n, int d, int m, int mpad, int kind, double var, int* status, cudaStream_t s);

// vif_lowrank.cu
cudaError_t scale_coords(const double* X, int64_t n, int d, const double* inv_ls, const double* center,
                         double* Xs, float* Xs32, cudaStream_t s);
cudaError_t build_sigma_m(const double* Zs, int m, int d, CovParams cp, double* Sm, int lda,
                          cudaStream_t s);
template <typename T>
cudaError_t linv_transpose(const double* Linv, int m, int lda, T* LinvT, int ldt, cudaStream_t s);
template <typename T>
cudaError_t lowrank_A(const T* Xs, const T* Zs, const T* LinvT, int ldt, T* A, int64_t n, int d,
                      int m, int mpad, int kind, double var, cudaStream_t s);
cudaError_t residual_diag_stats(const double* A, int64_t n, int m, int mpad, double var, double tau,
                                float* A32, double* cii, float* rs32, float* nrm32, cudaStream_t s);

// vif_factor.cu
// order: processing order of the points (a permutation of 0..n-1), or NULL for 0..n-1.
template <typename T>
cudaError_t vecchia_factor(const T* A, const T* Xs, const int32_t* N, const int32_t* order, const double* y,
                           int64_t n, int d, int m, int mpad, int mv, int fpad, CovParams cp, T* F,
                           double* Acoef, double* Dv, double* logD, int* status, cudaStream_t s);
// gsub (float32 path only): the Gram of each point's rows [A_N(i); a_i] from
// union_gram_tc, slot-major in the processing order with stride (m_v + 1)(m_v + 2) / 2
// (packed lower triangle); NULL: the kernel forms it itself.  rho (optional, n x 2
// floats): per point the largest and the mean |residual correlation| with its neighbours.
template <typename T>
cudaError_t vecchia_factor_gs(const T* A, const T* Xs, const int32_t* N, const int32_t* order, const double* y,
                              int64_t n, int d, int m, int mpad, int mv, int fpad, CovParams cp, T* F,
                              double* Acoef, double* Dv, double* logD, int* status, cudaStream_t s,
                              const float* gsub, float* rho = nullptr);
// The factor stage of many problems in one persistent launch per neighbour-block size: jobs
// (device array) whose points are listed back to back (job p owns positions off[p] ..
// off[p+1], off has njobs + 1 entries, off[0] = 0), all with m_v + 1 in the same block-size
// class as mv_max; warps take the next positions from the device counter `queue` (zeroed by
// the call).
template <typename T>
struct FactorJob {
  const T* A;
  const T* Xs;
  const int32_t* N;
  const int32_t* order;
  const double* y;
  int64_t n;
  int d, m, mpad, mv, fpad;
  CovParams cp;
  T* F;
  double *Acoef, *Dv, *logD;
  int* status;
};
// the block size class of m_v (jobs of one launch share it)
inline int factor_block_class(int mv) {
  const int Q = mv + 1;
  return Q <= 14 ? 2 : Q <= 21 ? 3 : Q <= 28 ? 4 : Q <= 35 ? 5 : Q <= 42 ? 6 : Q <= 49 ? 7 : 0;
}
template <typename T>
cudaError_t vecchia_factor_batched(const FactorJob<T>* jobs, const int64_t* off, int njobs, int mv_max,
                                   unsigned long long* queue, int nsm, cudaStream_t s);
// The same work as one launch whose job records travel in the kernel's parameter bank (up to
// FT_MAXJ jobs per table, 30 KB): block b serves job p with boff[p] <= b < boff[p+1], boff
// counting blocks of 4 points (job p has ceil(n_p / 4) of them), so the job's fields are
// block-uniform operands as in the single-problem kernel instead of per-thread registers.
constexpr int FT_MAXJ = 200;
constexpr int FT_BLOCK_POINTS = 4;   // points (one per warp) of a block of the table kernel
template <typename T>
struct FactorTable {
  FactorJob<T> job[FT_MAXJ];
  int boff[FT_MAXJ + 1];
  int njobs;
};
template <typename T>
cudaError_t vecchia_factor_table(const FactorTable<T>& tab, int mv_max, cudaStream_t s);
// vif_factor_tc.cu: the residual products A_N^T A_N on the tensor cores (float32 path).
// Groups of consecutive points of the processing order share one 128-row Gram.
struct UnionGroups {
  const int32_t* rows;        // ngroups x 128 rows of A (-1 padded)
  const int32_t* ptr;         // ngroups + 1 offsets into the processing order
  const unsigned char* loc;   // n x 32: group-local row of each of a slot's rows (0xFF beyond)
  int64_t ngroups;
};
constexpr int UG_MAX_POINTS = 128;   // points per group (the kernel's table of local rows)
cudaError_t union_gram_tc_init();
// var: sigma_1^2 (bounds |A_ij| and so the float16 scaling); nsm: SM count of the device
// (one persistent CTA per SM)
cudaError_t union_gram_tc(const float* A, int mpad, const UnionGroups& ug, int Q, double var, float* gsub,
                          int* status, cudaStream_t s, int nsm);
bool build_union_groups(const int32_t* N, const int32_t* order, int64_t n, int mv, int max_pts,
                        std::vector<int32_t>& rows, std::vector<int32_t>& ptr, std::vector<unsigned char>& loc);
// wrow: optional row weights (NULL = 1): G = F^T diag(wrow) F (+ identity on the first m).
// The float32 Gram runs on the tensor cores (vif_gram_tc.cu) and may use fewer slices
// than nsplit; status receives ST_TIMEOUT if one of its waits gives up.
template <typename T>
cudaError_t gram_FtF(const T* F, int64_t n, int fpad, int m, double* part, int nsplit, double* G,
                     int ldg, cudaStream_t s, const double* wrow = nullptr, int* status = nullptr);
// vif_gram_tc.cu: split-K float32 Gram partials on the tensor cores (64 x 64 pair layout)
cudaError_t gram_tc_init();
int gram_tc_nsplit(int64_t n, int fpad);
cudaError_t gram_tc(const float* F, int64_t n, int fpad, double* part, int nsplit, int* status, cudaStream_t s);
int gram_nsplit(int64_t n, int fpad);
cudaError_t nll_finish(const double* Lg, int ldg, int m, const double* logD_sum, int64_t n,
                       double* out, cudaStream_t s);

// vif_predict.cu
cudaError_t predict_setup(const double* A, const double* Xs, int64_t n, const double* Ap, const double* Xps,
                          int64_t np, int d, int m, int mpad, int mv, CovParams cp, double* cjj, double* cpp,
                          int32_t* Np, cudaStream_t s);
cudaError_t predict_resid(const double* A, const double* w, const double* y, int64_t n, int m, int mpad, double* r,
                          cudaStream_t s);
cudaError_t predict_eval(const double* A, const double* Xs, const double* Ap, const double* Xps, const int32_t* Np,
                         const double* r, const double* w, const double* LinvC, int ldg, int64_t np, int d, int m,
                         int mpad, int mv, CovParams cp, int latent, double nugget, double* mean, double* var,
                         int* status, cudaStream_t s);
cudaError_t predict_all(const double* A, const double* Xs, int64_t n, const double* Ap, const double* Xps,
                        int64_t np, int d, int m, int mpad, int mv, CovParams cp, const double* y, const double* Lg,
                        int ldg, double* LinvC, double* w, double* r, double* cjj, double* cpp, int32_t* Np,
                        int latent, double nugget, double* mean, double* var, int* status, double* trwork,
                        cudaStream_t s);

// vif_laplace.cu
// abort_flag[1] = polls: the bound on each wait of the level-scheduled solves (0: default)
cudaError_t lap_set_wait_polls(int* abort_flag, int polls, cudaStream_t s);
// rows of the level schedules of the two triangular solves are taken four at a time
// (slots {row, first term, end of terms, solo}); each level is padded with
// {-1, 0, 0, 0} to a multiple of this
constexpr int LAP_TRSV_RPS = 4;
// preconditioner / system form of the Laplace CG
constexpr int LAP_VIFDU = 0;   // VIFDU, Eq. pcls1: (W + Sigma_dagger^{-1}) x = v
constexpr int LAP_FITC = 2;    // FITC, Eq. pcls2: (W^{-1} + Sigma_dagger) x = v
// row slices of the F^T v product (partial buffer: LAP_FT_BLOCKS x fpad)
constexpr int LAP_FT_BLOCKS = 608;
struct LapOps {
  int64_t n;
  int m, mv, fpad, ldl;
  const int32_t *N, *ch_ptr, *ch_row, *ch_slot;
  const int4 *sched_fwd, *sched_rev;      // level-ordered slots of B^{-1} / B^{-T}
  const int4 *ord_fwd, *ord_rev;          // every row once in level order: {row, first term, end, 0}
  int64_t nsteps_fwd, nsteps_rev;         // schedule lengths / LAP_TRSV_RPS
  const double* ch_coef;                  // A_i[k] of each child term, CSR order (lap_child_coef)
  int64_t nnz;                            // child terms
  // FITC preconditioner with the system form of Eq. pcls2 (kind = LAP_FITC)
  int kind;                               // LAP_VIFDU or LAP_FITC
  const double *A, *Apad, *D, *W;         // rows of A (ld mpad), A zero-padded to ld fpad, D_i, W_i
  int mpad;
  double *dvinv, *anorm2;                 // 1/D_V; |a_i|^2
  const double* LinvMV;                   // inverse Cholesky factor of I + A D_V^{-1} A^T (ld fpad)
  const double *Acoef, *F, *LinvC, *LinvC3;
  double *rsD, *Ginv;          // 1/sqrt(D_i), 1/(W'_i + 1/D_i)
  double *t, *t2, *x1;         // n-vector scratch
  double *sm, *cm, *tmpm;      // m-vector scratch
  double* partial;             // LAP_FT_BLOCKS x fpad
  int *counter, *abort_flag, *status;   // counter: two 64-bit work-queue counters
};
cudaError_t lap_matvec(const LapOps& o, const double* x, const double* diagW, double* out, cudaStream_t s);
cudaError_t lap_precond(const LapOps& o, const double* w, double* out, cudaStream_t s);
cudaError_t lap_child_coef(const LapOps& o, double* ch_coef, cudaStream_t s);
// VIF-Laplace likelihood with SLQ (Eq. log_det_VIFLA, Eq. slq_v1): probe pieces and log-sums
cudaError_t lap_log_sum(const double* x, int64_t n, int64_t stride, double sgn, double* partial, double* out,
                        cudaStream_t s);
cudaError_t lap_probe_prep(int64_t n, const double* D, const double* W, const double* corr, const double* eps2,
                           const double* eps3, double* u, double* v, cudaStream_t s);
cudaError_t lap_vec_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
cudaError_t lap_solve_B(const LapOps& o, const double* rhs, double* out, cudaStream_t s);
cudaError_t lap_apply_Bt(const LapOps& o, const double* u, double* out, cudaStream_t s);
cudaError_t lap_rows_dot_add(const double* rows, int ld, int m, int64_t n, const double* c, const double* base,
                             double* out, cudaStream_t s);
// FITC / Eq. pcls2 pieces
cudaError_t lap_fitc_prepare_A(const double* A, int mpad, int m, int64_t n, int fpad, double* Apad, double* anorm2,
                               cudaStream_t s);
cudaError_t lap_fitc_dv(int64_t n, double var, const double* anorm2, const double* W, double* dvinv, cudaStream_t s);
cudaError_t lap_sigma_matvec(const LapOps& o, const double* x, const double* Winv_of, double* out, cudaStream_t s);
cudaError_t lap_precond_fitc(const LapOps& o, const double* w, double* out, cudaStream_t s);
cudaError_t lap_system_matvec(const LapOps& o, const double* x, double* out, cudaStream_t s);
cudaError_t lap_system_precond(const LapOps& o, const double* w, double* out, cudaStream_t s);
cudaError_t lap_fitc_probe(const LapOps& o, const double* eps1, const double* eps2, double* z, cudaStream_t s);
cudaError_t lap_div(int64_t n, const double* x, const double* d, double* out, cudaStream_t s);
cudaError_t lap_recip(const double* a, int64_t n, double* out, cudaStream_t s);
cudaError_t lap_bx_scaled(const LapOps& o, const double* x, double* t, cudaStream_t s);
cudaError_t lap_ftv(const double* F, int fpad, int m, int64_t n, const double* v, double* partial, double* out,
                    cudaStream_t s);
cudaError_t lap_spd_apply(const double* Linv, int ld, int m, const double* x, double* tmp, double* y, cudaStream_t s);
cudaError_t lap_sq_accumulate(int64_t n, const double* x, double* acc, cudaStream_t s);
cudaError_t lap_axpy_host(int64_t n, double a, const double* x, const double* y, double* out, cudaStream_t s);
cudaError_t lap_pointwise(const double* y, const double* b, const double* D, const double* corr, int64_t n, double* W,
                          double* v, double* Ginv, double* omega, double* rsD, double* ll, cudaStream_t s);
cudaError_t lap_dot(const double* a, const double* b, int64_t n, double* partial, double* out, cudaStream_t s);
cudaError_t lap_axpy(int64_t n, const double* scal, const double* x, const double* y, double* out, int mode,
                     cudaStream_t s);
cudaError_t lap_alpha(double* sc, cudaStream_t s);
cudaError_t lap_beta(double* sc, cudaStream_t s);
// many right-hand sides (the SLQ probes, Sec. 4.1): n x L row-major block vectors, L <= LAP_MR_MAXL
constexpr int LAP_MR_MAXL = 64;
constexpr int LAP_MR_FT_BLOCKS = 304;   // row slices of the block F^T T product
constexpr int LAP_MR_DOT_BLOCKS = 256;
struct LapMulti {
  int L;
  double *t, *t2, *x1;        // n x L scratch
  double *sm, *cm, *tmpm;     // m x L scratch
  double* partial;            // LAP_MR_FT_BLOCKS x fpad x L
  double* dpart;              // LAP_MR_DOT_BLOCKS x L
};
cudaError_t lap_mr_matvec(const LapOps& o, const LapMulti& w, const double* X, double* out, cudaStream_t s);
cudaError_t lap_mr_precond(const LapOps& o, const LapMulti& w, const double* R, double* out, cudaStream_t s);
cudaError_t lap_mr_sigma_matvec(const LapOps& o, const LapMulti& w, const double* X, double* out, cudaStream_t s,
                                bool add_winv);
cudaError_t lap_mr_scale2(const LapMulti& w, int64_t n, const double* a, const double* b, const double* x,
                          double* out, cudaStream_t s);
cudaError_t lap_mr_ftv(const LapOps& o, const LapMulti& w, const double* F, const double* T, double* out,
                       cudaStream_t s);
cudaError_t lap_mr_precond_fitc(const LapOps& o, const LapMulti& w, const double* R, double* out, cudaStream_t s);
cudaError_t lap_mr_system_matvec(const LapOps& o, const LapMulti& w, const double* X, double* out, cudaStream_t s);
cudaError_t lap_mr_system_precond(const LapOps& o, const LapMulti& w, const double* R, double* out, cudaStream_t s);
cudaError_t lap_mr_dot(const LapMulti& w, int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
cudaError_t lap_mr_alpha(const LapMulti& w, const int* active, const double* rz, const double* pAp, double* alpha,
                         cudaStream_t s);
cudaError_t lap_mr_beta(const LapMulti& w, const int* active, double* rz, const double* rznew, double* beta,
                        cudaStream_t s);
cudaError_t lap_mr_update_xr(const LapMulti& w, int64_t n, const double* alpha, const double* p, const double* Ap,
                             double* x, double* r, cudaStream_t s);
cudaError_t lap_mr_update_p(const LapMulti& w, int64_t n, const double* beta, const double* z, double* p,
                            cudaStream_t s);
cudaError_t lap_mr_column(int64_t n, int L, int j, double* X, double* v, bool get, cudaStream_t s);
cudaError_t lap_mr_gather(int64_t n, int Ls, int Ld, const int* map, const double* src, double* dst,
                          cudaStream_t s);
cudaError_t lap_mr_copy_col(int64_t n, const double* src, int Ls, int js, double* dst, int Ld, int jd,
                            cudaStream_t s);
// gradient of the VIF-Laplace likelihood (Sec. 4.1, App. B, App. D)
cudaError_t lap_ste_diag(int64_t n, int l, const double* U, const double* Y, const double* b, int form, double* g,
                         cudaStream_t s);
cudaError_t lap_grad_forms(int64_t n, const double* a, const double* c, const double* x, const double* t,
                           const double* w, const double* d, double* partial, double* out0, double* out1,
                           double* out2, cudaStream_t s);

// vif_mlp.cu
size_t mlp_bytes();
cudaError_t mlp_init(void* net, uint64_t seed, cudaStream_t s);
cudaError_t mlp_set(void* net, const float* p, cudaStream_t s);
// rho: n x 2 floats (largest and mean |residual correlation| with the neighbours) or NULL (zeros)
cudaError_t mlp_features(const double* W, const double* D, const double* Acoef, const float* rho, const int32_t* N,
                         const int32_t* ch_ptr, const int32_t* ch_row, const int32_t* ch_slot, int64_t n, int mv,
                         float* F, cudaStream_t s);
cudaError_t mlp_forward_f32(const void* net, const float* F, int64_t n, float* c, cudaStream_t s);
cudaError_t mlp_forward_f64(const void* net, const float* F, int64_t n, double* c, cudaStream_t s);
int mlp_backward_blocks(int64_t n);
cudaError_t mlp_backward(const void* net, const float* F, const float* gc, int64_t n, float* partial, float* grad,
                         cudaStream_t s);
cudaError_t mlp_adam(void* net, const float* grad, float lr, cudaStream_t s);
cudaError_t mlp_rademacher(uint64_t seed, int64_t n, double* z, cudaStream_t s);
cudaError_t mlp_lp_grad(const int32_t* N, const double* Acoef, int64_t n, int mv, const double* sv, const double* u,
                        const double* W, const double* corr, double coeff, float* gc, cudaStream_t s);
cudaError_t mlp_zero(float* x, int64_t n, cudaStream_t s);
const float* mlp_master(const void* net);

// vif_knn.cu
struct KnnParams {
  int64_t n;
  int d, m, mpad, mv, kprime;
  int kind;
  double var;
  double tau_v;     // residual variances <= tau_v count as zero (correlation set to 0)
  float gamma;      // float32 dot-product error factor
  float epsK;       // bound on the float32 kernel-evaluation error
};
cudaError_t knn_causal(const KnnParams& p, const float* A32, const double* A64, const float* Xs32,
                       const double* Xs64, const double* cii, const float* rs32, const float* nrm32,
                       float* cand_key, int32_t* cand_idx, float* cand_e, float* lowbound,
                       int32_t* N, int* counters, int32_t* fallback_list, cudaStream_t s);

}  // namespace vif

// vif_api.cu: sets the message that vif_last_error(NULL) returns.
void vif_internal_set_global_error(const char* msg);
