// C ABI of libvif: context management and the host orchestration of the
// kernels (see include/vif.h for the contract of each entry point).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "vif_internal.cuh"

using namespace vif;

struct vif_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  int d = 0, m = 0, mv = 0, mpad = 32, fpad = 64, ldm = 32;
  int precision = 0, likelihood = 0;
  double center[16] = {0};
  // device buffers
  double *X = nullptr, *Z = nullptr;          // raw coordinates
  double *Xs = nullptr, *Zs = nullptr;        // scaled coordinates (float64)
  float *Xs32 = nullptr, *Zs32 = nullptr;     // scaled coordinates (float32, mixed path)
  double *hyp = nullptr;                      // [0..15] 1/lambda, [16..31] center
  int32_t* N = nullptr;                       // n x mv
  int32_t* order = nullptr;                   // processing order of the per-point kernels
  std::vector<int32_t> h_order;               // the same order on the host
  // float32 path: groups of points sharing one tensor-core Gram of their rows of A
  int32_t *ug_rows = nullptr, *ug_ptr = nullptr;
  unsigned char* ug_loc = nullptr;
  float* gsub = nullptr;                      // per slot: Gram of the point's rows (packed triangle)
  int64_t ug_ngroups = 0;
  bool ug_ready = false;
  int factor_mode = 0;                        // 0 autotuned, 1 CUDA cores, 2 tensor cores
  int factor_choice = -1;                     // autotuned: -1 undecided, 0 CUDA cores, 1 tensor cores
  float factor_ms[2] = {0.f, 0.f};            // the autotuner's timings (CUDA cores, tensor cores)
  int nsm = 1;
  double *Sm = nullptr, *Linv = nullptr;      // m x ldm
  double* trw = nullptr;                      // triangular-inverse workspace
  void* LinvT = nullptr;                      // mpad x mpad (float or double)
  void* A = nullptr;                          // n x mpad
  void* F = nullptr;                          // n x fpad
  double *Acoef = nullptr, *Dv = nullptr, *logD = nullptr;
  double* part = nullptr;
  int nsplit = 1;
  double* G = nullptr;                        // (m+1) x fpad
  double* y = nullptr;                        // n
  double* red = nullptr;                      // reduction scratch (256)
  double* dscal = nullptr;                    // [0] sum log D, [1..3] nll, logdetC, quad
  int* status = nullptr;                      // [0] code [1] index [2..] counters
  double* h_pin = nullptr;                    // pinned host staging
  // float64 twins of A, F, L^{-T} for prediction from a mixed-precision context
  double *pA = nullptr, *pF = nullptr, *pLinvT = nullptr;
  // prediction buffers, grown on demand
  int64_t p_cap = 0;
  double *pXp = nullptr, *pXps = nullptr, *pAp = nullptr, *pcpp = nullptr, *pmean = nullptr, *pvar = nullptr;
  int32_t* pNp = nullptr;
  double *pcjj = nullptr, *pw = nullptr, *pr = nullptr, *pLinvC = nullptr;
  // Laplace buffers (allocated on the first vif_laplace_mode call)
  bool lap_ready = false;
  int32_t *ch_ptr = nullptr, *ch_row = nullptr, *ch_slot = nullptr;
  int4 *sched_fwd = nullptr, *sched_rev = nullptr;      // level schedules of B^{-1} and B^{-T}
  int4 *ord_fwd = nullptr, *ord_rev = nullptr;          // the rows in level order (block solves)
  int64_t nsteps_fwd = 0, nsteps_rev = 0, ch_nnz = 0;
  double* ch_coef = nullptr;                            // coefficient of each child term
  double* slq_eps = nullptr;                            // normals of one SLQ probe (m + 2n)
  double *l_Apad = nullptr, *l_anorm2 = nullptr, *l_dvinv = nullptr;   // FITC preconditioner
  double* l_pacc = nullptr;                             // SBPV sums of squares (np)
  int64_t l_pacc_cap = 0;
  // gradient by stochastic trace estimation: probe solves U, P^{-1} z_i (g_cap x n each), dL/db~, v,
  // the bilinear forms of one perturbed theta (6 + 3 g_cap) and a three-way reduction scratch
  double *g_U = nullptr, *g_Y = nullptr, *g_g = nullptr, *g_v = nullptr, *g_sc = nullptr, *g_red = nullptr;
  double *g_a = nullptr, *g_av = nullptr, *g_dv = nullptr;   // FITC form: Sigma_dagger^{-1} b~, .. v, D_V
  int64_t g_cap = 0;
  // block CG over up to mr_cap probes: n x L vectors, m x L and reduction scratch, per-column scalars
  double *mr_v = nullptr, *mr_x = nullptr, *mr_r = nullptr, *mr_z = nullptr, *mr_p = nullptr, *mr_Ap = nullptr,
         *mr_t = nullptr, *mr_t2 = nullptr, *mr_x1 = nullptr, *mr_sm = nullptr, *mr_cm = nullptr, *mr_tm = nullptr,
         *mr_part = nullptr, *mr_dpart = nullptr, *mr_sc = nullptr;
  int *mr_active = nullptr, *mr_map = nullptr;
  int mr_cap = 0;
  double *l_b = nullptr, *l_W = nullptr, *l_v = nullptr, *l_Ginv = nullptr, *l_om = nullptr, *l_rsD = nullptr,
         *l_ll = nullptr, *l_x = nullptr, *l_r = nullptr, *l_z = nullptr, *l_p = nullptr, *l_Ap = nullptr,
         *l_t = nullptr, *l_t2 = nullptr, *l_x1 = nullptr, *l_sdi = nullptr, *l_sm = nullptr, *l_cm = nullptr,
         *l_tm = nullptr, *l_part = nullptr, *l_LinvC = nullptr, *l_G3 = nullptr, *l_LinvC3 = nullptr,
         *l_sc = nullptr, *l_red = nullptr, *l_corr = nullptr;
  int *l_counter = nullptr, *l_abort = nullptr;
  float *m_feat = nullptr, *m_gc = nullptr, *m_part = nullptr, *m_grad = nullptr;
  float* m_rho = nullptr;   // latent-GP contexts: max and mean |residual correlation| per point
  double *gr_buf = nullptr, *gr_LinvC = nullptr, *gr_out = nullptr;   // analytic gradient scratch
  int64_t knn_rescored = 0, knn_fallback = 0;
  bool have_factors = false;
  bool timing = false;
  cudaEvent_t ev[VIF_NSTAGES + 1] = {};
  char err[1024] = {0};
};

namespace vif {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool cov_valid(const vif_cov* cv, int d, char* why, size_t cap) {
  const char* msg = nullptr;
  if (!cv) {
    msg = "covariance parameters are NULL";
  } else if (cv->kind < 0 || cv->kind > 3) {
    snprintf(why, cap, "unknown kernel kind %d", cv->kind);
    return false;
  } else if (!(cv->variance > 0.0) || !std::isfinite(cv->variance)) {
    msg = "variance must be positive and finite";
  } else if (!(cv->nugget >= 0.0) || !std::isfinite(cv->nugget)) {
    msg = "nugget must be >= 0 and finite";
  } else if (!cv->lengthscale || (cv->n_ls != 1 && cv->n_ls != d)) {
    snprintf(why, cap, "lengthscale must hold 1 or d=%d values", d);
    return false;
  } else {
    for (int t = 0; t < cv->n_ls; ++t)
      if (!(cv->lengthscale[t] > 0.0) || !std::isfinite(cv->lengthscale[t]))
        msg = "length scales must be positive and finite";
  }
  if (msg) snprintf(why, cap, "%s", msg);
  return msg == nullptr;
}

CovParams cov_params(const vif_cov* cv) {
  CovParams cp;
  cp.kind = cv->kind;
  cp.var = cv->variance;
  // Sigma_m jitter and residual diagonal (nugget, or a jitter for latent processes)
  cp.jitter = (cv->kind == VIF_SE ? 1e-8 : 1e-10) * cv->variance;
  cp.tdiag = cv->nugget > 0.0 ? cv->nugget : 1e-10 * cv->variance;
  return cp;
}

vif_status status_error(const int* st, char* why, size_t cap) {
  if (st[0] == ST_OK) return VIF_OK;
  if (st[0] == ST_TIMEOUT) {
    snprintf(why, cap, "device wait timed out at %d", st[1]);
    return VIF_ERR_TIMEOUT;
  }
  if (st[0] == ST_BAD_NEIGHBOR) {
    snprintf(why, cap, "neighbour table row %d holds an index that is not a predecessor", st[1]);
    return VIF_ERR_STATE;
  }
  const char* what = st[0] == ST_NOTPD_SIGMAM  ? "Sigma_m (inducing points)"
                     : st[0] == ST_NOTPD_FACTOR ? "residual Vecchia block of point"
                     : st[0] == ST_NOTPD_CAP    ? "capacitance matrix"
                                                 : "preconditioner";
  snprintf(why, cap, "Cholesky pivot not positive: %s, index %d", what, st[1]);
  return VIF_ERR_NOT_PD;
}

}  // namespace vif

namespace {

// message of the last failed vif_build (the context is gone by then)
char g_build_err[1024] = {0};

vif_status set_err(vif_ctx* c, vif_status st, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return set_err(ctx, e_ == cudaErrorMemoryAllocation ? VIF_ERR_NOMEM : VIF_ERR_CUDA,       \
                     "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);       \
  } while (0)

template <typename T>
vif_status dalloc(vif_ctx* ctx, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(ctx, VIF_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                   cudaGetErrorString(e));
  }
  return VIF_OK;
}

#define CKS(call)                 \
  do {                            \
    vif_status s_ = (call);       \
    if (s_ != VIF_OK) return s_;  \
  } while (0)

// Copy n elements into a device buffer from a host or device source.
vif_status upload(vif_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return VIF_OK;
  cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(dst, src, bytes, k, ctx->stream));
  return VIF_OK;
}

vif_status download(vif_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return VIF_OK;
  cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(dst, src, bytes, k, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VIF_OK;
}

vif_status check_cov(vif_ctx* ctx, const vif_cov* cv, int d) {
  char why[160];
  if (!cov_valid(cv, d, why, sizeof(why))) return set_err(ctx, VIF_ERR_ARG, "%s", why);
  return VIF_OK;
}

// Scale X and Z by 1/lambda around the data centre (float64 and, if asked, float32).
vif_status apply_scaling(vif_ctx* ctx, const vif_cov* cv, bool want32) {
  double h[32];
  for (int t = 0; t < 16; ++t) {
    h[t] = (t < ctx->d) ? 1.0 / cv->lengthscale[cv->n_ls == 1 ? 0 : t] : 0.0;
    h[16 + t] = ctx->center[t];
  }
  memcpy(ctx->h_pin, h, sizeof(h));
  CK(cudaMemcpyAsync(ctx->hyp, ctx->h_pin, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
  CK(scale_coords(ctx->X, ctx->n, ctx->d, ctx->hyp, ctx->hyp + 16, ctx->Xs, want32 ? ctx->Xs32 : nullptr,
                  ctx->stream));
  if (ctx->m > 0)
    CK(scale_coords(ctx->Z, ctx->m, ctx->d, ctx->hyp, ctx->hyp + 16, ctx->Zs, want32 ? ctx->Zs32 : nullptr,
                    ctx->stream));
  // the pinned staging buffer is reused by later calls: wait for the copy
  CK(cudaStreamSynchronize(ctx->stream));
  return VIF_OK;
}

// A = K_nm L_m^{-T}: float64 on the SIMT kernel from L_m^{-T}; float32 on the tensor
// cores from L_m^{-1} (the float32 LinvT buffer then holds the packed operand).
template <typename T>
cudaError_t lowrank_A_any(vif_ctx* ctx, const CovParams& cp, T* A, T* LinvT, const T* Xs, const T* Zs) {
  if constexpr (sizeof(T) == 4)
    return lowrank_A_tc(Xs, Zs, ctx->Linv, ctx->ldm, LinvT, A, ctx->n, ctx->d, ctx->m, ctx->mpad, cp.kind, cp.var,
                        ctx->status, ctx->stream);
  else
    return lowrank_A<T>(Xs, Zs, LinvT, ctx->mpad, A, ctx->n, ctx->d, ctx->m, ctx->mpad, cp.kind, cp.var,
                        ctx->stream);
}

// Sigma_m, its Cholesky factor and L_m^{-T} in precision T; then A.
template <typename T>
vif_status compute_lowrank(vif_ctx* ctx, const CovParams& cp, T* A, T* LinvT, const T* Xs, const T* Zs) {
  if (ctx->m > 0) {
    CK(build_sigma_m(ctx->Zs, ctx->m, ctx->d, cp, ctx->Sm, ctx->ldm, ctx->stream));
    CK(dense_cholesky(ctx->Sm, ctx->m, ctx->ldm, ctx->status, ST_NOTPD_SIGMAM, ctx->stream));
    CK(dense_trtri_lower(ctx->Sm, ctx->Linv, ctx->m, ctx->ldm, ctx->trw, ctx->stream));
    if constexpr (sizeof(T) == 8) CK(linv_transpose<T>(ctx->Linv, ctx->m, ctx->ldm, LinvT, ctx->mpad, ctx->stream));
  }
  CK(lowrank_A_any<T>(ctx, cp, A, LinvT, Xs, Zs));
  return VIF_OK;
}

// compute_lowrank with stage events: [0,1) Sigma_m and its factors, [1,2) A, then the
// factor stage starts at event 2.
template <typename T>
vif_status compute_lowrank_parts(vif_ctx* ctx, const CovParams& cp, T* A, T* LinvT, const T* Xs, const T* Zs) {
  if (ctx->m > 0) {
    CK(build_sigma_m(ctx->Zs, ctx->m, ctx->d, cp, ctx->Sm, ctx->ldm, ctx->stream));
    CK(dense_cholesky(ctx->Sm, ctx->m, ctx->ldm, ctx->status, ST_NOTPD_SIGMAM, ctx->stream));
    CK(dense_trtri_lower(ctx->Sm, ctx->Linv, ctx->m, ctx->ldm, ctx->trw, ctx->stream));
    if constexpr (sizeof(T) == 8) CK(linv_transpose<T>(ctx->Linv, ctx->m, ctx->ldm, LinvT, ctx->mpad, ctx->stream));
  }
  if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], ctx->stream));
  CK(lowrank_A_any<T>(ctx, cp, A, LinvT, Xs, Zs));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev[2], ctx->stream));
  return VIF_OK;
}

// Whether the float32 path forms the per-point Grams on the tensor cores: when the groups
// exist and the build asked for it, or the autotuner found it faster.
bool factor_on_tc(const vif_ctx* ctx) {
  return ctx->ug_ready && (ctx->factor_mode == 2 || (ctx->factor_mode == 0 && ctx->factor_choice == 1));
}

// The residual Vecchia factors and the rows of [F z] (Sec. 2.1): on the float32 path with
// the per-point Grams of A_N^T A_N from the tensor cores (tc), or all on the CUDA cores.
template <typename T>
vif_status run_factor(vif_ctx* ctx, const CovParams& cp, T* A, const T* Xs, T* F, bool tc) {
  const float* gsub = nullptr;
  if (sizeof(T) == 4 && tc && ctx->ug_ready) {
    const UnionGroups ug{ctx->ug_rows, ctx->ug_ptr, ctx->ug_loc, ctx->ug_ngroups};
    CK(union_gram_tc((const float*)A, ctx->mpad, ug, ctx->mv + 1, cp.var, ctx->gsub, ctx->status, ctx->stream,
                     ctx->nsm));
    gsub = ctx->gsub;
  }
  CK(vecchia_factor_gs<T>(A, Xs, ctx->N, ctx->order, ctx->y, ctx->n, ctx->d, ctx->m, ctx->mpad, ctx->mv,
                          ctx->fpad, cp, F, ctx->Acoef, ctx->Dv, ctx->logD, ctx->status, ctx->stream, gsub,
                          ctx->m_rho));
  return VIF_OK;
}

// The likelihood pipeline of Sec. 2.1-2.2 in precision T on the given buffers:
// A, the residual Vecchia factors and rows of [F z], the Gram, the augmented
// capacitance Cholesky and the scalar (left on the device in dscal[1..3]).
template <typename T>
vif_status run_pipeline(vif_ctx* ctx, const CovParams& cp, T* A, T* LinvT, T* F, const T* Xs, const T* Zs) {
#define MARK(k) \
  if (ctx->timing) CK(cudaEventRecord(ctx->ev[k], ctx->stream))
  MARK(0);
  CKS(compute_lowrank_parts<T>(ctx, cp, A, LinvT, Xs, Zs));
  CKS(run_factor<T>(ctx, cp, A, Xs, F, factor_on_tc(ctx)));
  MARK(3);
  CK(gram_FtF<T>(F, ctx->n, ctx->fpad, ctx->m, ctx->part, ctx->nsplit, ctx->G, ctx->fpad, ctx->stream, nullptr,
                 ctx->status));
  MARK(4);
  CK(reduce_sum(ctx->logD, ctx->n, ctx->red, ctx->dscal, ctx->stream));
  CK(dense_cholesky(ctx->G, ctx->m + 1, ctx->fpad, ctx->status, ST_NOTPD_CAP, ctx->stream));
  CK(nll_finish(ctx->G, ctx->fpad, ctx->m, ctx->dscal, ctx->n, ctx->dscal + 1, ctx->stream));
  MARK(5);
#undef MARK
  return VIF_OK;
}

vif_status read_status(vif_ctx* ctx, double* scal_out, int nscal) {
  // one D2H copy of the status words and the requested scalars
  CK(cudaMemcpyAsync(ctx->h_pin, ctx->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (nscal > 0)
    CK(cudaMemcpyAsync(ctx->h_pin + 2, ctx->dscal + 1, nscal * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int* st = reinterpret_cast<const int*>(ctx->h_pin);
  if (st[0] != ST_OK) {
    char why[200];
    const vif_status e = status_error(st, why, sizeof(why));
    return set_err(ctx, e, "%s", why);
  }
  for (int k = 0; k < nscal; ++k) scal_out[k] = ctx->h_pin[2 + k];
  return VIF_OK;
}

void free_ctx(vif_ctx* c) {
  if (!c) return;
  void* bufs[] = {c->X,    c->Z,     c->Xs, c->Zs,   c->Xs32, c->Zs32, c->hyp, c->N,   c->order, c->Sm, c->trw,
                  c->Linv, c->LinvT, c->A,  c->F,    c->Acoef, c->Dv,  c->logD, c->part, c->G,
                  c->y,    c->red,   c->dscal, c->status, c->ug_rows, c->ug_ptr, c->ug_loc, c->gsub};
  for (void* b : bufs)
    if (b) cudaFree(b);
  void* pbufs[] = {c->pA,     c->pF,    c->pLinvT, c->pXp,    c->pXps,   c->pAp,    c->pcpp,   c->pmean,
                   c->pvar,   c->pNp,   c->pcjj,   c->pw,     c->pr,     c->pLinvC, c->ch_ptr, c->ch_row,
                   c->ch_slot, c->l_b,  c->l_W,    c->l_v,    c->l_Ginv, c->l_om,   c->l_rsD,  c->l_ll,
                   c->l_x,    c->l_r,   c->l_z,    c->l_p,    c->l_Ap,   c->l_t,    c->l_t2,   c->l_x1,
                   c->l_sdi,  c->l_sm,  c->l_cm,   c->l_tm,   c->l_part, c->l_LinvC, c->l_G3,  c->l_LinvC3,
                   c->l_sc,   c->l_red, c->l_corr, c->sched_fwd, c->sched_rev, c->ord_fwd, c->ord_rev, c->ch_coef, c->slq_eps, c->l_Apad, c->l_anorm2, c->l_dvinv, c->l_pacc, c->l_counter, c->l_abort, c->m_feat, c->m_rho, c->gr_buf, c->gr_LinvC, c->gr_out,
                   c->g_U,    c->g_Y,   c->g_g,    c->g_v,    c->g_sc,   c->g_red,  c->g_a,    c->g_av,
                   c->g_dv,
                   c->mr_v,   c->mr_x,  c->mr_r,   c->mr_z,   c->mr_p,   c->mr_Ap,  c->mr_t,   c->mr_t2,
                   c->mr_x1,  c->mr_sm, c->mr_cm,  c->mr_tm,  c->mr_part, c->mr_dpart, c->mr_sc, c->mr_active, c->mr_map,
                   c->m_gc,   c->m_part, c->m_grad};
  for (void* b : pbufs)
    if (b) cudaFree(b);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

// Neighbour search under the build hyperparameters (float64 A plus a float32 copy).
vif_status build_neighbors(vif_ctx* ctx, const vif_cov* cv) {
  const int64_t n = ctx->n;
  const int mv = ctx->mv;
  if (mv == 0 || n == 0) return VIF_OK;
  CovParams cp = cov_params(cv);
  CKS(apply_scaling(ctx, cv, true));
  double* A64 = nullptr;
  double* LinvT64 = nullptr;
  float *A32 = nullptr, *rs32 = nullptr, *nrm32 = nullptr, *ckey = nullptr, *ce = nullptr, *lowb = nullptr;
  double* cii = nullptr;
  int32_t *cidx = nullptr, *fb = nullptr;
  const int kprime = (mv <= 24) ? 32 : 64;
  vif_status st = VIF_OK;
  auto cleanup = [&]() {
    void* b[] = {A64, LinvT64, A32, rs32, nrm32, ckey, ce, lowb, cii, cidx, fb};
    for (void* x : b)
      if (x) cudaFree(x);
  };
  do {
    if ((st = dalloc(ctx, &A64, (size_t)n * ctx->mpad)) != VIF_OK) break;
    if ((st = dalloc(ctx, &LinvT64, (size_t)ctx->mpad * ctx->mpad)) != VIF_OK) break;
    if ((st = dalloc(ctx, &A32, (size_t)n * ctx->mpad)) != VIF_OK) break;
    if ((st = dalloc(ctx, &rs32, n)) != VIF_OK) break;
    if ((st = dalloc(ctx, &nrm32, n)) != VIF_OK) break;
    if ((st = dalloc(ctx, &cii, n)) != VIF_OK) break;
    if ((st = dalloc(ctx, &ckey, (size_t)n * kprime)) != VIF_OK) break;
    if ((st = dalloc(ctx, &ce, (size_t)n * kprime)) != VIF_OK) break;
    if ((st = dalloc(ctx, &cidx, (size_t)n * kprime)) != VIF_OK) break;
    if ((st = dalloc(ctx, &lowb, n)) != VIF_OK) break;
    if ((st = dalloc(ctx, &fb, n)) != VIF_OK) break;
    cudaError_t e = cudaMemsetAsync(ctx->status, 0, 16 * sizeof(int), ctx->stream);
    if (e != cudaSuccess) {
      st = set_err(ctx, VIF_ERR_CUDA, "%s", cudaGetErrorString(e));
      break;
    }
    if ((st = compute_lowrank<double>(ctx, cp, A64, LinvT64, ctx->Xs, ctx->Zs)) != VIF_OK) break;
    const double tau = 1e-6 * cv->variance;
    e = residual_diag_stats(A64, n, ctx->m, ctx->mpad, cv->variance, tau, A32, cii, rs32, nrm32, ctx->stream);
    if (e != cudaSuccess) {
      st = set_err(ctx, VIF_ERR_CUDA, "residual_diag_stats: %s", cudaGetErrorString(e));
      break;
    }
    // error constants of the float32 filter (u = 2^-24)
    const double u = std::ldexp(1.0, -24);
    // float32 dot products are summed in chunks of 32 (see the filter kernel):
    // |error| <= gamma_k sum|a_ik a_jk|, k = 32 + ceil(m/32) + 2 (chunk sum, total,
    // rounding of A to float32), with sum|a_ik a_jk| <= ||a_i|| ||a_j||.
    const int kk = 32 + (std::max(ctx->m, 1) + 31) / 32 + 2;
    const double gam = kk * u / (1.0 - kk * u) + 1e-12;
    // max |scaled coordinate| norm over the data (centred), from the host copy kept at build
    double R = 0.0;
    {
      std::vector<double> hx((size_t)n * ctx->d);
      e = cudaMemcpyAsync(hx.data(), ctx->Xs, hx.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) {
        st = set_err(ctx, VIF_ERR_CUDA, "%s", cudaGetErrorString(e));
        break;
      }
      for (int64_t i = 0; i < n; ++i) {
        double s2 = 0;
        for (int t = 0; t < ctx->d; ++t) s2 += hx[(size_t)i * ctx->d + t] * hx[(size_t)i * ctx->d + t];
        R = std::max(R, std::sqrt(s2));
      }
    }
    const double epsK = cv->variance * u * (4.0 * R + 2.0 * ctx->d + 36.0);
    KnnParams kp;
    kp.n = n;
    kp.d = ctx->d;
    kp.m = ctx->m;
    kp.mpad = ctx->mpad;
    kp.mv = mv;
    kp.kprime = kprime;
    kp.kind = cv->kind;
    kp.var = cv->variance;
    kp.tau_v = tau;
    kp.gamma = (float)(gam * (1.0 + 1e-6));
    kp.epsK = (float)(epsK * (1.0 + 1e-6));
    e = knn_causal(kp, A32, A64, ctx->Xs32, ctx->Xs, cii, rs32, nrm32, ckey, cidx, ce, lowb, ctx->N,
                   ctx->status + 4, fb, ctx->stream);
    if (e != cudaSuccess) {
      st = set_err(ctx, VIF_ERR_CUDA, "knn_causal: %s", cudaGetErrorString(e));
      break;
    }
    int hc[2];
    e = cudaMemcpyAsync(hc, ctx->status + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      st = set_err(ctx, VIF_ERR_CUDA, "%s", cudaGetErrorString(e));
      break;
    }
    ctx->knn_rescored = hc[0];
    ctx->knn_fallback = hc[1];
    double dummy[1];
    st = read_status(ctx, dummy, 0);
  } while (0);
  cleanup();
  return st;
}

}  // namespace

namespace {

// Processing order for the per-point kernels: points sorted by the Morton (Z-order)
// code of their ARD-scaled coordinates, so that consecutive warps gather
// neighbour rows that are close in space and likely still in L2.  This only
// changes the order in which independent points are processed, never a result.
std::vector<int32_t> morton_order(const std::vector<double>& hx, int64_t n, int d, const vif_cov* cov) {
  const int bits = std::min(21, 63 / d);
  std::vector<double> lo(d), hi(d);
  for (int t = 0; t < d; ++t) {
    lo[t] = hi[t] = hx[t];
    for (int64_t i = 0; i < n; ++i) {
      lo[t] = std::min(lo[t], hx[(size_t)i * d + t]);
      hi[t] = std::max(hi[t], hx[(size_t)i * d + t]);
    }
  }
  // equal cells in the scaled space: the longest scaled extent sets the resolution
  double ext = 0.0;
  for (int t = 0; t < d; ++t) ext = std::max(ext, (hi[t] - lo[t]) / cov->lengthscale[cov->n_ls == 1 ? 0 : t]);
  if (!(ext > 0.0)) ext = 1.0;
  const double cells = (double)((1ull << bits) - 1);
  std::vector<uint64_t> code(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t c = 0;
    for (int t = 0; t < d; ++t) {
      double v = (hx[(size_t)i * d + t] - lo[t]) / cov->lengthscale[cov->n_ls == 1 ? 0 : t] / ext;
      uint64_t q = (uint64_t)std::min(cells, std::max(0.0, v * cells));
      for (int b = 0; b < bits; ++b) c |= ((q >> b) & 1ull) << (b * d + t);
    }
    code[i] = c;
  }
  std::vector<int32_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = (int32_t)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
  return ord;
}

}  // namespace

namespace {

// float64 buffers of the likelihood pipeline (the context's own, or float64 twins
// allocated on first use for a mixed-precision context).
vif_status fp64_buffers(vif_ctx* ctx, double** A64, double** F64, double** LT64) {
  if (ctx->precision == VIF_FP64) {
    *A64 = (double*)ctx->A;
    *F64 = (double*)ctx->F;
    *LT64 = (double*)ctx->LinvT;
    return VIF_OK;
  }
  if (!ctx->pA) {
    CKS(dalloc(ctx, &ctx->pA, (size_t)ctx->n * ctx->mpad));
    CKS(dalloc(ctx, &ctx->pF, (size_t)ctx->n * ctx->fpad));
    CKS(dalloc(ctx, &ctx->pLinvT, (size_t)ctx->mpad * ctx->mpad));
    CK(cudaMemsetAsync(ctx->pA, 0, (size_t)ctx->n * ctx->mpad * sizeof(double), ctx->stream));
  }
  *A64 = ctx->pA;
  *F64 = ctx->pF;
  *LT64 = ctx->pLinvT;
  return VIF_OK;
}


// Groups of the float32 path's tensor-core Gram (vif_factor_tc.cu) from the neighbour sets
// N (host copy) and the processing order; the context keeps the SIMT factor kernel when the
// sets do not qualify (m = 0, m_v = 0, m_v + 1 > 32) or a group cannot be formed.
vif_status build_groups(vif_ctx* ctx, const int32_t* hN) {
  ctx->ug_ready = false;
  if (ctx->precision != VIF_MIXED || ctx->factor_mode == 1 || ctx->mv < 1 || ctx->mv + 1 > 32 || ctx->m < 1 ||
      (int64_t)ctx->h_order.size() != ctx->n)
    return VIF_OK;
  std::vector<int32_t> rows, ptr;
  std::vector<unsigned char> loc;
  if (!build_union_groups(hN, ctx->h_order.data(), ctx->n, ctx->mv, UG_MAX_POINTS, rows, ptr, loc)) return VIF_OK;
  for (void* b : {(void*)ctx->ug_rows, (void*)ctx->ug_ptr, (void*)ctx->ug_loc})
    if (b) cudaFree(b);
  ctx->ug_rows = nullptr;
  ctx->ug_ptr = nullptr;
  ctx->ug_loc = nullptr;
  CKS(dalloc(ctx, &ctx->ug_rows, rows.size()));
  CKS(dalloc(ctx, &ctx->ug_ptr, ptr.size()));
  CKS(dalloc(ctx, &ctx->ug_loc, loc.size()));
  if (!ctx->gsub) CKS(dalloc(ctx, &ctx->gsub, (size_t)ctx->n * ((ctx->mv + 1) * (ctx->mv + 2) / 2)));
  CK(cudaMemcpy(ctx->ug_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ug_ptr, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ug_loc, loc.data(), loc.size(), cudaMemcpyHostToDevice));
  ctx->ug_ngroups = (int64_t)ptr.size() - 1;
  ctx->ug_ready = true;
  ctx->factor_choice = -1;   // new groups: tune again
  return VIF_OK;
}

// Children lists of the neighbour DAG (the transpose of N, by column), for B^T.
// Slots {row, first term, end of terms, solo} of a sync-free triangular solve, rows
// ordered by level: level[r] is 0 for a row that reads no other row, else one more
// than the deepest row it reads.  Within a level, rows with more than TRSV_SOLO_TERMS
// terms get a step of their own (four copies of their slot, solo = 1: the whole warp on
// one row); the others fill steps of LAP_TRSV_RPS rows, the level padded with
// {-1, 0, 0, 0}, so the rows of one step never read one another.
constexpr int TRSV_SOLO_TERMS = 24;
static std::vector<int4> level_schedule(const std::vector<int32_t>& level, const std::vector<int32_t>& first,
                                        const std::vector<int32_t>& count, bool allow_solo) {
  int32_t nlev = 0;
  for (int32_t l : level) nlev = std::max(nlev, l + 1);
  auto solo = [&](size_t r) { return allow_solo && count[r] > TRSV_SOLO_TERMS; };
  std::vector<int64_t> cnt((size_t)nlev, 0), nsolo((size_t)nlev, 0);
  for (size_t r = 0; r < level.size(); ++r) (solo(r) ? nsolo : cnt)[(size_t)level[r]]++;
  std::vector<int64_t> start((size_t)nlev + 1, 0), split((size_t)nlev, 0);
  for (int32_t l = 0; l < nlev; ++l) {
    split[(size_t)l] = start[(size_t)l] + nsolo[(size_t)l] * LAP_TRSV_RPS;
    const int64_t padded = (cnt[(size_t)l] + LAP_TRSV_RPS - 1) / LAP_TRSV_RPS * LAP_TRSV_RPS;
    start[(size_t)l + 1] = split[(size_t)l] + padded;
  }
  std::vector<int4> sched((size_t)std::max<int64_t>(start[(size_t)nlev], LAP_TRSV_RPS), make_int4(-1, 0, 0, 0));
  std::vector<int64_t> fs(start.begin(), start.end() - 1), fr(split);
  for (size_t r = 0; r < level.size(); ++r) {
    const size_t l = (size_t)level[r];
    const int4 slot = make_int4((int)r, first[r], first[r] + count[r], solo(r) ? 1 : 0);
    if (solo(r)) {
      for (int k = 0; k < LAP_TRSV_RPS; ++k) sched[(size_t)fs[l] + k] = slot;
      fs[l] += LAP_TRSV_RPS;
    } else {
      sched[(size_t)fr[l]++] = slot;
    }
  }
  return sched;
}

// Children lists of B (CSR over the rows that name j as a neighbour) and the level
// schedules of the two triangular solves, from the neighbour sets.
vif_status build_children(vif_ctx* ctx) {
  const int64_t n = ctx->n;
  const int mv = ctx->mv;
  if (n * std::max(mv, 1) >= ((int64_t)1 << 31))
    return set_err(ctx, VIF_ERR_ARG, "n * m_v must stay below 2^31 for the Laplace solves");
  std::vector<int32_t> N((size_t)n * std::max(mv, 1), -1);
  if (mv > 0) {
    CK(cudaMemcpyAsync(N.data(), ctx->N, (size_t)n * mv * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  std::vector<int32_t> ptr(n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int t = 0; t < mv; ++t) {
      int j = N[(size_t)i * mv + t];
      if (j >= 0) ptr[j + 1]++;
    }
  for (int64_t j = 0; j < n; ++j) ptr[j + 1] += ptr[j];
  const int64_t nnz = ptr[n];
  std::vector<int32_t> row(std::max<int64_t>(nnz, 1)), slot(std::max<int64_t>(nnz, 1));
  std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int t = 0; t < mv; ++t) {
      int j = N[(size_t)i * mv + t];
      if (j >= 0) {
        row[fill[j]] = (int32_t)i;
        slot[fill[j]] = t;
        fill[j]++;
      }
    }
  // B^{-1}: row i reads its neighbours (all earlier); B^{-T}: row j reads its children (all later)
  std::vector<int32_t> lev((size_t)n, 0), rlev((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int q = (int)std::min<int64_t>(i, mv);
    int32_t l = 0;
    for (int t = 0; t < q; ++t) {
      const int j = N[(size_t)i * mv + t];
      // the solves read row j while computing row i: it must be an earlier row
      if (j < 0 || j >= i) return set_err(ctx, VIF_ERR_ARG, "neighbour %d of row %lld is not a predecessor", j,
                                          (long long)i);
      l = std::max(l, lev[j] + 1);
    }
    lev[i] = l;
  }
  for (int64_t j = n - 1; j >= 0; --j) {
    int32_t l = 0;
    for (int32_t p = ptr[j]; p < ptr[j + 1]; ++p)
      if (row[p] > j) l = std::max(l, rlev[row[p]] + 1);
    rlev[j] = l;
  }
  // terms: row i of B^{-1} reads N[i m_v + k], k < min(i, m_v); row j of B^{-T} its children
  std::vector<int32_t> f_first((size_t)n), f_cnt((size_t)n), r_cnt((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    f_first[(size_t)i] = (int32_t)(i * mv);
    f_cnt[(size_t)i] = (int32_t)std::min<int64_t>(i, mv);
    r_cnt[(size_t)i] = ptr[i + 1] - ptr[i];
  }
  const std::vector<int4> sf = level_schedule(lev, f_first, f_cnt, false);
  const std::vector<int4> sr = level_schedule(rlev, std::vector<int32_t>(ptr.begin(), ptr.end() - 1), r_cnt, true);
  // every row once in level order (counting sort by level), for the block solves
  auto row_order = [&](const std::vector<int32_t>& level, const std::vector<int32_t>& first,
                       const std::vector<int32_t>& count) {
    int32_t nlev = 0;
    for (int32_t l : level) nlev = std::max(nlev, l + 1);
    std::vector<int64_t> at((size_t)nlev + 1, 0);
    for (int32_t l : level) at[(size_t)l + 1]++;
    for (int32_t l = 0; l < nlev; ++l) at[(size_t)l + 1] += at[(size_t)l];
    std::vector<int4> ord((size_t)n);
    for (int64_t r = 0; r < n; ++r)
      ord[(size_t)at[(size_t)level[(size_t)r]]++] =
          make_int4((int)r, first[(size_t)r], first[(size_t)r] + count[(size_t)r], 0);
    return ord;
  };
  const std::vector<int4> of = row_order(lev, f_first, f_cnt);
  const std::vector<int4> orv = row_order(rlev, std::vector<int32_t>(ptr.begin(), ptr.end() - 1), r_cnt);
  if (!ctx->ch_ptr) {
    CKS(dalloc(ctx, &ctx->ch_ptr, (size_t)n + 1));
  }
  void* owned[] = {ctx->ch_row, ctx->ch_slot, ctx->sched_fwd, ctx->sched_rev, ctx->ch_coef, ctx->ord_fwd,
                   ctx->ord_rev};
  for (void* b : owned)
    if (b) cudaFree(b);
  ctx->ch_row = ctx->ch_slot = nullptr;
  ctx->sched_fwd = ctx->sched_rev = nullptr;
  ctx->ord_fwd = ctx->ord_rev = nullptr;
  ctx->ch_coef = nullptr;
  CKS(dalloc(ctx, &ctx->ch_row, (size_t)std::max<int64_t>(nnz, 1)));
  CKS(dalloc(ctx, &ctx->ch_slot, (size_t)std::max<int64_t>(nnz, 1)));
  CKS(dalloc(ctx, &ctx->sched_fwd, sf.size()));
  CKS(dalloc(ctx, &ctx->sched_rev, sr.size()));
  CKS(dalloc(ctx, &ctx->ch_coef, (size_t)std::max<int64_t>(nnz, 1)));
  CKS(dalloc(ctx, &ctx->ord_fwd, (size_t)n));
  CKS(dalloc(ctx, &ctx->ord_rev, (size_t)n));
  ctx->ch_nnz = nnz;
  ctx->nsteps_fwd = (int64_t)(sf.size() / LAP_TRSV_RPS);
  ctx->nsteps_rev = (int64_t)(sr.size() / LAP_TRSV_RPS);
  CK(cudaMemcpy(ctx->ch_ptr, ptr.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ch_row, row.data(), row.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ch_slot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->sched_fwd, sf.data(), sf.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->sched_rev, sr.data(), sr.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ord_fwd, of.data(), of.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ord_rev, orv.data(), orv.size() * sizeof(int4), cudaMemcpyHostToDevice));
  return VIF_OK;
}

vif_status lap_alloc(vif_ctx* ctx) {
  if (ctx->lap_ready) return VIF_OK;
  const int64_t n = ctx->n;
  double** vecs[] = {&ctx->l_b, &ctx->l_W,  &ctx->l_v,  &ctx->l_Ginv, &ctx->l_om, &ctx->l_rsD, &ctx->l_ll,
                     &ctx->l_x, &ctx->l_r,  &ctx->l_z,  &ctx->l_p,    &ctx->l_Ap, &ctx->l_t,   &ctx->l_t2,
                     &ctx->l_x1, &ctx->l_sdi, &ctx->l_corr};
  for (double** v : vecs) CKS(dalloc(ctx, v, (size_t)n));
  CKS(dalloc(ctx, &ctx->l_sm, (size_t)ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_cm, (size_t)ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_tm, (size_t)ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_part, (size_t)LAP_FT_BLOCKS * ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_LinvC, (size_t)std::max(ctx->m, 1) * ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_G3, (size_t)(ctx->m + 1) * ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_LinvC3, (size_t)std::max(ctx->m, 1) * ctx->fpad));
  CKS(dalloc(ctx, &ctx->l_sc, 16));
  CKS(dalloc(ctx, &ctx->l_red, 256));
  CKS(dalloc(ctx, &ctx->l_counter, 4));
  CKS(dalloc(ctx, &ctx->l_abort, 2));   // [0] abort flag, [1] poll bound of the waits (0: default)
  CK(cudaMemsetAsync(ctx->l_sm, 0, ctx->fpad * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->l_cm, 0, ctx->fpad * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->l_G3, 0, (size_t)(ctx->m + 1) * ctx->fpad * sizeof(double), ctx->stream));
  CKS(build_children(ctx));
  ctx->lap_ready = true;
  return VIF_OK;
}

// Prediction buffers for np points (grown on demand) and the n-sized ones.
vif_status predict_buffers(vif_ctx* ctx, int64_t np) {
  const int d = ctx->d, m = ctx->m, mpad = ctx->mpad, fpad = ctx->fpad, mv = ctx->mv;
  const int64_t n = ctx->n;
  if (np > ctx->p_cap) {
    double* pb[] = {ctx->pXp, ctx->pXps, ctx->pAp, ctx->pcpp, ctx->pmean, ctx->pvar};
    for (double* b : pb)
      if (b) cudaFree(b);
    if (ctx->pNp) cudaFree(ctx->pNp);
    ctx->pXp = ctx->pXps = ctx->pAp = ctx->pcpp = ctx->pmean = ctx->pvar = nullptr;
    ctx->pNp = nullptr;
    ctx->p_cap = 0;
    CKS(dalloc(ctx, &ctx->pXp, (size_t)np * d));
    CKS(dalloc(ctx, &ctx->pXps, (size_t)np * d));
    CKS(dalloc(ctx, &ctx->pAp, (size_t)np * mpad));
    CKS(dalloc(ctx, &ctx->pcpp, (size_t)np));
    CKS(dalloc(ctx, &ctx->pmean, (size_t)np));
    CKS(dalloc(ctx, &ctx->pvar, (size_t)np));
    CKS(dalloc(ctx, &ctx->pNp, (size_t)np * std::max(mv, 1)));
    ctx->p_cap = np;
  }
  if (!ctx->pcjj) {
    CKS(dalloc(ctx, &ctx->pcjj, (size_t)n));
    CKS(dalloc(ctx, &ctx->pw, (size_t)mpad));
    CKS(dalloc(ctx, &ctx->pr, (size_t)n));
    CKS(dalloc(ctx, &ctx->pLinvC, (size_t)std::max(m, 1) * fpad));
    CK(cudaMemsetAsync(ctx->pw, 0, (size_t)mpad * sizeof(double), ctx->stream));
  }
  return VIF_OK;
}

}  // namespace

void vif_internal_set_global_error(const char* msg) { snprintf(g_build_err, sizeof(g_build_err), "%s", msg); }

extern "C" {

vif_status vif_build(const double* X, int64_t n, int32_t d, const double* Z, int32_t m, int32_t mv,
                     const vif_cov* cov, const vif_opts* opts, void* stream, vif_ctx** out) {
  if (!out) return VIF_ERR_ARG;
  *out = nullptr;
  if (!X || n < 1 || d < 1 || d > 16 || m < 0 || m > 2048 || mv < 0 || mv > 48 || (m > 0 && !Z) || !opts)
    return VIF_ERR_ARG;
  if (opts->precision != VIF_FP64 && opts->precision != VIF_MIXED) return VIF_ERR_ARG;
  if (opts->likelihood != VIF_GAUSSIAN && opts->likelihood != VIF_BERNOULLI_LOGIT) return VIF_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (opts->reserved[k] != 0) return VIF_ERR_ARG;
  if (opts->factor_path < 0 || opts->factor_path > 2) return VIF_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return VIF_ERR_CUDA;
  }
  vif_ctx* ctx = new vif_ctx();
  vif_status st = check_cov(ctx, cov, d);
  if (st != VIF_OK) {
    free_ctx(ctx);
    return st;
  }
  cudaGetDevice(&ctx->dev);
  ctx->stream = (cudaStream_t)stream;
  ctx->n = n;
  ctx->d = d;
  ctx->m = m;
  ctx->mv = mv;
  ctx->mpad = std::max(32, ((m + 31) / 32) * 32);
  ctx->ldm = ctx->mpad;
  ctx->fpad = ((m + 1 + 63) / 64) * 64;
  ctx->precision = opts->precision;
  ctx->likelihood = opts->likelihood;
  ctx->timing = opts->stage_timing != 0;
  ctx->factor_mode = opts->factor_path;
  if (ctx->timing)
    for (auto& e : ctx->ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        free_ctx(ctx);
        return VIF_ERR_CUDA;
      }
  const bool mixed = ctx->precision == VIF_MIXED;
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  if (cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->dev) != cudaSuccess) {
    cudaGetLastError();
    ctx->nsm = 1;
  }
  if (mixed) {
    cudaError_t e = lowrank_A_tc_init();
    if (e == cudaSuccess) e = gram_tc_init();
    if (e == cudaSuccess) e = union_gram_tc_init();
    if (e != cudaSuccess) {
      vif_internal_set_global_error(cudaGetErrorString(e));
      free_ctx(ctx);
      return VIF_ERR_CUDA;
    }
  }
#define ALLOC(ptr, cnt)                                 \
  do {                                                  \
    if ((st = dalloc(ctx, &(ptr), (cnt))) != VIF_OK) { \
      *out = nullptr;                                   \
      vif_status s2 = st;                               \
      free_ctx(ctx);                                    \
      return s2;                                        \
    }                                                   \
  } while (0)
  ALLOC(ctx->X, (size_t)n * d);
  ALLOC(ctx->Z, (size_t)std::max(m, 1) * d);
  ALLOC(ctx->Xs, (size_t)n * d);
  ALLOC(ctx->Zs, (size_t)std::max(m, 1) * d);
  ALLOC(ctx->Xs32, (size_t)n * d);
  ALLOC(ctx->Zs32, (size_t)std::max(m, 1) * d);
  ALLOC(ctx->hyp, 32);
  ALLOC(ctx->N, (size_t)n * std::max(mv, 1));
  ALLOC(ctx->order, (size_t)n);
  ALLOC(ctx->Sm, (size_t)ctx->ldm * ctx->ldm);
  ALLOC(ctx->Linv, (size_t)ctx->ldm * ctx->ldm);
  ALLOC(ctx->trw, trtri_work_doubles(m + 1));
  {
    unsigned char* p = nullptr;
    size_t lt_bytes = (size_t)ctx->mpad * ctx->mpad * esz;
    if (esz == 4) lt_bytes = std::max(lt_bytes, lowrank_A_tc_pack_floats(ctx->mpad) * sizeof(float));
    ALLOC(p, lt_bytes);
    ctx->LinvT = p;
    p = nullptr;
    ALLOC(p, (size_t)n * ctx->mpad * esz);
    ctx->A = p;
    p = nullptr;
    ALLOC(p, (size_t)n * ctx->fpad * esz);
    ctx->F = p;
  }
  ALLOC(ctx->Acoef, (size_t)n * std::max(mv, 1));
  if (ctx->likelihood != VIF_GAUSSIAN) {
    ALLOC(ctx->m_rho, 2 * (size_t)n);
    cudaMemset(ctx->m_rho, 0, 2 * sizeof(float) * (size_t)n);   // read before the first factorization
  }
  ALLOC(ctx->Dv, (size_t)n);
  ALLOC(ctx->logD, (size_t)n);
  ctx->nsplit = gram_nsplit(n, ctx->fpad);
  {
    int nt = ctx->fpad / 64;
    ALLOC(ctx->part, (size_t)ctx->nsplit * (nt * (nt + 1) / 2) * 64 * 64);
  }
  ALLOC(ctx->G, (size_t)(m + 1) * ctx->fpad);
  ALLOC(ctx->y, (size_t)n);
  ALLOC(ctx->red, 256);
  ALLOC(ctx->dscal, 16);
  ALLOC(ctx->status, 16);
#undef ALLOC
  if (cudaMallocHost((void**)&ctx->h_pin, 4096) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(ctx);
    return VIF_ERR_NOMEM;
  }
  // upload coordinates, centre of the data box (for float32 conditioning)
  std::vector<double> hx((size_t)n * d);
  if (is_device_ptr(X)) {
    if (cudaMemcpy(hx.data(), X, hx.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      free_ctx(ctx);
      return VIF_ERR_CUDA;
    }
  } else {
    memcpy(hx.data(), X, hx.size() * sizeof(double));
  }
  for (int t = 0; t < d; ++t) {
    double lo = hx[t], hi = hx[t];
    for (int64_t i = 0; i < n; ++i) {
      lo = std::min(lo, hx[(size_t)i * d + t]);
      hi = std::max(hi, hx[(size_t)i * d + t]);
    }
    ctx->center[t] = 0.5 * (lo + hi);
  }
  {
    ctx->h_order = morton_order(hx, n, d, cov);
    if (cudaMemcpy(ctx->order, ctx->h_order.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      free_ctx(ctx);
      return VIF_ERR_CUDA;
    }
  }
  if ((st = upload(ctx, ctx->X, X, (size_t)n * d * sizeof(double))) != VIF_OK ||
      (m > 0 && (st = upload(ctx, ctx->Z, Z, (size_t)m * d * sizeof(double))) != VIF_OK)) {
    free_ctx(ctx);
    return st;
  }
  // buffers whose padding must be zero
  cudaMemsetAsync(ctx->A, 0, (size_t)n * ctx->mpad * esz, ctx->stream);
  cudaMemsetAsync(ctx->G, 0, (size_t)(m + 1) * ctx->fpad * sizeof(double), ctx->stream);
  if (mv > 0) cudaMemsetAsync(ctx->N, 0xff, (size_t)n * mv * sizeof(int32_t), ctx->stream);
  st = opts->no_neighbor_search ? VIF_OK : build_neighbors(ctx, cov);
  if (st != VIF_OK) {
    snprintf(g_build_err, sizeof(g_build_err), "%s", ctx->err);
    free_ctx(ctx);
    return st;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    free_ctx(ctx);
    return VIF_ERR_CUDA;
  }
  if (mixed && mv > 0 && !opts->no_neighbor_search) {
    std::vector<int32_t> hN((size_t)n * mv);
    if (cudaMemcpy(hN.data(), ctx->N, hN.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (st = build_groups(ctx, hN.data())) != VIF_OK) {
      snprintf(g_build_err, sizeof(g_build_err), "%s", ctx->err[0] ? ctx->err : "group construction failed");
      free_ctx(ctx);
      return st != VIF_OK ? st : VIF_ERR_CUDA;
    }
  }
  *out = ctx;
  return VIF_OK;
}

// The autotuner of the float32 factor stage (first evaluation of a context whose groups
// exist): time the stage once on the tensor cores and once on the CUDA cores, on the A just
// formed, and keep the faster.  The CUDA-core run comes last, so the factors left in the
// context are those the evaluation itself produced.
vif_status tune_factor(vif_ctx* ctx, const CovParams& cp) {
  cudaEvent_t ev[3];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  struct G {
    cudaEvent_t* e;
    ~G() {
      for (int k = 0; k < 3; ++k) cudaEventDestroy(e[k]);
    }
  } guard{ev};
  float* A = (float*)ctx->A;
  float* F = (float*)ctx->F;
  CK(cudaEventRecord(ev[0], ctx->stream));
  CKS(run_factor<float>(ctx, cp, A, ctx->Xs32, F, true));
  CK(cudaEventRecord(ev[1], ctx->stream));
  CKS(run_factor<float>(ctx, cp, A, ctx->Xs32, F, false));
  CK(cudaEventRecord(ev[2], ctx->stream));
  CK(cudaEventSynchronize(ev[2]));
  CK(cudaEventElapsedTime(&ctx->factor_ms[1], ev[0], ev[1]));
  CK(cudaEventElapsedTime(&ctx->factor_ms[0], ev[1], ev[2]));
  ctx->factor_choice = ctx->factor_ms[1] < ctx->factor_ms[0] ? 1 : 0;
  return VIF_OK;
}

vif_status vif_nll(vif_ctx* ctx, const vif_cov* theta, const double* y, double* nll_out, double* grad_out) {
  if (!ctx) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  if (!y || !nll_out) return set_err(ctx, VIF_ERR_ARG, "y and nll_out are required");
  CKS(check_cov(ctx, theta, ctx->d));
  if (grad_out && !(theta->nugget > 0.0))
    return set_err(ctx, VIF_ERR_ARG, "the gradient needs a positive nugget");
  if (ctx->likelihood != VIF_GAUSSIAN)
    return set_err(ctx, VIF_ERR_STATE, "vif_nll needs a context built for the Gaussian likelihood");
  const bool mixed = ctx->precision == VIF_MIXED;
  CovParams cp = cov_params(theta);
  CK(cudaMemsetAsync(ctx->status, 0, 4 * sizeof(int), ctx->stream));
  CKS(upload(ctx, ctx->y, y, (size_t)ctx->n * sizeof(double)));
  if (grad_out) {
    // the analytic gradient (vif_grad.cu) from a float64 evaluation
    double *A64 = nullptr, *F64 = nullptr, *LT64 = nullptr;
    CKS(fp64_buffers(ctx, &A64, &F64, &LT64));
    CKS(apply_scaling(ctx, theta, false));
    CKS(run_pipeline<double>(ctx, cp, A64, LT64, F64, ctx->Xs, ctx->Zs));
    double sc64[1];
    CKS(read_status(ctx, sc64, 1));
    const int q = theta->n_ls + 2;
    if (!ctx->gr_buf) {
      CKS(dalloc(ctx, &ctx->gr_buf, grad_scratch_doubles(ctx->n, ctx->m, ctx->mv, 18)));
      CKS(dalloc(ctx, &ctx->gr_LinvC, (size_t)ctx->fpad * ctx->fpad));
      CKS(dalloc(ctx, &ctx->gr_out, 64));
    }
    std::vector<double> hls(theta->lengthscale, theta->lengthscale + theta->n_ls);
    GradInputs in{};
    in.A = A64;
    in.F = F64;
    in.Xs = ctx->Xs;
    in.Zs = ctx->Zs;
    in.Acoef = ctx->Acoef;
    in.Dv = ctx->Dv;
    in.y = ctx->y;
    in.G = ctx->G;
    in.Linv = ctx->Linv;
    in.ls = hls.data();
    in.N = ctx->N;
    in.n = ctx->n;
    in.d = ctx->d;
    in.m = ctx->m;
    in.mpad = ctx->mpad;
    in.fpad = ctx->fpad;
    in.mv = ctx->mv;
    in.ldl = ctx->ldm;
    in.nls = theta->n_ls;
    in.cp = cp;
    CK(vif_grad_fp64(in, ctx->gr_buf, ctx->gr_LinvC, ctx->trw, ctx->gr_out, ctx->stream));
    double g3[3 * 18];
    CKS(download(ctx, g3, ctx->gr_out, sizeof(double) * 3 * q));
    for (int k = 0; k < q; ++k) grad_out[k] = g3[k] + g3[q + k] + g3[2 * q + k];
    if (!mixed) {   // the float64 evaluation above is the likelihood
      ctx->have_factors = true;
      *nll_out = sc64[0];
      return VIF_OK;
    }
    CK(cudaMemsetAsync(ctx->status, 0, 4 * sizeof(int), ctx->stream));
  }
  CKS(apply_scaling(ctx, theta, mixed));
  if (mixed) {
    CKS(run_pipeline<float>(ctx, cp, (float*)ctx->A, (float*)ctx->LinvT, (float*)ctx->F, ctx->Xs32, ctx->Zs32));
    if (ctx->ug_ready && ctx->factor_mode == 0 && ctx->factor_choice < 0) CKS(tune_factor(ctx, cp));
  } else {
    CKS(run_pipeline<double>(ctx, cp, (double*)ctx->A, (double*)ctx->LinvT, (double*)ctx->F, ctx->Xs, ctx->Zs));
  }
  double sc[3];
  CKS(read_status(ctx, sc, 3));
  ctx->have_factors = true;
  *nll_out = sc[0];
  return VIF_OK;
}

vif_status vif_predict(vif_ctx* ctx, const vif_cov* theta, const double* y, const double* Xp, int64_t np,
                       int32_t latent, double* mean, double* var) {
  if (!ctx) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  if (!y || !Xp || !mean || np < 1) return set_err(ctx, VIF_ERR_ARG, "y, Xp, mean and np >= 1 are required");
  CKS(check_cov(ctx, theta, ctx->d));
  if (ctx->likelihood != VIF_GAUSSIAN)
    return set_err(ctx, VIF_ERR_STATE, "vif_predict needs a context built for the Gaussian likelihood");
  if (ctx->mv > 48) return set_err(ctx, VIF_ERR_ARG, "m_v too large for prediction");
  const int64_t n = ctx->n;
  const int d = ctx->d, m = ctx->m, mpad = ctx->mpad, fpad = ctx->fpad, mv = ctx->mv;
  double *A64 = nullptr, *F64 = nullptr, *LT64 = nullptr;
  CKS(fp64_buffers(ctx, &A64, &F64, &LT64));
  CKS(predict_buffers(ctx, np));
  CovParams cp = cov_params(theta);
  CK(cudaMemsetAsync(ctx->status, 0, 4 * sizeof(int), ctx->stream));
  CKS(upload(ctx, ctx->y, y, (size_t)n * sizeof(double)));
  CKS(apply_scaling(ctx, theta, false));
  CKS(run_pipeline<double>(ctx, cp, A64, LT64, F64, ctx->Xs, ctx->Zs));
  CKS(upload(ctx, ctx->pXp, Xp, (size_t)np * d * sizeof(double)));
  CK(scale_coords(ctx->pXp, np, d, ctx->hyp, ctx->hyp + 16, ctx->pXps, nullptr, ctx->stream));
  CK(lowrank_A<double>(ctx->pXps, ctx->Zs, LT64, mpad, ctx->pAp, np, d, m, mpad, cp.kind, cp.var, ctx->stream));
  CK(predict_all(A64, ctx->Xs, n, ctx->pAp, ctx->pXps, np, d, m, mpad, mv, cp, ctx->y, ctx->G, fpad, ctx->pLinvC,
                 ctx->pw, ctx->pr, ctx->pcjj, ctx->pcpp, ctx->pNp, latent ? 1 : 0, theta->nugget, ctx->pmean,
                 ctx->pvar, ctx->status, ctx->trw, ctx->stream));
  double sc[1];
  CKS(read_status(ctx, sc, 1));
  ctx->have_factors = true;
  CKS(download(ctx, mean, ctx->pmean, (size_t)np * sizeof(double)));
  if (var) CKS(download(ctx, var, ctx->pvar, (size_t)np * sizeof(double)));
  return VIF_OK;
}

}  // extern "C"

namespace {

// Factors of the latent-GP VIF prior for theta (A, B, D, F, C = I + F^T F and the
// inverse of its Cholesky factor) and the operator bundle of the Laplace kernels
// (y: host or device responses, or NULL to keep those already on the device).
vif_status lap_setup(vif_ctx* ctx, const vif_cov* theta, const double* y, LapOps* o) {
  cudaStream_t s = ctx->stream;
  double *A64 = nullptr, *F64 = nullptr, *LT64 = nullptr;
  CKS(fp64_buffers(ctx, &A64, &F64, &LT64));
  CKS(lap_alloc(ctx));
  CovParams cp = cov_params(theta);
  CK(cudaMemsetAsync(ctx->status, 0, 4 * sizeof(int), s));
  CK(cudaMemsetAsync(ctx->l_abort, 0, 2 * sizeof(int), s));
  if (y) CKS(upload(ctx, ctx->y, y, (size_t)ctx->n * sizeof(double)));   // NULL: y already resident
  CKS(apply_scaling(ctx, theta, false));
  CKS(run_pipeline<double>(ctx, cp, A64, LT64, F64, ctx->Xs, ctx->Zs));
  if (ctx->m > 0) CK(dense_trtri_lower(ctx->G, ctx->l_LinvC, ctx->m, ctx->fpad, ctx->trw, s));
  double dummy[1];
  CKS(read_status(ctx, dummy, 0));
  o->n = ctx->n;
  o->m = ctx->m;
  o->mv = ctx->mv;
  o->fpad = ctx->fpad;
  o->ldl = ctx->fpad;
  o->N = ctx->N;
  o->ch_ptr = ctx->ch_ptr;
  o->ch_row = ctx->ch_row;
  o->ch_slot = ctx->ch_slot;
  o->Acoef = ctx->Acoef;
  o->F = F64;
  o->LinvC = ctx->l_LinvC;
  o->LinvC3 = ctx->l_LinvC3;
  o->rsD = ctx->l_rsD;
  o->Ginv = ctx->l_Ginv;
  o->t = ctx->l_t;
  o->t2 = ctx->l_t2;
  o->x1 = ctx->l_x1;
  o->sm = ctx->l_sm;
  o->cm = ctx->l_cm;
  o->tmpm = ctx->l_tm;
  o->partial = ctx->l_part;
  o->sched_fwd = ctx->sched_fwd;
  o->sched_rev = ctx->sched_rev;
  o->nsteps_fwd = ctx->nsteps_fwd;
  o->nsteps_rev = ctx->nsteps_rev;
  o->ord_fwd = ctx->ord_fwd;
  o->ord_rev = ctx->ord_rev;
  o->ch_coef = ctx->ch_coef;
  o->nnz = ctx->ch_nnz;
  o->counter = ctx->l_counter;
  o->abort_flag = ctx->l_abort;
  o->status = ctx->status;
  o->kind = LAP_VIFDU;
  o->A = A64;
  o->Apad = ctx->l_Apad;
  o->D = ctx->Dv;
  o->W = ctx->l_W;
  o->mpad = ctx->mpad;
  o->dvinv = ctx->l_dvinv;
  o->anorm2 = ctx->l_anorm2;
  o->LinvMV = ctx->l_LinvC3;
  CK(lap_child_coef(*o, ctx->ch_coef, s));   // the children's coefficients of the new A
  return VIF_OK;
}

// C_3 = I + F^T diag(omega) F, its Cholesky factor and the inverse factor.
vif_status lap_c3(vif_ctx* ctx, const LapOps& o) {
  if (ctx->m == 0) return VIF_OK;
  cudaStream_t s = ctx->stream;
  CK(gram_FtF<double>(o.F, ctx->n, ctx->fpad, ctx->m, ctx->part, ctx->nsplit, ctx->l_G3, ctx->fpad, s, ctx->l_om));
  CK(dense_cholesky(ctx->l_G3, ctx->m, ctx->fpad, ctx->status, ST_NOTPD_PRECOND, s));
  CK(dense_trtri_lower(ctx->l_G3, ctx->l_LinvC3, ctx->m, ctx->fpad, ctx->trw, s));
  return VIF_OK;
}

// FITC preconditioner at the current W (App. E.2): D_V^{-1}, M_V = I + A D_V^{-1} A^T (whitened, in
// l_G3), its Cholesky factor and inverse factor (in l_LinvC3).  A's padded copy and row norms
// are formed on the first call after lap_setup (fresh = true).
vif_status lap_fitc_setup(vif_ctx* ctx, LapOps& o, bool fresh, double var) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  if (!ctx->l_dvinv) {
    CKS(dalloc(ctx, &ctx->l_dvinv, (size_t)n));
    CKS(dalloc(ctx, &ctx->l_anorm2, (size_t)n));
    if (ctx->m > 0) CKS(dalloc(ctx, &ctx->l_Apad, (size_t)n * ctx->fpad));
    fresh = true;
  }
  o.dvinv = ctx->l_dvinv;
  o.anorm2 = ctx->l_anorm2;
  o.Apad = ctx->l_Apad;
  if (fresh) {
    if (ctx->m > 0) {
      CK(lap_fitc_prepare_A(o.A, ctx->mpad, ctx->m, n, ctx->fpad, ctx->l_Apad, ctx->l_anorm2, s));
    } else {
      CK(cudaMemsetAsync(ctx->l_anorm2, 0, (size_t)n * sizeof(double), s));
    }
  }
  CK(lap_fitc_dv(n, var, ctx->l_anorm2, ctx->l_W, ctx->l_dvinv, s));
  if (ctx->m == 0) return VIF_OK;
  CK(gram_FtF<double>(ctx->l_Apad, n, ctx->fpad, ctx->m, ctx->part, ctx->nsplit, ctx->l_G3, ctx->fpad, s,
                      ctx->l_dvinv));
  CK(dense_cholesky(ctx->l_G3, ctx->m, ctx->fpad, ctx->status, ST_NOTPD_PRECOND, s));
  CK(dense_trtri_lower(ctx->l_G3, ctx->l_LinvC3, ctx->m, ctx->fpad, ctx->trw, s));
  return VIF_OK;
}

// Preconditioned CG from x = 0 on (W + Sigma_dagger^{-1}) x = v (v in l_v, x in l_x).
// Optionally records the CG step lengths alpha_j, the direction updates beta_j and the
// starting value r_0^T P^{-1} r_0 (the Lanczos coefficients of App. D), and copies
// P^{-1} v to z0_out (device, n).
vif_status lap_pcg(vif_ctx* ctx, const LapOps& o, double tol, int max_it, int* iters, double* rel, bool* capped,
                   std::vector<double>* alphas = nullptr, std::vector<double>* betas = nullptr,
                   double* rz0 = nullptr, double* z0_out = nullptr) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  double* sc = ctx->l_sc;   // [0]=rz [1]=pAp [2]=alpha [3]=rr [4]=rz_new [5]=beta [6]=vv
  double* hs = ctx->h_pin + 16;
  CK(cudaMemsetAsync(ctx->l_x, 0, n * sizeof(double), s));
  CK(cudaMemcpyAsync(ctx->l_r, ctx->l_v, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(lap_dot(ctx->l_v, ctx->l_v, n, ctx->l_red, sc + 6, s));
  CK(lap_system_precond(o, ctx->l_r, ctx->l_z, s));
  CK(cudaMemcpyAsync(ctx->l_p, ctx->l_z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (z0_out) CK(cudaMemcpyAsync(z0_out, ctx->l_z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(lap_dot(ctx->l_r, ctx->l_z, n, ctx->l_red, sc + 0, s));
  CK(cudaMemcpyAsync(hs, sc, 7 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double vnorm = std::sqrt(hs[6]);
  if (rz0) *rz0 = hs[0];
  int it = 0;
  *rel = 0.0;
  *capped = false;
  if (vnorm > 0.0) {
    for (it = 1; it <= max_it; ++it) {
      CK(lap_system_matvec(o, ctx->l_p, ctx->l_Ap, s));
      CK(lap_dot(ctx->l_p, ctx->l_Ap, n, ctx->l_red, sc + 1, s));
      CK(lap_alpha(sc, s));
      CK(lap_axpy(n, sc + 2, ctx->l_x, ctx->l_p, ctx->l_x, 0, s));
      CK(lap_axpy(n, sc + 2, ctx->l_r, ctx->l_Ap, ctx->l_r, 1, s));
      CK(lap_dot(ctx->l_r, ctx->l_r, n, ctx->l_red, sc + 3, s));
      CK(cudaMemcpyAsync(hs, sc, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(ctx->h_pin + 9, ctx->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      // hs[2] = alpha of this step; hs[5] = beta of the previous one (set at its end)
      if (alphas) alphas->push_back(hs[2]);
      if (betas && it >= 2) betas->push_back(hs[5]);
      *rel = std::sqrt(hs[3]) / vnorm;
      if (reinterpret_cast<const int*>(ctx->h_pin + 9)[0] != ST_OK) break;
      if (*rel <= tol) break;
      CK(lap_system_precond(o, ctx->l_r, ctx->l_z, s));
      CK(lap_dot(ctx->l_r, ctx->l_z, n, ctx->l_red, sc + 4, s));
      CK(lap_beta(sc, s));
      CK(lap_axpy(n, sc + 5, ctx->l_z, nullptr, ctx->l_p, 2, s));
    }
    if (it > max_it) {
      it = max_it;
      *capped = true;
    }
  }
  double dummy[1];
  CKS(read_status(ctx, dummy, 0));
  *iters = it;
  return VIF_OK;
}

// Block-CG buffers for L <= LAP_MR_MAXL columns (grown on demand) and their bundle.
vif_status mr_buffers(vif_ctx* ctx, int L, LapMulti* w) {
  const int64_t n = ctx->n;
  const size_t fp = (size_t)std::max(ctx->fpad, 1);
  if (L > ctx->mr_cap) {
    double** vecs[] = {&ctx->mr_v, &ctx->mr_x, &ctx->mr_r, &ctx->mr_z, &ctx->mr_p, &ctx->mr_Ap, &ctx->mr_t,
                       &ctx->mr_t2, &ctx->mr_x1};
    double** small[] = {&ctx->mr_sm, &ctx->mr_cm, &ctx->mr_tm, &ctx->mr_part, &ctx->mr_dpart};
    for (double** b : vecs) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    for (double** b : small) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    ctx->mr_cap = 0;
    for (double** b : vecs) CKS(dalloc(ctx, b, (size_t)n * L));
    CKS(dalloc(ctx, &ctx->mr_sm, fp * L));
    CKS(dalloc(ctx, &ctx->mr_cm, fp * L));
    CKS(dalloc(ctx, &ctx->mr_tm, fp * L));
    CKS(dalloc(ctx, &ctx->mr_part, (size_t)LAP_MR_FT_BLOCKS * fp * L));
    CKS(dalloc(ctx, &ctx->mr_dpart, (size_t)LAP_MR_DOT_BLOCKS * L));
    if (!ctx->mr_sc) {
      CKS(dalloc(ctx, &ctx->mr_sc, 7 * (size_t)LAP_MR_MAXL));
      CKS(dalloc(ctx, &ctx->mr_active, (size_t)LAP_MR_MAXL));
      CKS(dalloc(ctx, &ctx->mr_map, (size_t)LAP_MR_MAXL));
    }
    ctx->mr_cap = L;
  }
  w->L = L;
  w->t = ctx->mr_t;
  w->t2 = ctx->mr_t2;
  w->x1 = ctx->mr_x1;
  w->sm = ctx->mr_sm;
  w->cm = ctx->mr_cm;
  w->tmpm = ctx->mr_tm;
  w->partial = ctx->mr_part;
  w->dpart = ctx->mr_dpart;
  return VIF_OK;
}

// Preconditioned CG from X = 0 on the system of o.kind (Eq. pcls1 with VIFDU, Eq. pcls2 with FITC)
// with right-hand sides V, for the L columns of mr_v at once: each column takes the steps of
// lap_pcg with its own step lengths and stopping test.  A column that meets its test leaves the
// block: its solution is parked in mr_v (whose right-hand sides are no longer needed) and the
// others are packed into the first columns, so later products only cover unfinished columns.
// On return mr_x holds every column's solution (n x L).  Per column: iterations, final relative
// residual, whether the cap was hit, the Lanczos coefficients alpha_j, beta_j and v^T P^{-1} v
// (App. D); with z0_cols (device, L x n probe-major) also P^{-1} v.
vif_status lap_pcg_multi(vif_ctx* ctx, const LapOps& o, const LapMulti& w, double tol, int max_it,
                         std::vector<int>& iters, std::vector<double>& rel, std::vector<char>& capped,
                         std::vector<std::vector<double>>& alphas, std::vector<std::vector<double>>& betas,
                         std::vector<double>& rz0, double* z0_cols) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  const int L = w.L;
  const size_t bytes = (size_t)n * L * sizeof(double);
  double* sc = ctx->mr_sc;   // per current column, stride Lc: rz, pAp, alpha, rr, rz_new, beta (, v^T v)
  double* hs = ctx->h_pin + 64;   // 7 L <= 448 doubles of pinned staging
  CK(cudaMemsetAsync(ctx->mr_x, 0, bytes, s));
  CK(cudaMemsetAsync(sc, 0, 7 * (size_t)L * sizeof(double), s));
  CK(cudaMemcpyAsync(ctx->mr_r, ctx->mr_v, bytes, cudaMemcpyDeviceToDevice, s));
  CK(lap_mr_dot(w, n, ctx->mr_v, ctx->mr_v, sc + 6 * L, s));
  CK(lap_mr_system_precond(o, w, ctx->mr_r, ctx->mr_z, s));
  CK(cudaMemcpyAsync(ctx->mr_p, ctx->mr_z, bytes, cudaMemcpyDeviceToDevice, s));
  if (z0_cols)
    for (int j = 0; j < L; ++j) CK(lap_mr_column(n, L, j, ctx->mr_z, z0_cols + (size_t)j * n, true, s));
  CK(lap_mr_dot(w, n, ctx->mr_r, ctx->mr_z, sc, s));
  CK(cudaMemcpyAsync(hs, sc, 7 * (size_t)L * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> vnorm(L);
  std::vector<int> col(L);            // current slot -> column
  std::vector<char> keep(L);
  for (int j = 0; j < L; ++j) {
    vnorm[j] = std::sqrt(hs[6 * L + j]);
    rz0[j] = hs[j];
    keep[j] = vnorm[j] > 0.0 ? 1 : 0;
    col[j] = j;
    iters[j] = 0;
    rel[j] = 0.0;
    capped[j] = 0;
    alphas[j].clear();
    betas[j].clear();
  }
  int Lc = L;
  // park the solutions of the slots with keep = 0 in mr_v, pack the others (x, r, p and rz of sc)
  auto repack = [&]() -> vif_status {
    std::vector<int> map, ncol;
    std::vector<double> nrz;
    for (int jj = 0; jj < Lc; ++jj) {
      if (keep[jj]) {
        map.push_back(jj);
        ncol.push_back(col[jj]);
        nrz.push_back(hs[jj]);
      } else {
        CK(lap_mr_copy_col(n, ctx->mr_x, Lc, jj, ctx->mr_v, L, col[jj], s));
      }
    }
    const int Lk = (int)map.size();
    if (Lk > 0 && Lk < Lc) {
      const size_t kb = (size_t)n * Lk * sizeof(double);
      CK(cudaMemcpyAsync(ctx->mr_map, map.data(), Lk * sizeof(int), cudaMemcpyHostToDevice, s));
      CK(lap_mr_gather(n, Lc, Lk, ctx->mr_map, ctx->mr_x, ctx->mr_t, s));
      CK(lap_mr_gather(n, Lc, Lk, ctx->mr_map, ctx->mr_r, ctx->mr_t2, s));
      CK(lap_mr_gather(n, Lc, Lk, ctx->mr_map, ctx->mr_p, ctx->mr_x1, s));
      CK(cudaMemcpyAsync(ctx->mr_x, ctx->mr_t, kb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ctx->mr_r, ctx->mr_t2, kb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ctx->mr_p, ctx->mr_x1, kb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(sc, nrz.data(), Lk * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));   // the host vectors above go out of scope
    }
    col = ncol;
    Lc = Lk;
    keep.assign(Lc, 1);
    return VIF_OK;
  };
  CKS(repack());
  {
    const std::vector<int> ones(LAP_MR_MAXL, 1);
    CK(cudaMemcpyAsync(ctx->mr_active, ones.data(), LAP_MR_MAXL * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  for (int it = 1; Lc > 0 && it <= max_it; ++it) {
    LapMulti wc = w;
    wc.L = Lc;
    double *rz = sc, *pAp = sc + Lc, *alpha = sc + 2 * Lc, *rr = sc + 3 * Lc;
    CK(lap_mr_system_matvec(o, wc, ctx->mr_p, ctx->mr_Ap, s));
    CK(lap_mr_dot(wc, n, ctx->mr_p, ctx->mr_Ap, pAp, s));
    CK(lap_mr_alpha(wc, ctx->mr_active, rz, pAp, alpha, s));
    CK(lap_mr_update_xr(wc, n, alpha, ctx->mr_p, ctx->mr_Ap, ctx->mr_x, ctx->mr_r, s));
    CK(lap_mr_dot(wc, n, ctx->mr_r, ctx->mr_r, rr, s));
    CK(cudaMemcpyAsync(hs, sc, 6 * (size_t)Lc * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_pin + 9, ctx->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // alpha of this step; beta of the previous one (set at its end)
    bool any_done = false;
    for (int jj = 0; jj < Lc; ++jj) {
      const int j = col[jj];
      alphas[j].push_back(hs[2 * Lc + jj]);
      if (it >= 2) betas[j].push_back(hs[5 * Lc + jj]);
      rel[j] = std::sqrt(hs[3 * Lc + jj]) / vnorm[j];
      iters[j] = it;
      if (rel[j] <= tol) {
        keep[jj] = 0;
        any_done = true;
      } else if (it == max_it) {
        capped[j] = 1;
      }
    }
    if (reinterpret_cast<const int*>(ctx->h_pin + 9)[0] != ST_OK) break;
    if (any_done) CKS(repack());
    if (Lc == 0 || it == max_it) break;
    wc.L = Lc;
    double *rzn = sc + 4 * Lc, *beta = sc + 5 * Lc;
    CK(lap_mr_system_precond(o, wc, ctx->mr_r, ctx->mr_z, s));
    CK(lap_mr_dot(wc, n, ctx->mr_r, ctx->mr_z, rzn, s));
    CK(lap_mr_beta(wc, ctx->mr_active, sc, rzn, beta, s));
    CK(lap_mr_update_p(wc, n, beta, ctx->mr_z, ctx->mr_p, s));
  }
  // every column's solution into mr_x (n x L)
  for (int jj = 0; jj < Lc; ++jj) CK(lap_mr_copy_col(n, ctx->mr_x, Lc, jj, ctx->mr_v, L, col[jj], s));
  CK(cudaMemcpyAsync(ctx->mr_x, ctx->mr_v, bytes, cudaMemcpyDeviceToDevice, s));
  double dummy[1];
  CKS(read_status(ctx, dummy, 0));
  return VIF_OK;
}

// e_1^T log(T) e_1 for the symmetric tridiagonal T with diagonal d[0..k-1] and
// off-diagonal e[0..k-2]: the Gauss quadrature of log whose nodes are the eigenvalues
// of T and whose weights are the squared first components of its eigenvectors (App. D).
// The eigenvalues come from implicit symmetric QR steps with a Wilkinson shift (Golub &
// Van Loan, Sec. 8.3): each step chases a bulge down the unreduced block with Givens
// rotations T <- G T G^T; only the first row of the accumulated rotations is kept.
// Returns false if T is not positive definite or a block fails to converge.
bool tridiag_log_quadrature(std::vector<double> d, std::vector<double> e, double* out) {
  const int k = (int)d.size();
  *out = 0.0;
  if (k == 0) return true;
  e.resize(k, 0.0);
  std::vector<double> z(k, 0.0);   // first row of the accumulated rotations
  z[0] = 1.0;
  const double eps = 4.0 * 2.220446049250313e-16;
  int hi = k - 1, guard = 0;
  while (hi > 0) {
    for (int i = 0; i < hi; ++i)
      if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    if (e[hi - 1] == 0.0) {
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    if (++guard > 60 * k) return false;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to d[hi]
    const double dd = 0.5 * (d[hi - 1] - d[hi]), bb = e[hi - 1];
    const double mu = d[hi] - bb * bb / (dd + std::copysign(std::hypot(dd, bb), dd == 0.0 ? 1.0 : dd));
    double x = d[lo] - mu, y = e[lo];
    for (int j = lo; j < hi; ++j) {
      // rotation G = [[c, s], [-s, c]] on coordinates (j, j+1) with G [x; y] = [r; 0]
      const double r = std::hypot(x, y);
      const double c = r == 0.0 ? 1.0 : x / r, sn = r == 0.0 ? 0.0 : y / r;
      if (j > lo) e[j - 1] = r;   // the bulge below e[j-1] is annihilated
      const double p = d[j], q = d[j + 1], b = e[j];
      d[j] = c * c * p + 2.0 * c * sn * b + sn * sn * q;
      d[j + 1] = sn * sn * p - 2.0 * c * sn * b + c * c * q;
      e[j] = c * sn * (q - p) + (c * c - sn * sn) * b;
      if (j + 1 < hi) {   // the rotation of columns (j, j+1) pushes e[j+1] into a bulge at (j+2, j)
        y = sn * e[j + 1];
        e[j + 1] = c * e[j + 1];
        x = e[j];
      }
      const double zj = z[j], zj1 = z[j + 1];
      z[j] = c * zj + sn * zj1;
      z[j + 1] = -sn * zj + c * zj1;
    }
  }
  double q = 0.0;
  for (int j = 0; j < k; ++j) {
    if (!(d[j] > 0.0)) return false;
    q += z[j] * z[j] * std::log(d[j]);
  }
  *out = q;
  return true;
}

// mlp scratch: features (n x 10 float), gc (n float), backward partials, gradient
vif_status mlp_scratch(vif_ctx* ctx) {
  if (ctx->m_feat) return VIF_OK;
  CKS(dalloc(ctx, &ctx->m_feat, (size_t)ctx->n * VIF_MLP_NIN));
  CKS(dalloc(ctx, &ctx->m_gc, (size_t)ctx->n));
  CKS(dalloc(ctx, &ctx->m_part, (size_t)mlp_backward_blocks(ctx->n) * ((VIF_MLP_NPARAM + 63) / 64 * 64)));
  CKS(dalloc(ctx, &ctx->m_grad, (size_t)VIF_MLP_NPARAM + 64));
  return VIF_OK;
}

// c = network(features(W)) into l_corr.
vif_status mlp_correction_c(vif_ctx* ctx, const void* net) {
  CKS(mlp_scratch(ctx));
  CK(mlp_features(ctx->l_W, ctx->Dv, ctx->Acoef, ctx->m_rho, ctx->N, ctx->ch_ptr, ctx->ch_row, ctx->ch_slot,
                  ctx->n, ctx->mv, ctx->m_feat, ctx->stream));
  CK(mlp_forward_f64(net, ctx->m_feat, ctx->n, ctx->l_corr, ctx->stream));
  return VIF_OK;
}

// Newton search of the Laplace mode (Eq. one_it_newton_mode), shared by vif_laplace_mode
// and vif_laplace_nll.  Leaves the mode in l_b and W, G^{-1}, omega, 1/sqrt(D) and the
// log-likelihood terms at the mode in the Laplace buffers.
vif_status laplace_run(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_laplace_opts* lo, LapOps* op,
                       vif_laplace_stats* stats, bool* converged_out, bool* capped_out) {
  if (!y || !lo) return set_err(ctx, VIF_ERR_ARG, "y and opts are required");
  CKS(check_cov(ctx, theta, ctx->d));
  if (ctx->likelihood != VIF_BERNOULLI_LOGIT)
    return set_err(ctx, VIF_ERR_STATE, "the Laplace approximation needs a context built for VIF_BERNOULLI_LOGIT");
  if (theta->nugget != 0.0) return set_err(ctx, VIF_ERR_ARG, "a latent GP has no nugget: set nugget = 0");
  if (!(lo->rel_tol > 0.0) || lo->max_pcg < 1 || lo->max_newton < 1 || lo->wait_polls < 0)
    return set_err(ctx, VIF_ERR_ARG, "invalid Laplace options");
  if (lo->precond != 0 && lo->precond != 1 && lo->precond != LAP_FITC)
    return set_err(ctx, VIF_ERR_ARG, "unknown preconditioner");
  if (lo->precond == 1 && !lo->mlp_weights)
    return set_err(ctx, VIF_ERR_ARG, "the learned correction needs mlp_weights");
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } guard{e0, e1};
  CK(cudaEventRecord(e0, s));
  LapOps& o = *op;
  CKS(lap_setup(ctx, theta, y, &o));
  if (lo->wait_polls > 0) CK(lap_set_wait_polls(ctx->l_abort, lo->wait_polls, s));
  const bool fitc = lo->precond == LAP_FITC;
  if (fitc) o.kind = LAP_FITC;
  bool fresh = true;   // FITC: A's padded copy is due after lap_setup
  const bool learned = lo->precond == 1;
  const double* corr = learned ? ctx->l_corr : nullptr;
  CK(cudaMemsetAsync(ctx->l_b, 0, n * sizeof(double), s));
  CK(cudaMemsetAsync(ctx->l_corr, 0, n * sizeof(double), s));
  CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, corr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                   ctx->l_ll, s));
  int newton = 0, pcg_total = 0;
  double rel = 0.0, psi_old = 0.0, psi = 0.0, ms_pcg = 0.0;
  bool have_old = false, converged = false, pcg_capped = false;
  cudaEvent_t p0, p1;
  CK(cudaEventCreate(&p0));
  CK(cudaEventCreate(&p1));
  EvGuard guard2{p0, p1};
  double* sc = ctx->l_sc;
  for (newton = 1; newton <= lo->max_newton; ++newton) {
    if (learned) {
      CKS(mlp_correction_c(ctx, lo->mlp_weights));
      CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, corr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om,
                       ctx->l_rsD, ctx->l_ll, s));
    }
    if (fitc) {
      // Eq. pcls2: (W^{-1} + Sigma_dagger)(W b) = Sigma_dagger v
      CKS(lap_fitc_setup(ctx, o, fresh, theta->variance));
      fresh = false;
      CK(lap_sigma_matvec(o, ctx->l_v, nullptr, ctx->l_sdi, s));
      CK(cudaMemcpyAsync(ctx->l_v, ctx->l_sdi, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      CKS(lap_c3(ctx, o));
    }
    CK(cudaEventRecord(p0, s));
    int it = 0;
    bool capped = false;
    CKS(lap_pcg(ctx, o, lo->rel_tol, lo->max_pcg, &it, &rel, &capped));
    CK(cudaEventRecord(p1, s));
    CK(cudaEventSynchronize(p1));
    float tms = 0.f;
    CK(cudaEventElapsedTime(&tms, p0, p1));
    ms_pcg += tms;
    pcg_total += it;
    pcg_capped = pcg_capped || capped;
    if (fitc) {
      CK(lap_div(n, ctx->l_x, ctx->l_W, ctx->l_b, s));   // b = (W b) / W
    } else {
      CK(cudaMemcpyAsync(ctx->l_b, ctx->l_x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // objective at the new b: sum log p(y|b) - b^T Sigma_dagger^{-1} b / 2
    CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, corr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                     ctx->l_ll, s));
    CK(lap_matvec(o, ctx->l_b, nullptr, ctx->l_sdi, s));
    CK(lap_dot(ctx->l_ll, nullptr, n, ctx->l_red, sc + 7, s));
    CK(lap_dot(ctx->l_b, ctx->l_sdi, n, ctx->l_red, sc + 8, s));
    CK(cudaMemcpyAsync(ctx->h_pin + 8, sc + 7, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    psi = ctx->h_pin[8] - 0.5 * ctx->h_pin[9];
    if (have_old && std::fabs(psi - psi_old) <= 1e-10 * std::fabs(psi)) {
      converged = true;
      break;
    }
    psi_old = psi;
    have_old = true;
  }
  if (newton > lo->max_newton) newton = lo->max_newton;
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float tot = 0.f;
  CK(cudaEventElapsedTime(&tot, e0, e1));
  stats->newton_iters = newton;
  stats->pcg_iters_total = pcg_total;
  stats->final_rel_res = rel;
  stats->ms_pcg = ms_pcg;
  stats->ms_total = tot;
  stats->objective = psi;
  *converged_out = converged;
  *capped_out = pcg_capped;
  return VIF_OK;
}

}  // namespace

extern "C" {

vif_status vif_laplace_mode(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_laplace_opts* lo,
                            double* mode_out, vif_laplace_stats* stats) {
  if (!ctx) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  if (!mode_out) return set_err(ctx, VIF_ERR_ARG, "mode_out is required");
  LapOps o;
  vif_laplace_stats st{};
  bool converged = false, capped = false;
  CKS(laplace_run(ctx, theta, y, lo, &o, &st, &converged, &capped));
  CKS(download(ctx, mode_out, ctx->l_b, (size_t)ctx->n * sizeof(double)));
  if (stats) *stats = st;
  if (!converged || capped)
    return set_err(ctx, VIF_ERR_NOT_CONVERGED, "Newton %s, CG %s", converged ? "converged" : "hit its cap",
                   capped ? "hit its cap" : "converged");
  return VIF_OK;
}

}  // extern "C"

namespace {

// The body of vif_laplace_nll.  With keepU / keepY (device, nprobe x n, probe-major) it also
// keeps each probe's CG solution u_i = (W + Sigma_dagger^{-1})^{-1} z_i and y_i = P^{-1} z_i, the
// vectors the stochastic trace estimates of the gradient reuse (Sec. 4.1).  *newton_ok and
// *cg_ok report whether Newton converged and no CG solve hit its cap (outputs written either way).
vif_status laplace_nll_core(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_laplace_opts* lo,
                            int32_t nprobe, const double* eps, double slq_tol, int32_t slq_max_iter,
                            double* nll_out, double* probe_q, double* probe_zpz, vif_laplace_nll_stats* stats,
                            LapOps* op, double* keepU, double* keepY, bool* newton_ok, bool* cg_ok) {
  if (!nll_out || !eps || nprobe < 1 || !(slq_tol > 0.0) || slq_max_iter < 1)
    return set_err(ctx, VIF_ERR_ARG, "nll_out, eps, nprobe >= 1, slq_tol > 0 and slq_max_iter >= 1 are required");
  LapOps& o = *op;
  vif_laplace_stats ms{};
  bool converged = false, capped = false;
  CKS(laplace_run(ctx, theta, y, lo, &o, &ms, &converged, &capped));
  const int64_t n = ctx->n;
  const int m = ctx->m;
  cudaStream_t s = ctx->stream;
  const bool learned = lo->precond == 1;
  const bool fitc = lo->precond == LAP_FITC;
  // the preconditioner at the mode's W: C_3 of VIFDU (App. E.1) or M_V of FITC (App. E.2)
  if (fitc) {
    CKS(lap_fitc_setup(ctx, o, false, theta->variance));
  } else {
    CKS(lap_c3(ctx, o));
  }
  // log-determinant pieces and the two other terms of Eq. log_det_VIFLA
  double* sc = ctx->l_sc;
  CK(reduce_sum(ctx->logD, n, ctx->red, sc + 9, s));                        // sum log D_i
  if (fitc) {
    CK(lap_log_sum(ctx->l_dvinv, n, 1, -1.0, ctx->l_red, sc + 10, s));      // log det D_V
  } else {
    CK(lap_log_sum(ctx->l_Ginv, n, 1, -1.0, ctx->l_red, sc + 10, s));       // sum log(W'_i + 1/D_i)
  }
  if (m > 0) {
    CK(lap_log_sum(ctx->G, m, (int64_t)ctx->fpad + 1, 2.0, ctx->l_red, sc + 11, s));      // log det C
    CK(lap_log_sum(ctx->l_G3, m, (int64_t)ctx->fpad + 1, 2.0, ctx->l_red, sc + 12, s));   // log det C_3 / M_V
  } else {
    CK(cudaMemsetAsync(sc + 11, 0, 2 * sizeof(double), s));
  }
  CK(lap_log_sum(ctx->l_W, n, 1, 1.0, ctx->l_red, sc + 15, s));             // log det W
  CK(lap_dot(ctx->l_ll, nullptr, n, ctx->l_red, sc + 13, s));              // log p(y | b~)
  CK(lap_matvec(o, ctx->l_b, nullptr, ctx->l_sdi, s));
  CK(lap_dot(ctx->l_b, ctx->l_sdi, n, ctx->l_red, sc + 14, s));            // b~^T Sigma_dagger^{-1} b~
  double h[7];
  CK(cudaMemcpyAsync(ctx->h_pin + 32, sc + 9, 7 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  memcpy(h, ctx->h_pin + 32, sizeof(h));
  // probes
  double *A64 = nullptr, *F64 = nullptr, *LT64 = nullptr;
  CKS(fp64_buffers(ctx, &A64, &F64, &LT64));
  if (!ctx->slq_eps) CKS(dalloc(ctx, &ctx->slq_eps, (size_t)m + 2 * (size_t)n));
  const size_t per = (size_t)m + 2 * (size_t)n;
  const auto t0 = std::chrono::steady_clock::now();
  double qsum = 0.0, wsum = 0.0;
  int slq_iters = 0;
  bool slq_capped = false;
  // probe i into l_v:
  //   VIFDU: z = B^T W'^{1/2} eps3 + Sigma_dagger^{-1} (B^{-1} D^{1/2} eps2 + A^T eps1)   (Sec. 4.3)
  //   FITC:  z = D_V^{1/2} eps2 + Sigma_mn^T L_m^{-T} eps1   (App. E.2)
  auto draw = [&](int i) -> vif_status {
    CKS(upload(ctx, ctx->slq_eps, eps + (size_t)i * per, per * sizeof(double)));
    const double* e1 = ctx->slq_eps;
    const double* e2 = ctx->slq_eps + m;
    const double* e3 = ctx->slq_eps + m + n;
    if (fitc) {
      CK(lap_fitc_probe(o, e1, e2, ctx->l_v, s));
      return VIF_OK;
    }
    CK(lap_probe_prep(n, ctx->Dv, ctx->l_W, learned ? ctx->l_corr : nullptr, e2, e3, ctx->l_r, ctx->l_z, s));
    CK(lap_solve_B(o, ctx->l_r, ctx->l_p, s));
    if (m > 0) {
      CK(lap_rows_dot_add(A64, ctx->mpad, m, n, e1, ctx->l_p, ctx->l_Ap, s));
    } else {
      CK(cudaMemcpyAsync(ctx->l_Ap, ctx->l_p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(lap_matvec(o, ctx->l_Ap, nullptr, ctx->l_x, s));
    CK(lap_apply_Bt(o, ctx->l_z, ctx->l_r, s));
    CK(lap_vec_add(n, ctx->l_x, ctx->l_r, ctx->l_v, s));
    return VIF_OK;
  };
  // T_i from the CG coefficients of probe i (App. D) and its Gauss quadrature
  auto quadrature = [&](int i, const std::vector<double>& al, const std::vector<double>& be, double zpz) -> vif_status {
    std::vector<double> d(al.size()), od(al.size() > 0 ? al.size() - 1 : 0);
    for (size_t j = 0; j < al.size(); ++j) {
      d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
      if (j > 0) od[j - 1] = std::sqrt(be[j - 1]) / al[j - 1];
    }
    double q = 0.0;
    if (!tridiag_log_quadrature(d, od, &q))
      return set_err(ctx, VIF_ERR_NOT_PD, "Lanczos matrix of probe %d is not positive definite", i);
    if (probe_q) probe_q[i] = q;
    if (probe_zpz) probe_zpz[i] = zpz;
    qsum += q;
    wsum += zpz * q;
    return VIF_OK;
  };
  // the probes' CGs (Eq. pcls1 with VIFDU, Eq. pcls2 with FITC) run side by side in blocks of up to
  // LAP_MR_MAXL columns, sharing every operator application
  for (int b0 = 0; b0 < nprobe; b0 += LAP_MR_MAXL) {
    const int L = std::min(LAP_MR_MAXL, nprobe - b0);
    LapMulti w;
    CKS(mr_buffers(ctx, L, &w));
    for (int j = 0; j < L; ++j) {
      CKS(draw(b0 + j));
      CK(lap_mr_column(n, L, j, ctx->mr_v, ctx->l_v, false, s));
    }
    std::vector<int> its(L);
    std::vector<double> rels(L), rz0(L);
    std::vector<char> caps(L);
    std::vector<std::vector<double>> al(L), be(L);
    CKS(lap_pcg_multi(ctx, o, w, slq_tol, slq_max_iter, its, rels, caps, al, be, rz0,
                      keepY ? keepY + (size_t)b0 * n : nullptr));
    if (keepU)
      for (int j = 0; j < L; ++j) CK(lap_mr_column(n, L, j, ctx->mr_x, keepU + (size_t)(b0 + j) * n, true, s));
    for (int j = 0; j < L; ++j) {
      slq_iters += its[j];
      slq_capped = slq_capped || caps[j];
      CKS(quadrature(b0 + j, al[j], be[j], rz0[j]));
    }
  }
  const double ms_slq =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  const double logdet_sigma = h[2] + h[0];
  // VIFDU: log det P = sum log(W' + 1/D) - log det C + log det C_3 (App. E.1), Eq. slq_v1;
  // FITC: log det P = log det D_V + log det M_V (whitened, App. E.2), Eq. slq_v2 with log det W
  const double logdet_P = fitc ? h[1] + h[3] : h[1] - h[2] + h[3];
  const double base = fitc ? h[6] : logdet_sigma;
  const double slq = (double)n / nprobe * qsum;
  const double logdet = base + slq + logdet_P;
  const double nll = -h[4] + 0.5 * h[5] + 0.5 * logdet;
  *nll_out = nll;
  if (stats) {
    stats->nll = nll;
    stats->neg_log_lik = -h[4];
    stats->quad = h[5];
    stats->logdet_sigma = logdet_sigma;
    stats->logdet_precond = logdet_P;
    stats->slq_term = slq;
    stats->logdet = logdet;
    stats->logdet_exact_norm = base + wsum / nprobe + logdet_P;
    stats->newton_iters = ms.newton_iters;
    stats->pcg_iters_mode = ms.pcg_iters_total;
    stats->pcg_iters_slq = slq_iters;
    stats->reserved = 0;
    stats->ms_mode = ms.ms_total;
    stats->ms_slq = ms_slq;
  }
  *newton_ok = converged;
  *cg_ok = !capped && !slq_capped;
  return VIF_OK;
}

vif_status not_converged(vif_ctx* ctx, bool newton_ok, bool cg_ok) {
  if (newton_ok && cg_ok) return VIF_OK;
  return set_err(ctx, VIF_ERR_NOT_CONVERGED, "Newton %s, CG %s", newton_ok ? "converged" : "hit its cap",
                 cg_ok ? "converged" : "hit its cap");
}

// Gradient buffers for nprobe probes (grown on demand).
vif_status grad_buffers(vif_ctx* ctx, int nprobe) {
  const int64_t n = ctx->n;
  if (nprobe > ctx->g_cap) {
    for (double** b : {&ctx->g_U, &ctx->g_Y, &ctx->g_sc}) {
      if (*b) cudaFree(*b);
      *b = nullptr;
    }
    CKS(dalloc(ctx, &ctx->g_U, (size_t)nprobe * n));
    CKS(dalloc(ctx, &ctx->g_Y, (size_t)nprobe * n));
    CKS(dalloc(ctx, &ctx->g_sc, 6 + 3 * (size_t)nprobe));
    ctx->g_cap = nprobe;
  }
  if (!ctx->g_g) {
    CKS(dalloc(ctx, &ctx->g_g, (size_t)n));
    CKS(dalloc(ctx, &ctx->g_v, (size_t)n));
    CKS(dalloc(ctx, &ctx->g_a, (size_t)n));
    CKS(dalloc(ctx, &ctx->g_av, (size_t)n));
    CKS(dalloc(ctx, &ctx->g_dv, (size_t)n));
    CKS(dalloc(ctx, &ctx->g_red, 3 * 256));
  }
  return VIF_OK;
}

// The theta-dependent quantities whose central differences give the gradient, at the perturbed
// hyperparameters tk with N, Z, the mode b~ and W held fixed (out: 6 + 3 nprobe host values):
//   [0] sum log D_i  [1] log det C  [2] sum log(W_i + 1/D_i)  [3] log det C_3
//   [4] b~^T Sigma_dagger^{-1} b~  [5] v^T Sigma_dagger^{-1} b~
//   [6 + i] u_i^T Sigma_dagger^{-1} y_i  [6 + l + i] y_i^T Sigma_dagger^{-1} y_i  [6 + 2l + i] (B y_i)^T W (B y_i)
vif_status grad_forms(vif_ctx* ctx, const vif_cov* tk, LapOps& o, int nprobe, double* out) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  const int m = ctx->m;
  CKS(lap_setup(ctx, tk, nullptr, &o));
  CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, nullptr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                   ctx->l_ll, s));
  CKS(lap_c3(ctx, o));
  double* gs = ctx->g_sc;
  CK(reduce_sum(ctx->logD, n, ctx->red, gs + 0, s));
  if (m > 0) {
    CK(lap_log_sum(ctx->G, m, (int64_t)ctx->fpad + 1, 2.0, ctx->l_red, gs + 1, s));
    CK(lap_log_sum(ctx->l_G3, m, (int64_t)ctx->fpad + 1, 2.0, ctx->l_red, gs + 3, s));
  } else {
    CK(cudaMemsetAsync(gs + 1, 0, sizeof(double), s));
    CK(cudaMemsetAsync(gs + 3, 0, sizeof(double), s));
  }
  CK(lap_log_sum(ctx->l_Ginv, n, 1, -1.0, ctx->l_red, gs + 2, s));
  CK(lap_matvec(o, ctx->l_b, nullptr, ctx->l_sdi, s));
  CK(lap_grad_forms(n, ctx->l_b, ctx->g_v, ctx->l_sdi, nullptr, nullptr, nullptr, ctx->g_red, gs + 4, gs + 5,
                    nullptr, s));
  for (int i = 0; i < nprobe; ++i) {
    const double* Ui = ctx->g_U + (size_t)i * n;
    const double* Yi = ctx->g_Y + (size_t)i * n;
    // lap_matvec leaves D^{-1/2} B y_i in o.t, so that (B y_i)^T W (B y_i) = sum t^2 W D
    CK(lap_matvec(o, Yi, nullptr, ctx->l_sdi, s));
    CK(lap_grad_forms(n, Ui, Yi, ctx->l_sdi, o.t, ctx->l_W, ctx->Dv, ctx->g_red, gs + 6 + i, gs + 6 + nprobe + i,
                      gs + 6 + 2 * nprobe + i, s));
  }
  CK(cudaMemcpyAsync(out, gs, (6 + 3 * (size_t)nprobe) * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double dummy[1];
  CKS(read_status(ctx, dummy, 0));
  return VIF_OK;
}

// The FITC form (Eq. pcls2) of grad_forms, at tk with N, Z, b~ and W fixed (out: 4 + 3 nprobe values):
//   [0] log det D_V  [1] log det M_V  [2] a^T Sigma_dagger a  [3] av^T Sigma_dagger a
//   [4 + i] u_i^T Sigma_dagger y_i  [4 + l + i] y_i^T D_V y_i  [4 + 2l + i] |A y_i|^2
// (a = Sigma_dagger^{-1} b~ and av = Sigma_dagger^{-1} v at theta; y^T P y = y^T D_V y + |A y|^2).  The
// probe terms are taken in blocks of up to LAP_MR_MAXL columns.
vif_status grad_forms_fitc(vif_ctx* ctx, const vif_cov* tk, LapOps& o, int nprobe, double* out) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  const int m = ctx->m;
  CKS(lap_setup(ctx, tk, nullptr, &o));
  o.kind = LAP_FITC;
  CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, nullptr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                   ctx->l_ll, s));
  CKS(lap_fitc_setup(ctx, o, true, tk->variance));
  double* gs = ctx->g_sc;
  CK(lap_log_sum(ctx->l_dvinv, n, 1, -1.0, ctx->l_red, gs + 0, s));
  if (m > 0) {
    CK(lap_log_sum(ctx->l_G3, m, (int64_t)ctx->fpad + 1, 2.0, ctx->l_red, gs + 1, s));
  } else {
    CK(cudaMemsetAsync(gs + 1, 0, sizeof(double), s));
  }
  CK(lap_sigma_matvec(o, ctx->g_a, nullptr, ctx->l_sdi, s));
  CK(lap_grad_forms(n, ctx->g_a, ctx->g_av, ctx->l_sdi, nullptr, nullptr, nullptr, ctx->g_red, gs + 2, gs + 3,
                    nullptr, s));
  CK(lap_recip(ctx->l_dvinv, n, ctx->g_dv, s));
  for (int b0 = 0; b0 < nprobe; b0 += LAP_MR_MAXL) {
    const int L = std::min(LAP_MR_MAXL, nprobe - b0);
    LapMulti w;
    CKS(mr_buffers(ctx, L, &w));
    for (int j = 0; j < L; ++j) {
      CK(lap_mr_column(n, L, j, ctx->mr_x, ctx->g_U + (size_t)(b0 + j) * n, false, s));
      CK(lap_mr_column(n, L, j, ctx->mr_r, ctx->g_Y + (size_t)(b0 + j) * n, false, s));
    }
    CK(lap_mr_sigma_matvec(o, w, ctx->mr_r, ctx->mr_Ap, s, false));
    CK(lap_mr_dot(w, n, ctx->mr_x, ctx->mr_Ap, gs + 4 + b0, s));
    CK(lap_mr_scale2(w, n, ctx->g_dv, nullptr, ctx->mr_r, ctx->mr_z, s));
    CK(lap_mr_dot(w, n, ctx->mr_z, ctx->mr_r, gs + 4 + nprobe + b0, s));
    if (m > 0) {
      CK(lap_mr_ftv(o, w, o.Apad, ctx->mr_r, w.sm, s));
      CK(lap_mr_dot(w, m, w.sm, w.sm, gs + 4 + 2 * nprobe + b0, s));
    } else {
      CK(cudaMemsetAsync(gs + 4 + 2 * nprobe + b0, 0, L * sizeof(double), s));
    }
  }
  CK(cudaMemcpyAsync(out, gs, (4 + 3 * (size_t)nprobe) * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double dummy[1];
  CKS(read_status(ctx, dummy, 0));
  return VIF_OK;
}

}  // namespace

extern "C" {

vif_status vif_laplace_nll(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_laplace_opts* lo,
                           int32_t nprobe, const double* eps, double slq_tol, int32_t slq_max_iter, double* nll_out,
                           double* probe_q, double* probe_zpz, vif_laplace_nll_stats* stats) {
  if (!ctx) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  LapOps o;
  bool newton_ok = true, cg_ok = true;
  CKS(laplace_nll_core(ctx, theta, y, lo, nprobe, eps, slq_tol, slq_max_iter, nll_out, probe_q, probe_zpz, stats,
                       &o, nullptr, nullptr, &newton_ok, &cg_ok));
  return not_converged(ctx, newton_ok, cg_ok);
}

vif_status vif_laplace_nll_grad(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_laplace_opts* lo,
                                int32_t nprobe, const double* eps, double slq_tol, int32_t slq_max_iter,
                                double* nll_out, double* grad_out, double* probe_terms, double* trace_out,
                                vif_laplace_grad_stats* stats) {
  if (!ctx) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  if (!theta || !lo || !grad_out) return set_err(ctx, VIF_ERR_ARG, "theta, opts and grad_out are required");
  if (lo->precond != 0 && lo->precond != LAP_FITC)
    return set_err(ctx, VIF_ERR_ARG, "the gradient takes the VIFDU (0) or the FITC (2) preconditioner");
  const bool fitc = lo->precond == LAP_FITC;
  if (nprobe < 1) return set_err(ctx, VIF_ERR_ARG, "nprobe >= 1 is required");
  CKS(check_cov(ctx, theta, ctx->d));
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  CKS(lap_alloc(ctx));
  CKS(grad_buffers(ctx, nprobe));
  LapOps o;
  bool newton_ok = true, cg_ok = true;
  vif_laplace_grad_stats st{};
  CKS(laplace_nll_core(ctx, theta, y, lo, nprobe, eps, slq_tol, slq_max_iter, nll_out, nullptr, nullptr, &st.nll,
                       &o, ctx->g_U, ctx->g_Y, &newton_ok, &cg_ok));
  const auto t0 = std::chrono::steady_clock::now();
  // dL/db~_j = 1/2 dlog det(Sigma_dagger W + I)/db_j by the probe estimate of the diagonal of
  // (W + Sigma_dagger^{-1})^{-1} (VIFDU) or of (W^{-1} + Sigma_dagger)^{-1} (FITC) (App. B), and
  // v = (W + Sigma_dagger^{-1})^{-1} dL/db~ by CG with the mode's options: on Eq. pcls1, or on Eq. pcls2
  // as v = W^{-1} (W^{-1} + Sigma_dagger)^{-1} Sigma_dagger dL/db~
  CK(lap_ste_diag(n, nprobe, ctx->g_U, ctx->g_Y, ctx->l_b, fitc ? 1 : 0, ctx->g_g, s));
  if (fitc) {
    CK(lap_sigma_matvec(o, ctx->g_g, nullptr, ctx->l_v, s));
  } else {
    CK(cudaMemcpyAsync(ctx->l_v, ctx->g_g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  int vit = 0;
  double vrel = 0.0;
  bool vcap = false;
  CKS(lap_pcg(ctx, o, lo->rel_tol, lo->max_pcg, &vit, &vrel, &vcap));
  cg_ok = cg_ok && !vcap;
  if (fitc) {
    CK(lap_div(n, ctx->l_x, ctx->l_W, ctx->g_v, s));
    // a = Sigma_dagger^{-1} b~ and av = Sigma_dagger^{-1} v at theta
    CK(lap_matvec(o, ctx->l_b, nullptr, ctx->g_a, s));
    CK(lap_matvec(o, ctx->g_v, nullptr, ctx->g_av, s));
  } else {
    CK(cudaMemcpyAsync(ctx->g_v, ctx->l_x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  // central differences in each parameter (sigma1^2, lambda_1..), relative step 1e-4
  const int q = 1 + theta->n_ls;
  const int nf = (fitc ? 4 : 6) + 3 * nprobe;
  std::vector<double> fp((size_t)q * nf), fm((size_t)q * nf), hk(q);
  const std::vector<double> ls(theta->lengthscale, theta->lengthscale + theta->n_ls);
  for (int k = 0; k < q; ++k) {
    for (int sgn = 0; sgn < 2; ++sgn) {
      vif_cov tk = *theta;
      std::vector<double> lk = ls;
      tk.lengthscale = lk.data();
      double* par = k == 0 ? &tk.variance : &lk[k - 1];
      const double h = 1e-4 * std::fabs(*par);
      hk[k] = h;
      *par += sgn ? -h : h;
      double* dst = (sgn ? fm : fp).data() + (size_t)k * nf;
      if (fitc) {
        CKS(grad_forms_fitc(ctx, &tk, o, nprobe, dst));
      } else {
        CKS(grad_forms(ctx, &tk, o, nprobe, dst));
      }
    }
  }
  // leave the factors of theta (and the preconditioner pieces at the mode) in the context
  CKS(lap_setup(ctx, theta, nullptr, &o));
  CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, nullptr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                   ctx->l_ll, s));
  CK(cudaStreamSynchronize(s));
  // assembly (App. B, App. D), T_k the control-variate estimate of the trace:
  //   VIFDU: dL/dth_k = 1/2 b~^T Delta_k b~ + 1/2 (dlog det Sigma_dagger + T_k) - v^T Delta_k b~,
  //          s_ik = d(u_i^T Sigma_dagger^{-1} y_i), c_ik = d((B y_i)^T W (B y_i) + y_i^T Sigma_dagger^{-1} y_i)
  //   FITC:  dL/dth_k = -1/2 a^T dSigma_k a + av^T dSigma_k a + 1/2 T_k,
  //          s_ik = d(u_i^T Sigma_dagger y_i), c_ik = d(y_i^T D_V y_i + |A y_i|^2)
  for (int k = 0; k < q; ++k) {
    const double* P = fp.data() + (size_t)k * nf;
    const double* M = fm.data() + (size_t)k * nf;
    const double h2 = 2.0 * hk[k];
    auto d = [&](int j) { return (P[j] - M[j]) / h2; };
    const int o0 = fitc ? 4 : 6;
    auto s_i = [&](int i) { return d(o0 + i); };
    auto c_i = [&](int i) { return d(o0 + 2 * nprobe + i) + d(o0 + nprobe + i); };
    const double tau = fitc ? d(0) + d(1) : d(2) - d(1) + d(3);   // dlog det P = Tr(P^{-1} dP/dth_k)
    double smean = 0.0;
    for (int i = 0; i < nprobe; ++i) smean += s_i(i);
    smean /= nprobe;
    double num = 0.0, den = 0.0, cvmean = 0.0;
    for (int i = 0; i < nprobe; ++i) {
      const double si = s_i(i), ci = c_i(i);
      num += (si - smean) * (ci - tau);
      den += (ci - tau) * (ci - tau);
      if (probe_terms) {
        probe_terms[((size_t)i * q + k) * 2 + 0] = si;
        probe_terms[((size_t)i * q + k) * 2 + 1] = ci;
      }
    }
    const double copt = den > 0.0 ? num / den : 0.0;
    for (int i = 0; i < nprobe; ++i) cvmean += s_i(i) - copt * c_i(i);
    const double T = cvmean / nprobe + copt * tau;
    grad_out[k] = fitc ? -0.5 * d(2) + d(3) + 0.5 * T : 0.5 * d(4) + 0.5 * (d(0) + d(1) + T) - d(5);
    if (trace_out) {
      trace_out[(size_t)k * 4 + 0] = smean;
      trace_out[(size_t)k * 4 + 1] = copt;
      trace_out[(size_t)k * 4 + 2] = tau;
      trace_out[(size_t)k * 4 + 3] = T;
    }
  }
  st.pcg_iters_v = vit;
  st.reserved = 0;
  st.ms_grad = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return not_converged(ctx, newton_ok, cg_ok);
}

vif_status vif_laplace_predict(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_laplace_opts* lo,
                               const double* Xp, int64_t np, int32_t nsample, const double* eps, double cg_tol,
                               int32_t cg_max_iter, double* mean, double* var, vif_laplace_stats* stats) {
  if (!ctx) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  if (!Xp || !mean || np < 1) return set_err(ctx, VIF_ERR_ARG, "Xp, mean and np >= 1 are required");
  if (var && (nsample < 1 || !eps || !(cg_tol > 0.0) || cg_max_iter < 1))
    return set_err(ctx, VIF_ERR_ARG, "variances need nsample >= 1 normals, cg_tol > 0 and cg_max_iter >= 1");
  if (ctx->mv > 48) return set_err(ctx, VIF_ERR_ARG, "m_v too large for prediction");
  if (lo && lo->precond == 1) return set_err(ctx, VIF_ERR_ARG, "prediction uses VIFDU (0) or FITC (2)");
  LapOps o;
  vif_laplace_stats ms{};
  bool converged = false, capped = false;
  CKS(laplace_run(ctx, theta, y, lo, &o, &ms, &converged, &capped));
  const int64_t n = ctx->n;
  const int d = ctx->d, m = ctx->m, mpad = ctx->mpad, fpad = ctx->fpad, mv = ctx->mv;
  cudaStream_t s = ctx->stream;
  const bool fitc = lo->precond == LAP_FITC;
  double *A64 = nullptr, *F64 = nullptr, *LT64 = nullptr;
  CKS(fp64_buffers(ctx, &A64, &F64, &LT64));
  CKS(predict_buffers(ctx, np));
  if (!ctx->l_pacc) CKS(dalloc(ctx, &ctx->l_pacc, (size_t)np));
  else if (np > ctx->l_pacc_cap) {
    cudaFree(ctx->l_pacc);
    ctx->l_pacc = nullptr;
    CKS(dalloc(ctx, &ctx->l_pacc, (size_t)np));
  }
  ctx->l_pacc_cap = std::max<int64_t>(ctx->l_pacc_cap, np);
  CovParams cp = cov_params(theta);
  // prediction points: scaled coordinates, a_p, neighbour sets (Prop. 3.1 with B_p = I, reading R7)
  CKS(upload(ctx, ctx->pXp, Xp, (size_t)np * d * sizeof(double)));
  CK(scale_coords(ctx->pXp, np, d, ctx->hyp, ctx->hyp + 16, ctx->pXps, nullptr, s));
  CK(lowrank_A<double>(ctx->pXps, ctx->Zs, LT64, mpad, ctx->pAp, np, d, m, mpad, cp.kind, cp.var, s));
  CK(predict_setup(A64, ctx->Xs, n, ctx->pAp, ctx->pXps, np, d, m, mpad, mv, cp, ctx->pcjj, ctx->pcpp, ctx->pNp, s));
  // the predictive-mean operator K_p Sigma_dagger^{-1} v: w = C^{-1} F^T D^{-1/2} B v, r = v - A^T w,
  // then a_p . w + sum_k A_p[k] r_{N_k} per prediction point (Prop. 2.1 algebra)
  auto mean_operator = [&](const double* v, double* out, double* vout) -> vif_status {
    if (m > 0) {
      CK(lap_bx_scaled(o, v, ctx->l_t, s));
      CK(lap_ftv(F64, fpad, m, n, ctx->l_t, ctx->l_part, ctx->l_sm, s));
      CK(lap_spd_apply(ctx->l_LinvC, fpad, m, ctx->l_sm, ctx->l_tm, ctx->pw, s));
    }
    CK(predict_resid(A64, ctx->pw, v, n, m, mpad, ctx->pr, s));
    CK(predict_eval(A64, ctx->Xs, ctx->pAp, ctx->pXps, ctx->pNp, ctx->pr, ctx->pw, ctx->l_LinvC, fpad, np, d, m,
                    mpad, mv, cp, 1, 0.0, out, vout, ctx->status, s));
    return VIF_OK;
  };
  // omega_p and the first part of Omega_p (the latent variance of Prop. 2.1 with b~ for y)
  CKS(mean_operator(ctx->l_b, ctx->pmean, ctx->pvar));
  int cg_total = 0;
  bool cg_capped = false;
  double rel = 0.0;
  if (var) {
    // Alg. 1 (SBPV): z4 ~ N(0, Sigma_dagger), z6 = Sigma_dagger^{-1} z4 + W^{1/2} z2, z7 solves the
    // Newton system, z8 = K_p Sigma_dagger^{-1} z7; the variances gain mean(z8 o z8)
    if (!ctx->slq_eps) CKS(dalloc(ctx, &ctx->slq_eps, (size_t)m + 2 * (size_t)n));
    CK(cudaMemsetAsync(ctx->l_pacc, 0, (size_t)np * sizeof(double), s));
    const size_t per = (size_t)m + 2 * (size_t)n;
    if (fitc) CKS(lap_fitc_setup(ctx, o, false, theta->variance));
    else CKS(lap_c3(ctx, o));
    // the draws' CGs run side by side in blocks of up to LAP_MR_MAXL columns
    for (int b0 = 0; b0 < nsample; b0 += LAP_MR_MAXL) {
      const int L = std::min(LAP_MR_MAXL, nsample - b0);
      LapMulti w;
      CKS(mr_buffers(ctx, L, &w));
      for (int j = 0; j < L; ++j) {
        CKS(upload(ctx, ctx->slq_eps, eps + (size_t)(b0 + j) * per, per * sizeof(double)));
        const double* z3 = ctx->slq_eps;
        const double* z1 = ctx->slq_eps + m;
        const double* z2 = ctx->slq_eps + m + n;
        CK(lap_probe_prep(n, ctx->Dv, ctx->l_W, nullptr, z1, z2, ctx->l_r, ctx->l_z, s));
        CK(lap_solve_B(o, ctx->l_r, ctx->l_p, s));
        if (m > 0) {
          CK(lap_rows_dot_add(A64, mpad, m, n, z3, ctx->l_p, ctx->l_Ap, s));
        } else {
          CK(cudaMemcpyAsync(ctx->l_Ap, ctx->l_p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        CK(lap_matvec(o, ctx->l_Ap, nullptr, ctx->l_x, s));
        CK(lap_vec_add(n, ctx->l_x, ctx->l_z, ctx->l_v, s));
        if (fitc) {   // Eq. pcls2: z7 = W^{-1} (W^{-1} + Sigma_dagger)^{-1} Sigma_dagger z6
          CK(lap_sigma_matvec(o, ctx->l_v, nullptr, ctx->l_sdi, s));
          CK(cudaMemcpyAsync(ctx->l_v, ctx->l_sdi, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        CK(lap_mr_column(n, L, j, ctx->mr_v, ctx->l_v, false, s));
      }
      std::vector<int> its(L);
      std::vector<double> rels(L), rz0(L);
      std::vector<char> caps(L);
      std::vector<std::vector<double>> al(L), be(L);
      CKS(lap_pcg_multi(ctx, o, w, cg_tol, cg_max_iter, its, rels, caps, al, be, rz0, nullptr));
      for (int j = 0; j < L; ++j) {
        cg_total += its[j];
        cg_capped = cg_capped || caps[j];
        rel = std::max(rel, rels[j]);
        CK(lap_mr_column(n, L, j, ctx->mr_x, ctx->l_x, true, s));
        if (fitc) CK(lap_div(n, ctx->l_x, ctx->l_W, ctx->l_x, s));
        CKS(mean_operator(ctx->l_x, ctx->pcpp, nullptr));
        CK(lap_sq_accumulate(np, ctx->pcpp, ctx->l_pacc, s));
      }
    }
    CK(lap_axpy_host(np, 1.0 / nsample, ctx->pvar, ctx->l_pacc, ctx->pvar, s));
  }
  double sc[1];
  CKS(read_status(ctx, sc, 0));
  CKS(download(ctx, mean, ctx->pmean, (size_t)np * sizeof(double)));
  if (var) CKS(download(ctx, var, ctx->pvar, (size_t)np * sizeof(double)));
  if (stats) {
    *stats = ms;
    stats->pcg_iters_total = ms.pcg_iters_total + cg_total;
  }
  if (!converged || capped || cg_capped)
    return set_err(ctx, VIF_ERR_NOT_CONVERGED, "Newton %s, CG %s", converged ? "converged" : "hit its cap",
                   (capped || cg_capped) ? "hit its cap" : "converged");
  return VIF_OK;
}

vif_status vif_tridiag_log_quadrature(const double* diag, const double* offdiag, int32_t k, double* out) {
  if (!diag || !out || k < 0 || (k > 1 && !offdiag)) return VIF_ERR_ARG;
  std::vector<double> d(diag, diag + k), e(k > 1 ? offdiag : diag, k > 1 ? offdiag + (k - 1) : diag);
  return tridiag_log_quadrature(d, e, out) ? VIF_OK : VIF_ERR_NOT_PD;
}

size_t vif_mlp_bytes(void) { return mlp_bytes(); }

vif_status vif_mlp_init(void* net, uint64_t seed, void* stream) {
  if (!net) return VIF_ERR_ARG;
  if (mlp_init(net, seed, (cudaStream_t)stream) != cudaSuccess) return VIF_ERR_CUDA;
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? VIF_OK : VIF_ERR_CUDA;
}

vif_status vif_mlp_set_params(void* net, const float* params, void* stream) {
  if (!net || !params) return VIF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, VIF_MLP_NPARAM * sizeof(float)) != cudaSuccess) return VIF_ERR_NOMEM;
  cudaError_t e = cudaMemcpyAsync(tmp, params, VIF_MLP_NPARAM * sizeof(float), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = mlp_set(net, tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  return e == cudaSuccess ? VIF_OK : VIF_ERR_CUDA;
}

vif_status vif_mlp_get_params(const void* net, float* params) {
  if (!net || !params) return VIF_ERR_ARG;
  return cudaMemcpy(params, mlp_master(net), VIF_MLP_NPARAM * sizeof(float), cudaMemcpyDefault) == cudaSuccess
             ? VIF_OK
             : VIF_ERR_CUDA;
}

vif_status vif_mlp_forward(const void* net, const float* feats, int64_t n, float* c, void* stream) {
  if (!net || !feats || !c || n < 1) return VIF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (mlp_forward_f32(net, feats, n, c, s) != cudaSuccess) return VIF_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? VIF_OK : VIF_ERR_CUDA;
}

vif_status vif_mlp_backward(const void* net, const float* feats, const float* gc, int64_t n, float* grad,
                            void* stream) {
  if (!net || !feats || !gc || !grad || n < 1) return VIF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float* part = nullptr;
  const size_t pc = (size_t)mlp_backward_blocks(n) * ((VIF_MLP_NPARAM + 63) / 64 * 64);
  if (cudaMalloc((void**)&part, pc * sizeof(float)) != cudaSuccess) return VIF_ERR_NOMEM;
  cudaError_t e = mlp_backward(net, feats, gc, n, part, grad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  return e == cudaSuccess ? VIF_OK : VIF_ERR_CUDA;
}

vif_status vif_mlp_features(vif_ctx* ctx, const double* W, float* feats) {
  if (!ctx || !W || !feats) return VIF_ERR_ARG;
  if (!ctx->lap_ready) return set_err(ctx, VIF_ERR_STATE, "call vif_laplace_mode or vif_mlp_train first");
  CKS(mlp_scratch(ctx));
  CKS(upload(ctx, ctx->l_t, W, (size_t)ctx->n * sizeof(double)));
  CK(mlp_features(ctx->l_t, ctx->Dv, ctx->Acoef, ctx->m_rho, ctx->N, ctx->ch_ptr, ctx->ch_row, ctx->ch_slot,
                  ctx->n, ctx->mv, ctx->m_feat, ctx->stream));
  return download(ctx, feats, ctx->m_feat, (size_t)ctx->n * VIF_MLP_NIN * sizeof(float));
}

vif_status vif_mlp_train(vif_ctx* ctx, const vif_cov* theta, const double* y, const vif_mlp_train_opts* to,
                         void* net, vif_mlp_train_stats* stats) {
  if (!ctx || !to || !net || !y) return VIF_ERR_ARG;
  ctx->err[0] = 0;
  CKS(check_cov(ctx, theta, ctx->d));
  if (ctx->likelihood != VIF_BERNOULLI_LOGIT || theta->nugget != 0.0)
    return set_err(ctx, VIF_ERR_STATE, "training needs a Bernoulli-logit context and nugget 0");
  if (to->steps_per_system < 1 || to->probes < 1 || to->max_newton < 1 || !(to->lr > 0.f))
    return set_err(ctx, VIF_ERR_ARG, "invalid training options");
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  LapOps o;
  CKS(lap_setup(ctx, theta, y, &o));
  CKS(mlp_scratch(ctx));
  double* sc = ctx->l_sc;
  CK(cudaMemsetAsync(ctx->l_b, 0, n * sizeof(double), s));
  double loss_first = -1.0, loss_last = 0.0;
  int systems = 0;
  uint64_t probe_ctr = 0;
  const double coeff = -2.0 / to->probes;
  for (int newton = 1; newton <= to->max_newton; ++newton) {
    ++systems;
    CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, nullptr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                     ctx->l_ll, s));
    for (int step = 0; step < to->steps_per_system; ++step) {
      CKS(mlp_correction_c(ctx, net));
      CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, ctx->l_corr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om,
                       ctx->l_rsD, ctx->l_ll, s));
      CKS(lap_c3(ctx, o));
      CK(mlp_zero(ctx->m_gc, n, s));
      CK(cudaMemsetAsync(sc + 10, 0, sizeof(double), s));
      double loss = 0.0;
      for (int k = 0; k < to->probes; ++k) {
        // z -> l_x, A z -> l_r, u = P^-1 A z -> l_z, r = u - z -> l_p, s = P^-1 r -> l_Ap
        CK(mlp_rademacher(to->seed * 0x9E3779B97F4A7C15ull + (++probe_ctr), n, ctx->l_x, s));
        CK(lap_matvec(o, ctx->l_x, ctx->l_W, ctx->l_r, s));
        CK(lap_precond(o, ctx->l_r, ctx->l_z, s));
        {
          // r = u - z: l_p = l_z - 1 * l_x
          double one = 1.0;
          CK(cudaMemcpyAsync(sc + 11, &one, sizeof(double), cudaMemcpyHostToDevice, s));
          CK(lap_axpy(n, sc + 11, ctx->l_z, ctx->l_x, ctx->l_p, 1, s));
        }
        CK(lap_precond(o, ctx->l_p, ctx->l_Ap, s));
        CK(mlp_lp_grad(ctx->N, ctx->Acoef, n, ctx->mv, ctx->l_Ap, ctx->l_z, ctx->l_W, ctx->l_corr, coeff, ctx->m_gc,
                       s));
        CK(lap_dot(ctx->l_p, ctx->l_p, n, ctx->l_red, sc + 9, s));
        CK(cudaMemcpyAsync(ctx->h_pin + 16, sc + 9, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        loss += ctx->h_pin[16];
      }
      loss /= (double)to->probes * (double)n;
      if (loss_first < 0.0) loss_first = loss;
      loss_last = loss;
      CK(mlp_backward(net, ctx->m_feat, ctx->m_gc, n, ctx->m_part, ctx->m_grad, s));
      CK(mlp_adam(net, ctx->m_grad, to->lr, s));
    }
    // next Newton iterate with the plain preconditioner
    CK(lap_pointwise(ctx->y, ctx->l_b, ctx->Dv, nullptr, n, ctx->l_W, ctx->l_v, ctx->l_Ginv, ctx->l_om, ctx->l_rsD,
                     ctx->l_ll, s));
    CKS(lap_c3(ctx, o));
    int it = 0;
    double rel = 0.0;
    bool capped = false;
    CKS(lap_pcg(ctx, o, 1e-6, 1000, &it, &rel, &capped));
    CK(cudaMemcpyAsync(ctx->l_b, ctx->l_x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaStreamSynchronize(s));
  if (stats) {
    stats->systems = systems;
    stats->loss_first = loss_first;
    stats->loss_last = loss_last;
  }
  return VIF_OK;
}

}  // extern "C"

struct vif_batch {
  std::vector<vif_ctx*> ctx;
  std::vector<vif_cov> th;
  std::vector<std::vector<double>> ls;
  std::vector<const double*> ys;
  cudaStream_t origin = nullptr;   // internal capture stream (the legacy stream cannot be captured)
  cudaStream_t user = nullptr;     // caller's stream: replays are ordered on it
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> ev;
  cudaGraphExec_t exec = nullptr;
  double* hpin = nullptr;      // pinned hyperparameter staging, 32 doubles per problem
  double* dout = nullptr;      // device: NLL per problem
  int* dst = nullptr;          // device: status words per problem (4 each)
  double* hout = nullptr;      // pinned: NLL + status copy-back
  int branches = 8, split_div = 1;
  int batched_factor = 0;   // factor stage of the bucketed problems: 0 per problem, 1 persistent, 2 flat
  double best_ms = 0.0;
  // the dense float64 stages of every problem, one launch per step for all problems
  DenseBatch chol_sm, trtri_sm, chol_cap;
  // the factor stage of the problems in buckets (precision x block-size class), each one
  // persistent launch over all its problems' points; in_bucket[p]: problem p belongs to one
  struct FactorBucket {
    bool fp32;
    int mv_max, njobs;
    int64_t total;
    std::vector<FactorTable<float>> t32;    // the jobs again, as parameter-bank tables
    std::vector<FactorTable<double>> t64;
    void* djobs = nullptr;
    int64_t* doff = nullptr;
    unsigned long long* queue = nullptr;
  };
  std::vector<FactorBucket> fbuckets;
  std::vector<char> in_bucket;
  char err[512] = {0};
};

namespace {

// Capture-safe likelihood enqueue for one context on stream s (no host syncs), in phases
// around the batched dense stages: (pre) hyperparameters from pinned staging, scaled
// coordinates, Sigma_m; [Cholesky and inverse of every Sigma_m]; (mid) A, the residual
// Vecchia factors, the Gram and sum log D_i; [Cholesky of every augmented capacitance
// matrix]; (post) the scalar and the status words into the batch's slots.
struct CtxSwap {   // the context's stream, timing and Gram split for the duration of a phase
  vif_ctx* c;
  cudaStream_t keep;
  bool keep_t;
  int keep_split;
  CtxSwap(vif_ctx* ctx, cudaStream_t s, int split_div, bool fp64) : c(ctx) {
    keep = c->stream;
    keep_t = c->timing;
    keep_split = c->nsplit;
    c->stream = s;
    c->timing = false;
    // the float64 Gram's row slices follow the tuned split; the float32 (tensor-core) Gram
    // picks its own one-wave split, so a batched call sums its rows exactly as a single call
    if (fp64) c->nsplit = std::max(1, keep_split / split_div);
  }
  ~CtxSwap() {
    c->stream = keep;
    c->timing = keep_t;
    c->nsplit = keep_split;
  }
};

template <typename T>
vif_status enqueue_pre(vif_ctx* ctx, const vif_cov* th, const double* hyp_src, const double* ydev, cudaStream_t s,
                       int split_div) {
  CtxSwap sw(ctx, s, split_div, sizeof(T) == 8);
  const bool mixed = sizeof(T) == 4;
  if (cudaMemsetAsync(ctx->status, 0, 4 * sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(ctx->y, ydev, ctx->n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(ctx->hyp, hyp_src, 32 * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      scale_coords(ctx->X, ctx->n, ctx->d, ctx->hyp, ctx->hyp + 16, ctx->Xs, mixed ? ctx->Xs32 : nullptr, s) !=
          cudaSuccess ||
      (ctx->m > 0 && scale_coords(ctx->Z, ctx->m, ctx->d, ctx->hyp, ctx->hyp + 16, ctx->Zs,
                                  mixed ? ctx->Zs32 : nullptr, s) != cudaSuccess))
    return set_err(ctx, VIF_ERR_CUDA, "batch enqueue failed");
  if (ctx->m <= 0) return VIF_OK;
  const CovParams cp = cov_params(th);
  CK(build_sigma_m(ctx->Zs, ctx->m, ctx->d, cp, ctx->Sm, ctx->ldm, s));
  // the inverse's zeroed upper part and k-slice scratch (as dense_trtri_lower does)
  CK(cudaMemset2DAsync(ctx->Linv, ctx->ldm * sizeof(double), 0, ctx->m * sizeof(double), ctx->m, s));
  CK(cudaMemsetAsync(ctx->trw, 0, trtri_work_doubles(ctx->m) * sizeof(double), s));
  return VIF_OK;
}

// with_factor = false: the factor stage runs in a bucket launch (enqueue_gram follows it)
template <typename T>
vif_status enqueue_mid(vif_ctx* ctx, const vif_cov* th, cudaStream_t s, int split_div, bool with_factor = true,
                       bool with_gram = true) {
  CtxSwap sw(ctx, s, split_div, sizeof(T) == 8);
  const CovParams cp = cov_params(th);
  const bool mixed = sizeof(T) == 4;
  T* A = (T*)ctx->A;
  T* LinvT = (T*)ctx->LinvT;
  T* F = (T*)ctx->F;
  const T* Xs = mixed ? (const T*)ctx->Xs32 : (const T*)ctx->Xs;
  const T* Zs = mixed ? (const T*)ctx->Zs32 : (const T*)ctx->Zs;
  if constexpr (sizeof(T) == 8)
    if (ctx->m > 0) CK(linv_transpose<T>(ctx->Linv, ctx->m, ctx->ldm, LinvT, ctx->mpad, s));
  CK(lowrank_A_any<T>(ctx, cp, A, LinvT, Xs, Zs));
  if (with_factor) CKS(run_factor<T>(ctx, cp, A, Xs, F, factor_on_tc(ctx)));
  if (with_gram) {
    CK(gram_FtF<T>(F, ctx->n, ctx->fpad, ctx->m, ctx->part, ctx->nsplit, ctx->G, ctx->fpad, s, nullptr,
                   ctx->status));
    CK(reduce_sum(ctx->logD, ctx->n, ctx->red, ctx->dscal, s));
  }
  return VIF_OK;
}

template <typename T>
vif_status enqueue_gram(vif_ctx* ctx, cudaStream_t s, int split_div) {
  CtxSwap sw(ctx, s, split_div, sizeof(T) == 8);
  CK(gram_FtF<T>((T*)ctx->F, ctx->n, ctx->fpad, ctx->m, ctx->part, ctx->nsplit, ctx->G, ctx->fpad, s, nullptr,
                 ctx->status));
  CK(reduce_sum(ctx->logD, ctx->n, ctx->red, ctx->dscal, s));
  return VIF_OK;
}

// factor buckets: problems of one precision and block-size class (those on the CUDA-core
// factor path), their points back to back; built once per batch
template <typename T>
FactorJob<T> factor_job(vif_ctx* c, const vif_cov* th) {
  const bool mixed = sizeof(T) == 4;
  FactorJob<T> J{};
  J.A = (const T*)c->A;
  J.Xs = mixed ? (const T*)c->Xs32 : (const T*)c->Xs;
  J.N = c->N;
  J.order = c->order;
  J.y = c->y;
  J.n = c->n;
  J.d = c->d;
  J.m = c->m;
  J.mpad = c->mpad;
  J.mv = c->mv;
  J.fpad = c->fpad;
  J.cp = cov_params(th);
  J.F = (T*)c->F;
  J.Acoef = c->Acoef;
  J.Dv = c->Dv;
  J.logD = c->logD;
  J.status = c->status;
  return J;
}

cudaError_t batch_factor_init(vif_batch* b) {
  const int np = (int)b->ctx.size();
  b->in_bucket.assign(np, 0);
  for (int fp32 = 0; fp32 < 2; ++fp32)
    for (int cls = 2; cls <= 7; ++cls) {
      std::vector<int> members;
      for (int p = 0; p < np; ++p) {
        vif_ctx* c = b->ctx[p];
        if ((c->precision == VIF_MIXED) != (fp32 == 1) || factor_block_class(c->mv) != cls) continue;
        if (factor_on_tc(c)) continue;   // per-point Grams from the tensor cores: its own launches
        members.push_back(p);
      }
      if (members.empty()) continue;
      vif_batch::FactorBucket fb;
      fb.fp32 = fp32 == 1;
      fb.njobs = (int)members.size();
      fb.mv_max = 0;
      std::vector<int64_t> off(1, 0);
      std::vector<FactorJob<float>> j32;
      std::vector<FactorJob<double>> j64;
      for (int p : members) {
        vif_ctx* c = b->ctx[p];
        fb.mv_max = std::max(fb.mv_max, c->mv);
        off.push_back(off.back() + c->n);
        if (fp32) j32.push_back(factor_job<float>(c, &b->th[p]));
        else j64.push_back(factor_job<double>(c, &b->th[p]));
        b->in_bucket[p] = 1;
      }
      const size_t jb = fp32 ? sizeof(FactorJob<float>) * j32.size() : sizeof(FactorJob<double>) * j64.size();
      cudaError_t e = cudaMalloc(&fb.djobs, jb);
      if (e == cudaSuccess) e = cudaMalloc((void**)&fb.doff, sizeof(int64_t) * off.size());
      if (e == cudaSuccess) e = cudaMalloc((void**)&fb.queue, sizeof(unsigned long long));
      if (e == cudaSuccess)
        e = cudaMemcpy(fb.djobs, fp32 ? (const void*)j32.data() : (const void*)j64.data(), jb, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(fb.doff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice);
      fb.total = off.back();
      for (size_t j0 = 0; j0 < members.size(); j0 += FT_MAXJ) {
        const int nj = (int)std::min(members.size() - j0, (size_t)FT_MAXJ);
        auto fill = [&](auto& tab, const auto& jobs) {
          tab.njobs = nj;
          tab.boff[0] = 0;
          for (int k = 0; k < nj; ++k) {
            tab.job[k] = jobs[j0 + k];
            tab.boff[k + 1] = tab.boff[k] + (int)((jobs[j0 + k].n + FT_BLOCK_POINTS - 1) / FT_BLOCK_POINTS);
          }
        };
        if (fp32) {
          fb.t32.emplace_back();
          fill(fb.t32.back(), j32);
        } else {
          fb.t64.emplace_back();
          fill(fb.t64.back(), j64);
        }
      }
      b->fbuckets.push_back(std::move(fb));
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

vif_status enqueue_post(vif_ctx* ctx, double* nll_dst, int* st_dst, cudaStream_t s) {
  CK(nll_finish(ctx->G, ctx->fpad, ctx->m, ctx->dscal, ctx->n, ctx->dscal + 1, s));
  if (cudaMemcpyAsync(nll_dst, ctx->dscal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(st_dst, ctx->status, 4 * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return set_err(ctx, VIF_ERR_CUDA, "batch enqueue failed");
  return VIF_OK;
}

// the dense stages of every problem as batched launches (jobs fixed for the batch's life)
cudaError_t batch_dense_init(vif_batch* b) {
  std::vector<DenseJob> sm, cap;
  for (vif_ctx* c : b->ctx) {
    if (c->m > 0) sm.push_back({c->Sm, c->Linv, c->trw, c->status, c->m, c->ldm, ST_NOTPD_SIGMAM});
    cap.push_back({c->G, nullptr, nullptr, c->status, c->m + 1, c->fpad, ST_NOTPD_CAP});
  }
  cudaError_t e = dense_batch_init(sm, false, &b->chol_sm);
  if (e == cudaSuccess) e = dense_batch_init(sm, true, &b->trtri_sm);
  if (e == cudaSuccess) e = dense_batch_init(cap, false, &b->chol_cap);
  return e;
}

// bf: the factor stage of the bucketed problems as bucket launches, 1 persistent (warps take
// chunks from a device counter), 2 flat (one warp per point, the jobs in the parameter bank);
// 0 in each problem's branch
vif_status batch_capture(vif_batch* b, int branches, int split_div, int bf, cudaGraphExec_t* exec) {
  const int np = (int)b->ctx.size();
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VIF_ERR_CUDA;
  vif_status st = VIF_OK;
  int nev = 0;
  // origin -> every branch
  auto fork = [&]() {
    cudaEvent_t e = b->ev[nev++];
    cudaEventRecord(e, b->origin);
    for (int k = 0; k < branches; ++k) cudaStreamWaitEvent(b->br[k], e, 0);
  };
  // every branch -> origin
  auto join = [&]() {
    for (int k = 0; k < branches; ++k) {
      cudaEvent_t e = b->ev[nev++];
      cudaEventRecord(e, b->br[k]);
      cudaStreamWaitEvent(b->origin, e, 0);
    }
  };
  auto each = [&](auto&& fn) {
    for (int p = 0; p < np && st == VIF_OK; ++p) st = fn(p, b->ctx[p], b->br[p % branches]);
  };
  fork();
  each([&](int p, vif_ctx* c, cudaStream_t s) {
    const double* h = b->hpin + 32 * p;
    return c->precision == VIF_MIXED ? enqueue_pre<float>(c, &b->th[p], h, b->ys[p], s, split_div)
                                     : enqueue_pre<double>(c, &b->th[p], h, b->ys[p], s, split_div);
  });
  join();
  if (st == VIF_OK && (dense_batch_run(b->chol_sm, b->origin) != cudaSuccess ||
                       dense_batch_run(b->trtri_sm, b->origin) != cudaSuccess))
    st = VIF_ERR_CUDA;
  fork();
  each([&](int p, vif_ctx* c, cudaStream_t s) {
    const bool own = !(bf && b->in_bucket[p]);   // factor stage in this branch
    return c->precision == VIF_MIXED ? enqueue_mid<float>(c, &b->th[p], s, split_div, own, own)
                                     : enqueue_mid<double>(c, &b->th[p], s, split_div, own, own);
  });
  if (bf) {
    join();
    for (const auto& fb : b->fbuckets) {
      if (st != VIF_OK) break;
      cudaError_t e = cudaSuccess;
      if (bf == 2) {
        for (const auto& t : fb.t32)
          if (e == cudaSuccess) e = vecchia_factor_table<float>(t, fb.mv_max, b->origin);
        for (const auto& t : fb.t64)
          if (e == cudaSuccess) e = vecchia_factor_table<double>(t, fb.mv_max, b->origin);
      } else {
        e = fb.fp32 ? vecchia_factor_batched<float>((const FactorJob<float>*)fb.djobs, fb.doff, fb.njobs,
                                                    fb.mv_max, fb.queue, b->ctx[0]->nsm, b->origin)
                    : vecchia_factor_batched<double>((const FactorJob<double>*)fb.djobs, fb.doff, fb.njobs,
                                                     fb.mv_max, fb.queue, b->ctx[0]->nsm, b->origin);
      }
      if (e != cudaSuccess) st = VIF_ERR_CUDA;
    }
    fork();
    each([&](int p, vif_ctx* c, cudaStream_t s) {
      if (!b->in_bucket[p]) return VIF_OK;
      return c->precision == VIF_MIXED ? enqueue_gram<float>(c, s, split_div) : enqueue_gram<double>(c, s, split_div);
    });
  }
  join();
  if (st == VIF_OK && dense_batch_run(b->chol_cap, b->origin) != cudaSuccess) st = VIF_ERR_CUDA;
  fork();
  each([&](int p, vif_ctx* c, cudaStream_t s) { return enqueue_post(c, b->dout + p, b->dst + 4 * p, s); });
  join();
  cudaError_t e = cudaStreamEndCapture(b->origin, &g);
  if (st != VIF_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != VIF_OK ? st : VIF_ERR_CUDA;
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? VIF_OK : VIF_ERR_CUDA;
}

}  // namespace

extern "C" {

vif_status vif_batch_create(vif_ctx* const* ctxs, int32_t nprob, const vif_cov* thetas, const double* const* ys,
                            void* stream, vif_batch** out) {
  if (!out || !ctxs || !thetas || !ys || nprob < 1) return VIF_ERR_ARG;
  *out = nullptr;
  vif_batch* b = new vif_batch();
  auto fail = [&](vif_status st, const char* msg) {
    vif_internal_set_global_error(msg);
    vif_batch_destroy(b);
    return st;
  };
  b->user = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess)
    return fail(VIF_ERR_CUDA, "vif_batch_create: stream creation failed");
  for (int p = 0; p < nprob; ++p) {
    vif_ctx* c = ctxs[p];
    if (!c || !ys[p] || c->likelihood != VIF_GAUSSIAN) return fail(VIF_ERR_ARG, "vif_batch_create: bad problem");
    if (check_cov(c, &thetas[p], c->d) != VIF_OK) return fail(VIF_ERR_ARG, "vif_batch_create: bad theta");
    if (!is_device_ptr(ys[p])) return fail(VIF_ERR_ARG, "vif_batch_create: ys must be device pointers");
    b->ctx.push_back(c);
    b->ls.emplace_back(thetas[p].lengthscale, thetas[p].lengthscale + thetas[p].n_ls);
    b->ys.push_back(ys[p]);
  }
  for (int p = 0; p < nprob; ++p) {
    vif_cov t = thetas[p];
    t.lengthscale = b->ls[p].data();
    b->th.push_back(t);
  }
  if (cudaMallocHost((void**)&b->hpin, sizeof(double) * 32 * nprob) != cudaSuccess ||
      cudaMallocHost((void**)&b->hout, sizeof(double) * 3 * nprob) != cudaSuccess ||
      cudaMalloc((void**)&b->dout, sizeof(double) * nprob) != cudaSuccess ||
      cudaMalloc((void**)&b->dst, sizeof(int) * 4 * nprob) != cudaSuccess)
    return fail(VIF_ERR_NOMEM, "vif_batch_create: allocation failed");
  for (int p = 0; p < nprob; ++p) {
    double* h = b->hpin + 32 * p;
    const vif_ctx* c = b->ctx[p];
    for (int t = 0; t < 16; ++t) {
      h[t] = (t < c->d) ? 1.0 / b->th[p].lengthscale[b->th[p].n_ls == 1 ? 0 : t] : 0.0;
      h[16 + t] = c->center[t];
    }
  }
  if (batch_dense_init(b) != cudaSuccess) return fail(VIF_ERR_NOMEM, "vif_batch_create: dense plan failed");
  const int maxbr = 32;
  b->br.resize(maxbr);
  b->ev.resize(4 * (maxbr + 1));   // up to four fork / join pairs per capture
  for (auto& s : b->br)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return fail(VIF_ERR_CUDA, "vif_batch_create: stream creation failed");
  for (auto& e : b->ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(VIF_ERR_CUDA, "vif_batch_create: event creation failed");
  // autotuner: time one replay of each launch shape, keep the fastest
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  if (batch_factor_init(b) != cudaSuccess) {
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return fail(VIF_ERR_NOMEM, "vif_batch_create: factor buckets failed");
  }
  // concurrent branches, float64 Gram split divisor, factor stage as bucket launches
  const int shapes[][3] = {{4, 1, 0}, {8, 1, 0}, {16, 1, 0}, {32, 1, 0}, {8, 2, 0}, {16, 2, 0},
                           {8, 1, 1}, {32, 1, 1}, {8, 1, 2}, {32, 1, 2}};
  double best = 1e30;
  for (const auto& sh : shapes) {
    if (sh[0] > nprob && sh[0] != 4) continue;
    cudaGraphExec_t ex = nullptr;
    if (sh[2] && b->fbuckets.empty()) continue;
    if (batch_capture(b, sh[0], sh[1], sh[2], &ex) != VIF_OK) {
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      return fail(VIF_ERR_CUDA, "vif_batch_create: graph capture failed");
    }
    cudaGraphLaunch(ex, b->user);   // warm-up
    cudaEventRecord(t0, b->user);
    cudaGraphLaunch(ex, b->user);
    cudaEventRecord(t1, b->user);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best) {
      best = ms;
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = ex;
      b->branches = sh[0];
      b->split_div = sh[1];
      b->batched_factor = sh[2];
    } else {
      cudaGraphExecDestroy(ex);
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  b->best_ms = best;
  if (cudaGetLastError() != cudaSuccess || !b->exec) return fail(VIF_ERR_CUDA, "vif_batch_create: CUDA error");
  *out = b;
  return VIF_OK;
}

vif_status vif_batch_run(vif_batch* b, double* nll_out) {
  if (!b || !nll_out) return VIF_ERR_ARG;
  const int np = (int)b->ctx.size();
  if (cudaGraphLaunch(b->exec, b->user) != cudaSuccess) return VIF_ERR_CUDA;
  double* h = b->hout;
  if (cudaMemcpyAsync(h, b->dout, np * sizeof(double), cudaMemcpyDeviceToHost, b->user) != cudaSuccess ||
      cudaMemcpyAsync(h + np, b->dst, np * 4 * sizeof(int), cudaMemcpyDeviceToHost, b->user) != cudaSuccess ||
      cudaStreamSynchronize(b->user) != cudaSuccess)
    return VIF_ERR_CUDA;
  const int* st = reinterpret_cast<const int*>(h + np);
  for (int p = 0; p < np; ++p)
    if (st[4 * p] != ST_OK) {
      snprintf(b->err, sizeof(b->err), "problem %d: device status %d at index %d", p, st[4 * p], st[4 * p + 1]);
      vif_internal_set_global_error(b->err);
      return st[4 * p] == ST_TIMEOUT ? VIF_ERR_TIMEOUT : VIF_ERR_NOT_PD;
    }
  for (int p = 0; p < np; ++p) nll_out[p] = h[p];
  return VIF_OK;
}

vif_status vif_batch_info(const vif_batch* b, int32_t* branches, int32_t* split_div, double* ms) {
  if (!b) return VIF_ERR_ARG;
  if (branches) *branches = b->branches;
  if (split_div) *split_div = b->split_div;
  if (ms) *ms = b->best_ms;
  return VIF_OK;
}

vif_status vif_batch_set_shape(vif_batch* b, int32_t branches, int32_t split_div, int32_t batched_factor) {
  if (!b || branches < 1 || branches > (int32_t)b->br.size() || split_div < 1 || batched_factor < 0 ||
      batched_factor > 2)
    return VIF_ERR_ARG;
  if (batched_factor && b->fbuckets.empty()) return VIF_ERR_ARG;
  if (cudaStreamSynchronize(b->user) != cudaSuccess) return VIF_ERR_CUDA;
  cudaGraphExec_t ex = nullptr;
  if (batch_capture(b, branches, split_div, batched_factor, &ex) != VIF_OK) return VIF_ERR_CUDA;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = ex;
  b->branches = branches;
  b->split_div = split_div;
  b->batched_factor = batched_factor;
  return VIF_OK;
}

vif_status vif_batch_factor_info(const vif_batch* b, int32_t* batched_factor, int32_t* nbuckets,
                                 int32_t* nbucketed) {
  if (!b) return VIF_ERR_ARG;
  if (batched_factor) *batched_factor = b->batched_factor;
  if (nbuckets) *nbuckets = (int32_t)b->fbuckets.size();
  if (nbucketed) {
    int32_t k = 0;
    for (char c : b->in_bucket) k += c ? 1 : 0;
    *nbucketed = k;
  }
  return VIF_OK;
}

void vif_batch_destroy(vif_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->user);
  if (b->origin) {
    cudaStreamSynchronize(b->origin);
    cudaStreamDestroy(b->origin);
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->br)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto& fb : b->fbuckets) {
    if (fb.djobs) cudaFree(fb.djobs);
    if (fb.doff) cudaFree(fb.doff);
    if (fb.queue) cudaFree(fb.queue);
  }
  dense_batch_free(&b->chol_sm);
  dense_batch_free(&b->trtri_sm);
  dense_batch_free(&b->chol_cap);
  if (b->hpin) cudaFreeHost(b->hpin);
  if (b->hout) cudaFreeHost(b->hout);
  if (b->dout) cudaFree(b->dout);
  if (b->dst) cudaFree(b->dst);
  delete b;
}

vif_status vif_set_neighbors(vif_ctx* ctx, const int32_t* N) {
  if (!ctx || !N) return VIF_ERR_ARG;
  if (ctx->mv == 0) return VIF_OK;
  const size_t cnt = (size_t)ctx->n * ctx->mv;
  std::vector<int32_t> h(cnt);
  if (is_device_ptr(N)) {
    CK(cudaMemcpy(h.data(), N, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost));
  } else {
    memcpy(h.data(), N, cnt * sizeof(int32_t));
  }
  // row i: min(i, mv) distinct predecessors in ascending order, then -1
  for (int64_t i = 0; i < ctx->n; ++i) {
    const int q = (int)std::min<int64_t>(i, ctx->mv);
    const int32_t* r = h.data() + (size_t)i * ctx->mv;
    for (int t = 0; t < ctx->mv; ++t) {
      bool ok = (t < q) ? (r[t] >= 0 && r[t] < i && (t == 0 || r[t] > r[t - 1])) : (r[t] == -1);
      if (!ok) return set_err(ctx, VIF_ERR_ARG, "neighbour table row %lld is not a valid set", (long long)i);
    }
  }
  CK(cudaMemcpyAsync(ctx->N, h.data(), cnt * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->lap_ready) CKS(build_children(ctx));
  CKS(build_groups(ctx, h.data()));
  return VIF_OK;
}

vif_status vif_get_neighbors(const vif_ctx* cctx, int32_t* N) {
  vif_ctx* ctx = const_cast<vif_ctx*>(cctx);
  if (!ctx || !N) return VIF_ERR_ARG;
  if (ctx->mv == 0) return VIF_OK;
  return download(ctx, N, ctx->N, (size_t)ctx->n * ctx->mv * sizeof(int32_t));
}

vif_status vif_get_factors(const vif_ctx* cctx, double* Acoef, double* D) {
  vif_ctx* ctx = const_cast<vif_ctx*>(cctx);
  if (!ctx) return VIF_ERR_ARG;
  if (!ctx->have_factors) return set_err(ctx, VIF_ERR_STATE, "no factors yet: call vif_nll first");
  if (Acoef && ctx->mv > 0) CKS(download(ctx, Acoef, ctx->Acoef, (size_t)ctx->n * ctx->mv * sizeof(double)));
  if (D) CKS(download(ctx, D, ctx->Dv, (size_t)ctx->n * sizeof(double)));
  return VIF_OK;
}

vif_status vif_get_knn_stats(const vif_ctx* ctx, int64_t* n_rescored, int64_t* n_fallback) {
  if (!ctx) return VIF_ERR_ARG;
  if (n_rescored) *n_rescored = ctx->knn_rescored;
  if (n_fallback) *n_fallback = ctx->knn_fallback;
  return VIF_OK;
}

vif_status vif_get_stage_times(const vif_ctx* cctx, double* ms) {
  vif_ctx* ctx = const_cast<vif_ctx*>(cctx);
  if (!ctx || !ms) return VIF_ERR_ARG;
  if (!ctx->timing) return set_err(ctx, VIF_ERR_STATE, "context was built without stage_timing");
  if (!ctx->have_factors) return set_err(ctx, VIF_ERR_STATE, "no vif_nll call yet");
  for (int k = 0; k < VIF_NSTAGES; ++k) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev[k], ctx->ev[k + 1]));
    ms[k] = t;
  }
  return VIF_OK;
}

vif_status vif_get_factor_tuning(const vif_ctx* ctx, int32_t* path, double* ms) {
  if (!ctx || !path) return VIF_ERR_ARG;
  const bool tc = ctx->precision == VIF_MIXED && ctx->ug_ready &&
                  (ctx->factor_mode == 2 || (ctx->factor_mode == 0 && ctx->factor_choice == 1));
  const bool undecided = ctx->precision == VIF_MIXED && ctx->ug_ready && ctx->factor_mode == 0 &&
                         ctx->factor_choice < 0;
  *path = undecided ? 0 : (tc ? 2 : 1);
  if (ms) {
    ms[0] = ctx->factor_ms[0];
    ms[1] = ctx->factor_ms[1];
  }
  return VIF_OK;
}

const char* vif_last_error(const vif_ctx* ctx) { return ctx ? ctx->err : g_build_err; }

void vif_destroy(vif_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

}  // extern "C"
