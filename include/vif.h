/*
 * vif.h -- C ABI of libvif, a single-GPU (sm_103a) implementation of the
 * Vecchia-inducing-points full-scale (VIF) Gaussian-process approximation
 * (Gyger, Furrer & Sigrist, "Iterative Methods for Vecchia-Laplace
 * Approximations for Latent Gaussian Process Models" / VIF paper, 2025).
 *
 * Conventions for every entry point
 *   - Array arguments are float64 (or int32 where stated), row-major, owned by
 *     the caller.  A pointer may point to host memory (pageable or pinned) or
 *     to device memory of the context's device; the library detects which with
 *     cudaPointerGetAttributes and copies host data itself on the context's
 *     stream.  Host outputs are complete when the call returns.
 *   - Every call returns a vif_status; nothing is thrown across the ABI.  On an
 *     error the outputs are left untouched (VIF_ERR_NOT_CONVERGED still writes
 *     the last iterate) and vif_last_error() describes it.
 *   - The context owns all its device buffers; no call allocates caller memory.
 *     All work is enqueued on the stream given to vif_build (0 = legacy default).
 *   - Calls on one context must not overlap (a context is not thread-safe).
 *   - The CUDA path is the only path: there is no CPU fallback.  A call on a
 *     machine without a usable GPU returns VIF_ERR_CUDA.
 */
#ifndef VIF_H
#define VIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vif_ctx vif_ctx;

typedef enum {
  VIF_OK = 0,
  VIF_ERR_ARG = 1,            /* invalid argument (sizes, kinds, null pointers) */
  VIF_ERR_CUDA = 2,           /* CUDA runtime error (message in vif_last_error) */
  VIF_ERR_NOMEM = 3,          /* device allocation failed */
  VIF_ERR_NOT_PD = 4,         /* a Cholesky pivot was not positive; index in message */
  VIF_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out */
  VIF_ERR_NOT_CONVERGED = 6,  /* Newton / CG hit its iteration cap */
  VIF_ERR_STATE = 7           /* call out of order (e.g. predict before nll) */
} vif_status;

/* Covariance functions c_theta(s,s') = sigma1^2 k(r), r = ||(s-s')/lambda||
 * (Sec. 2; ARD transform q_lambda(s) = s/lambda of Eq. cov_trans_iso, Sec. 6).
 * Matern forms of Rasmussen & Williams: k_{1/2} = e^{-r},
 * k_{3/2} = (1+sqrt3 r) e^{-sqrt3 r}, k_{5/2} = (1+sqrt5 r+5r^2/3) e^{-sqrt5 r},
 * squared exponential ("Gaussian") k = e^{-r^2/2}. */
typedef enum { VIF_MATERN12 = 0, VIF_MATERN32 = 1, VIF_MATERN52 = 2, VIF_SE = 3 } vif_kernel;

typedef struct {
  int32_t kind;               /* vif_kernel */
  double variance;            /* marginal variance sigma1^2 > 0 */
  const double *lengthscale;  /* HOST array of n_ls length scales lambda > 0 */
  int32_t n_ls;               /* 1 (isotropic) or d (ARD) */
  double nugget;              /* error variance sigma^2 >= 0 (Gaussian likelihood, Eq. cov_mat_gauss);
                                 must be 0 for a latent GP (Laplace, Sec. 3) */
} vif_cov;

typedef enum { VIF_FP64 = 0, VIF_MIXED = 1 } vif_precision;
typedef enum { VIF_GAUSSIAN = 0, VIF_BERNOULLI_LOGIT = 1 } vif_likelihood;

typedef struct {
  int32_t precision;          /* vif_precision: arithmetic of the likelihood path.  VIF_MIXED stores
                                 A and F in float32 and computes the O(n m^2) products in float32;
                                 the Cholesky factors of Sigma_m and of the m x m capacitance matrix
                                 and the log-determinant sums stay float64. */
  int32_t likelihood;         /* vif_likelihood */
  int32_t no_neighbor_search; /* 0: vif_build runs the neighbour search (default); 1: it does not,
                                 and the caller supplies N(i) with vif_set_neighbors before vif_nll */
  int32_t stage_timing;       /* 1: record CUDA events around every stage of vif_nll (read them with
                                 vif_get_stage_times); 0: no events */
  int32_t factor_path;        /* VIF_MIXED only: where the residual products A_N^T A_N of the Vecchia
                                 factors are formed.  1: every point forms its own Gram on the CUDA
                                 cores; 2: on the tensor cores, groups of points sharing one 128-row
                                 Gram (when m >= 1 and m_v + 1 <= 32; else as 1); 0 (default):
                                 autotuned, the first vif_nll times both and keeps the faster
                                 (vif_get_factor_tuning reports the choice).  The choice changes
                                 how the float32 products are summed, not the method. */
  int32_t reserved[3];        /* must be zero */
} vif_opts;

/* vif_build -- fix the data S = {s_i} (X, n x d), the inducing points S* (Z, m x d,
 * Sec. 2.1 Eq. def_b_low), and the residual Vecchia neighbour sets N(i) (Sec. 2.1
 * neighbour rule) chosen with the correlation distance d_c of Sec. 6 under the
 * hyperparameters `cov`:  N(i) = the min(i, m_v) points j < i with the smallest
 * 1 - |rho_ij|, rho_ij = c_r(i,j)/sqrt(c_r(i,i) c_r(j,j)), c_r = Sigma - Sigma^l
 * without nugget, ties broken by lower index.  The search is an exact tiled
 * brute force (float32 filter with a rigorous error bound, float64 decision at
 * the boundary) and returns the same sets as the paper's cover tree (Alg. 3/4).
 *   X: n x d;  Z: m x d (m may be 0: classical Vecchia);  mv >= 0 (0: FITC).
 *   Limits: 1 <= d <= 16, 0 <= m <= 2048, 0 <= mv <= 48, n >= 1.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 *   *out receives the context; free it with vif_destroy. */
vif_status vif_build(const double *X, int64_t n, int32_t d, const double *Z, int32_t m,
                     int32_t mv, const vif_cov *cov, const vif_opts *opts, void *stream,
                     vif_ctx **out);

/* vif_nll -- negative log-likelihood of the VIF approximation (Sec. 2.1-2.2):
 *   L = n/2 log 2pi + 1/2 log det Sigma~_dagger + 1/2 y^T Sigma~_dagger^{-1} y,
 * with log det via Sylvester (det M det Sigma_m^{-1} det D) and the solve via
 * Woodbury (M of Eq. def_M), for the hyperparameters `theta` and the fixed
 * neighbour sets of the context.  y: n responses.  nll_out: HOST double.
 * grad_out: NULL, or a HOST array of n_ls + 2 doubles that receives the analytic gradient
 * of the likelihood (Sec. 2.2 with the derivatives of B and D of App. A) with respect to
 * (sigma1^2, lambda_1..lambda_{n_ls}, sigma^2), with N and Z held fixed, in float64 (a
 * mixed-precision context evaluates it from a float64 pass; its nll_out stays the mixed
 * likelihood).  It is formed in reverse mode, at the cost of about one more likelihood
 * evaluation whatever n_ls; needs nugget > 0, m_v <= 64 and n_ls <= 16. */
vif_status vif_nll(vif_ctx *ctx, const vif_cov *theta, const double *y, double *nll_out,
                   double *grad_out);

/* vif_predict -- predictive means and variances at Xp (np x d) by Prop. 2.1, the
 * variances through the expansion of App. C.1, with prediction points conditioned
 * on their m_v nearest training points by d_c (B_p = I).  Uses theta and y as given
 * (the factors are recomputed for theta).  latent = 1 gives the latent process b^p
 * (variance minus the nugget), 0 the response y^p.  mean, var: np outputs (var may
 * be NULL). */
vif_status vif_predict(vif_ctx *ctx, const vif_cov *theta, const double *y, const double *Xp,
                       int64_t np, int32_t latent, double *mean, double *var);

/* vif_laplace_mode -- mode b~ of the Laplace approximation for a Bernoulli-logit
 * likelihood with the VIF prior on the latent GP (Sec. 3, Eq. LA; VIF-Laplace of
 * Eq. log_det_VIFLA): Newton iterations b <- (W + Sigma_dagger^{-1})^{-1}(W b + grad)
 * (Eq. one_it_newton_mode) from b = 0, each linear system solved by preconditioned CG
 * on Eq. pcls1 with the VIFDU preconditioner P = B^T W B + Sigma_dagger^{-1} (Sec. 4.3,
 * App. E.1).  Needs a context built with likelihood = VIF_BERNOULLI_LOGIT and theta with
 * nugget 0.  CG starts from 0 and stops when ||v - (W + Sigma_dagger^{-1}) x||_2 <= rel_tol
 * ||v||_2 (recursive residual); Newton stops when the objective
 * log p(y|b) - b^T Sigma_dagger^{-1} b / 2 changes by at most 1e-10 relative.
 *   y: n responses in {0,1}.  mode_out: n values (host or device).  stats: host, may be NULL.
 *   precond: 0 = VIFDU; 1 = VIFDU with a learned diagonal correction c (W' = W exp(c),
 *   c from the two-layer network whose weights mlp_weights points to, see vif_mlp_*);
 *   2 = FITC, P = D_V + Sigma_mn^T Sigma_m^{-1} Sigma_mn with D_V = diag(Sigma - Sigma_mn^T
 *   Sigma_m^{-1} Sigma_mn) + W^{-1} (Sec. 4.3, App. E.2; its inducing points are the VIF's), each
 *   Newton system then solved in the form of Eq. pcls2, (W^{-1} + Sigma_dagger)(W b) = Sigma_dagger v,
 *   with the same stopping rule on that system. */
typedef struct {
  double rel_tol;             /* CG tolerance (e.g. 1e-6) */
  int32_t max_pcg;            /* CG iteration cap per Newton step (e.g. 1000) */
  int32_t max_newton;         /* Newton step cap (e.g. 50) */
  int32_t precond;            /* 0 VIFDU (Eq. pcls1), 1 VIFDU with learned diagonal correction,
                                 2 FITC with the VIF's inducing points (App. E.2, Eq. pcls2) */
  int32_t wait_polls;         /* 0: the default bound on every wait of the level-scheduled triangular
                                 solves (well over a second); > 0: give up a wait after this many polls
                                 of a value that is not yet written.  A diagnosis and testing knob: a
                                 small value makes the solves give up, the kernels return, and the call
                                 reports VIF_ERR_TIMEOUT with the context still usable; it applies to
                                 the solves of the Newton iterations.  < 0: VIF_ERR_ARG */
  const void *mlp_weights;    /* device pointer to the packed network weights when precond = 1 */
} vif_laplace_opts;

typedef struct {
  int32_t newton_iters;       /* Newton steps taken */
  int32_t pcg_iters_total;    /* CG iterations summed over the Newton steps */
  double final_rel_res;       /* relative residual of the last CG solve */
  double ms_pcg;              /* device time of the CG solves (CUDA events) */
  double ms_total;            /* device time of the whole call */
  double objective;           /* log p(y|b~) - b~^T Sigma_dagger^{-1} b~ / 2 */
} vif_laplace_stats;

vif_status vif_laplace_mode(vif_ctx *ctx, const vif_cov *theta, const double *y,
                            const vif_laplace_opts *opts, double *mode_out, vif_laplace_stats *stats);

/* vif_laplace_nll -- the VIF-Laplace negative log-marginal likelihood of Eq. log_det_VIFLA,
 *     L = -log p(y | b~) + b~^T Sigma_dagger^{-1} b~ / 2 + log det(Sigma_dagger W + I) / 2,
 * at the mode b~ found as by vif_laplace_mode (same options), with the log-determinant by
 * the preconditioned stochastic Lanczos quadrature of Eq. slq_v1 (Sec. 4.1, App. D):
 *     log det(Sigma_dagger W + I) ~ log det Sigma_dagger + (n / l) sum_i e_1^T log(T_i) e_1 + log det P,
 * P the VIFDU preconditioner at the mode (W' = W exp(c) when opts->precond = 1), log det P
 * in closed form (App. E.1), T_i the Lanczos tridiagonal matrix defined by the coefficients
 * of preconditioned CG on (W + Sigma_dagger^{-1}) x = z_i (from x = 0, stopping at
 * ||z_i - (W + Sigma_dagger^{-1}) x||_2 <= slq_tol ||z_i||_2 or after slq_max_iter steps),
 * and z_i ~ N(0, P) drawn by the recipe of Sec. 4.3 (the probes' CGs run side by side in blocks of up to
 * 64, each with its own coefficients and stopping test, sharing the operator applications),
 *     z_i = B^T W'^{1/2} eps3 + Sigma_dagger^{-1} (B^{-1} D^{1/2} eps2 + Sigma_mn^T L_m^{-T} eps1)
 * (Sigma_m = L_m L_m^T), from the standard normal numbers the caller supplies.
 *   eps: nprobe x (m + 2n) row-major float64 (host or device); row i is (eps1 (m), eps2 (n),
 *        eps3 (n)) of probe i.
 * With opts->precond = 2 (FITC) the estimate is that of Eq. slq_v2,
 *     log det(Sigma_dagger W + I) ~ log det W + (n / l) sum_i e_1^T log(T_i) e_1 + log det P,
 * T_i from CG on (W^{-1} + Sigma_dagger) x = z_i, z_i = D_V^{1/2} eps2 + Sigma_mn^T L_m^{-T} eps1
 * (eps3 unused), log det P = log det D_V + log det(I + L_m^{-1} Sigma_mn D_V^{-1} Sigma_mn^T L_m^{-T}).
 *   nll_out: host scalar.  probe_q, probe_zpz: host arrays of nprobe (may be NULL):
 *        e_1^T log(T_i) e_1 and z_i^T P^{-1} z_i.  stats: host, may be NULL.
 * Errors as vif_laplace_mode; VIF_ERR_NOT_PD if a Lanczos matrix is not positive definite;
 * VIF_ERR_NOT_CONVERGED (outputs still written) if Newton or a CG solve hit its cap. */
typedef struct {
  double nll;                 /* L of Eq. log_det_VIFLA with the estimate of Eq. slq_v1 */
  double neg_log_lik;         /* -log p(y | b~) */
  double quad;                /* b~^T Sigma_dagger^{-1} b~ */
  double logdet_sigma;        /* log det Sigma_dagger = log det C + sum_i log D_i */
  double logdet_precond;      /* log det P: sum_i log(W'_i + 1/D_i) - log det C + log det C_3 (VIFDU), or
                                 log det D_V + log det M_V (FITC) */
  double slq_term;            /* (n / l) sum_i e_1^T log(T_i) e_1 */
  double logdet;              /* estimate of log det(Sigma_dagger W + I) (Eq. slq_v1) */
  double logdet_exact_norm;   /* the same with z_i^T P^{-1} z_i in place of n */
  int32_t newton_iters;       /* Newton steps of the mode search */
  int32_t pcg_iters_mode;     /* CG iterations of the Newton solves */
  int32_t pcg_iters_slq;      /* CG iterations of the probe solves, summed */
  int32_t reserved;
  double ms_mode;             /* device time of the mode search */
  double ms_slq;              /* wall time of the probes (sampling, CG, quadrature) */
} vif_laplace_nll_stats;

vif_status vif_laplace_nll(vif_ctx *ctx, const vif_cov *theta, const double *y, const vif_laplace_opts *opts,
                           int32_t nprobe, const double *eps, double slq_tol, int32_t slq_max_iter,
                           double *nll_out, double *probe_q, double *probe_zpz, vif_laplace_nll_stats *stats);

/* vif_laplace_nll_grad -- vif_laplace_nll (same arguments, same nll_out and stats->nll) and the
 * gradient of L with respect to (sigma1^2, lambda_1..lambda_{n_ls}) by stochastic trace estimation
 * (Sec. 4.1 after Eq. slq_v2; App. B "Gradients"; App. D), in the VIFDU form (opts->precond = 0):
 *     dL/dth_k = b~^T Delta_k b~ / 2 + (dlog det Sigma_dagger/dth_k + T_k) / 2 - v^T Delta_k b~,
 * H = W + Sigma_dagger^{-1}, Delta_k = dSigma_dagger^{-1}/dth_k, the last term being dL/db~ . db~/dth_k
 * with db~/dth_k = -H^{-1} Delta_k b~ and v = H^{-1} dL/db~ (CG on Eq. pcls1 with the mode's rel_tol and
 * max_pcg).  The probes of the likelihood's SLQ are reused: with u_i = H^{-1} z_i (their CG solutions)
 * and y_i = P^{-1} z_i,
 *     dL/db~_j ~ dW_jj/db_j (1/l) sum_i u_ij y_ij / 2,   s_ik = u_i^T Delta_k y_i,
 *     T_k = (1/l) sum_i (s_ik - c_k c_ik) + c_k tau_k   (control variate of App. D),
 *     c_ik = y_i^T (dP/dth_k) y_i,  tau_k = Tr(P^{-1} dP/dth_k) = dlog det P/dth_k,
 *     c_k = sum_i (s_ik - mean_i s_ik)(c_ik - tau_k) / sum_i (c_ik - tau_k)^2  (0 if the sum is 0),
 * P = B^T W B + Sigma_dagger^{-1} (App. E.1).  Derivatives in theta (of the bilinear forms
 * x^T Sigma_dagger^{-1} y and (B y)^T W (B y), of log det Sigma_dagger and of log det P) are central
 * differences with step 1e-4 |th_k|, holding N, Z, the mode b~ and W fixed: the factors are rebuilt
 * twice per parameter, and those of theta are restored before the call returns.
 * FITC form (opts->precond = 2, Eq. pcls2 / slq_v2 and App. D's second form): with H_F = W^{-1} + Sigma_dagger,
 * a = Sigma_dagger^{-1} b~, av = Sigma_dagger^{-1} v and dSigma_k = dSigma_dagger/dth_k,
 *     dL/dth_k = -a^T dSigma_k a / 2 + av^T dSigma_k a + T_k / 2,   s_ik = u_i^T dSigma_k y_i,
 *     dL/db~_j ~ (dW_jj/db_j / W_jj) (1 - (1/l) sum_i u_ij y_ij / W_jj) / 2,
 * u_i = H_F^{-1} z_i, y_i = P^{-1} z_i with the FITC probes and P = D_V + Sigma_mn^T Sigma_m^{-1} Sigma_mn,
 * c_ik = y_i^T (dP/dth_k) y_i, tau_k = dlog det P/dth_k, v = W^{-1} H_F^{-1} Sigma_dagger dL/db~ (CG on
 * Eq. pcls2).
 *   grad_out: host, 1 + n_ls values (required).
 *   probe_terms: host, nprobe x (1 + n_ls) x 2 (s_ik, c_ik), or NULL.
 *   trace_out: host, (1 + n_ls) x 4 (mean_i s_ik, c_k, tau_k, T_k), or NULL.
 *   stats: host, may be NULL.
 * Errors as vif_laplace_nll; VIF_ERR_ARG for precond = 1 (the learned correction). */
typedef struct {
  vif_laplace_nll_stats nll;  /* as vif_laplace_nll */
  int32_t pcg_iters_v;        /* CG iterations of the solve v = H^{-1} dL/db~ */
  int32_t reserved;
  double ms_grad;             /* wall time after the likelihood: the solve for v and the differences */
} vif_laplace_grad_stats;

vif_status vif_laplace_nll_grad(vif_ctx *ctx, const vif_cov *theta, const double *y, const vif_laplace_opts *opts,
                                int32_t nprobe, const double *eps, double slq_tol, int32_t slq_max_iter,
                                double *nll_out, double *grad_out, double *probe_terms, double *trace_out,
                                vif_laplace_grad_stats *stats);

/* vif_laplace_predict -- VIF-Laplace posterior predictive distribution of the latent GP at np
 * new inputs (Prop. 3.1, prediction points conditioning on training points only as in
 * vif_predict), at the mode b~ found as by vif_laplace_mode (opts->precond 0 = VIFDU or 2 = FITC).
 *   mean: omega_p = K_p Sigma_dagger^{-1} b~,  K_p = Sigma_mnp^T Sigma_m^{-1} Sigma_mn - B_po (B^T D^{-1} B)^{-1}.
 *   var (may be NULL): diag(Omega_p) by Alg. 1 (SBPV, variance version): the latent variance of
 *        Prop. 2.1 with b~ for y, plus (1/l) sum_i z8_i o z8_i over nsample draws, where
 *        z4 = Sigma_mn^T L_m^{-T} z3 + B^{-1} D^{1/2} z1, z6 = Sigma_dagger^{-1} z4 + W^{1/2} z2,
 *        z7 = (W + Sigma_dagger^{-1})^{-1} z6 by preconditioned CG (stopping as vif_laplace_mode, with
 *        cg_tol and cg_max_iter; Eq. pcls2 for FITC) and z8 = K_p Sigma_dagger^{-1} z7.
 *   eps: nsample x (m + 2n) row-major float64 standard normal numbers (host or device), row i =
 *        (z3 (m), z1 (n), z2 (n)); unused when var is NULL.
 *   Xp: np x d (host or device); mean, var: np values (host or device).  stats: host, may be NULL
 *        (pcg_iters_total counts the Newton and the SBPV solves).
 * Errors as vif_laplace_mode; VIF_ERR_ARG for precond = 1 or m_v > 48. */
vif_status vif_laplace_predict(vif_ctx *ctx, const vif_cov *theta, const double *y, const vif_laplace_opts *opts,
                               const double *Xp, int64_t np, int32_t nsample, const double *eps, double cg_tol,
                               int32_t cg_max_iter, double *mean, double *var, vif_laplace_stats *stats);

/* vif_tridiag_log_quadrature -- e_1^T log(T) e_1 for a symmetric positive-definite
 * tridiagonal T (diagonal diag[0..k-1], off-diagonal offdiag[0..k-2], host arrays): the
 * Gauss quadrature of App. D, by implicit symmetric QR with Wilkinson shifts on the host
 * (no GPU involved).  VIF_ERR_NOT_PD if T is not positive definite. */
vif_status vif_tridiag_log_quadrature(const double *diag, const double *offdiag, int32_t k, double *out);

/* Learned diagonal correction of the VIFDU preconditioner (the paper has none):
 * c_i = 4 tanh(o_i / 4), o_i from a tanh network 10 -> 64 -> 64 -> 1 on local features
 * of point i, and the preconditioner uses W'_i = W_i exp(c_i).  The network lives in a
 * caller-allocated DEVICE buffer of vif_mlp_bytes() bytes (float32 master weights, Adam
 * moments, the float16 copy the kernels read).  Parameters are packed as W1 (64 x 10,
 * row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1): VIF_MLP_NPARAM floats. */
#define VIF_MLP_NIN 10
#define VIF_MLP_NH 64
#define VIF_MLP_NPARAM (VIF_MLP_NH * VIF_MLP_NIN + VIF_MLP_NH + VIF_MLP_NH * VIF_MLP_NH + VIF_MLP_NH + VIF_MLP_NH + 1)
size_t vif_mlp_bytes(void);
/* Glorot-uniform hidden layers and a zero output layer (c = 0: plain VIFDU). */
vif_status vif_mlp_init(void *net, uint64_t seed, void *stream);
/* Set / read the float32 parameters (params: VIF_MLP_NPARAM floats, host or device). */
vif_status vif_mlp_set_params(void *net, const float *params, void *stream);
vif_status vif_mlp_get_params(const void *net, float *params);
/* c = network(feats) for n feature rows (DEVICE n x 10 float in, DEVICE n float out). */
vif_status vif_mlp_forward(const void *net, const float *feats, int64_t n, float *c, void *stream);
/* grad = d(sum_i gc_i c_i)/d(params) (DEVICE inputs, DEVICE VIF_MLP_NPARAM floats out). */
vif_status vif_mlp_backward(const void *net, const float *feats, const float *gc, int64_t n, float *grad,
                            void *stream);
/* Network inputs of every point for the Laplace weights W (n, host or device), with the
 * residual Vecchia factors of the last vif_laplace_mode / vif_mlp_train call on ctx:
 *   0 (log W_i + 3)/2   1 (log D_i + 3)/2   2 log(1 + W_i D_i)   3 |N(i)|/m_v
 *   4 sum_k A_i[k]^2    5 sum of A_j[k]^2 over the points j that condition on i
 *   6 log(mean_k W_{N_k(i)} / W_i)   7 log(1 + sum_{j: N_k(j)=i} W_j A_j[k]^2 / W_i)
 *   8 max_k |rho(i, N_k(i))|          9 mean_k |rho(i, N_k(i))|
 * with rho the correlation of the residual process (Sec. 2.1: Sigma~ minus the predictive-
 * process part, the jitter on the diagonal) between i and its neighbours, whose largest
 * values chose N(i) (Sec. 6).  feats: n x 10 float (host or device). */
vif_status vif_mlp_features(vif_ctx *ctx, const double *W, float *feats);

typedef struct {
  int32_t steps_per_system;   /* Adam steps at each Newton iterate (each iterate is one system) */
  int32_t probes;             /* Rademacher probes per step */
  int32_t max_newton;         /* Newton iterates used as training systems */
  float lr;                   /* Adam learning rate */
  uint64_t seed;              /* probe generator seed */
} vif_mlp_train_opts;
typedef struct {
  int32_t systems;            /* training systems visited */
  double loss_first, loss_last;  /* probe loss ||P^{-1}Az - z||^2 / n at the first and last step */
} vif_mlp_train_stats;
/* Train the network on the Laplace systems of one problem (ctx built for
 * VIF_BERNOULLI_LOGIT, theta with nugget 0, responses y in {0,1}): Newton iterates of
 * the plain VIFDU solve (CG tolerance 1e-6) are the systems; at each, the network takes
 * steps_per_system Adam steps on the Hutchinson estimate of ||P^{-1} A - I||_F^2. */
vif_status vif_mlp_train(vif_ctx *ctx, const vif_cov *theta, const double *y, const vif_mlp_train_opts *opts,
                         void *net, vif_mlp_train_stats *stats);

/* vif_batch_* -- likelihoods of many independent problems per CUDA graph replay.
 * vif_batch_create captures the likelihood pipeline (vif_nll) of every context into
 * one graph whose problems run on concurrent branches, for fixed hyperparameters
 * thetas[k] and fixed DEVICE response vectors ys[k] (each ctxs[k]->n long; the
 * graph reads them at every replay, so their contents may change between runs).
 * A project autotuner times a few launch shapes (number of concurrent branches, Gram
 * split factor, factor stage per problem or per bucket: vif_batch_set_shape) on the first
 * capture and keeps the fastest.  vif_batch_run replays the
 * graph and writes nprob likelihoods to nll_out (HOST).  The contexts must stay alive
 * and must not be used by other calls while the batch exists.  stream: cudaStream_t
 * the replays are ordered on.  The paper has no batched interface; this is the
 * throughput form of vif_nll for many small problems. */
typedef struct vif_batch vif_batch;
vif_status vif_batch_create(vif_ctx *const *ctxs, int32_t nprob, const vif_cov *thetas,
                            const double *const *ys, void *stream, vif_batch **out);
vif_status vif_batch_run(vif_batch *batch, double *nll_out);
/* launch shape chosen by the autotuner: branches, Gram split divisor, best replay ms */
vif_status vif_batch_info(const vif_batch *batch, int32_t *branches, int32_t *split_div, double *ms);
/* vif_batch_set_shape -- replace the autotuner's choice: recapture the graph with the given
 * number of concurrent branches (1..32), float64 Gram split divisor (>= 1) and factor stage
 * of the bucketed problems (see vif_batch_factor_info): batched_factor = 0 in each problem's
 * branch, 1 one persistent launch per bucket (warps take 32-point chunks from a device
 * counter), 2 one flat launch per bucket (one warp per point, the problems' records in the
 * kernel's parameter bank, 200 problems per launch).  VIF_ERR_ARG for values out
 * of range or batched_factor > 0 with no bucket; the previous graph stays in use on any error. */
vif_status vif_batch_set_shape(vif_batch *batch, int32_t branches, int32_t split_div, int32_t batched_factor);
/* vif_batch_factor_info -- the factor stage's buckets.  A bucket holds the problems of one
 * precision and one neighbour-block size class (m_v + 1 up to 14, 21, 28, 35, 42 or 49) whose
 * factor stage runs on the CUDA cores; one launch can cover all their points.  batched_factor:
 * how the graph in use runs them (the codes of vif_batch_set_shape); nbuckets: buckets built;
 * nbucketed: problems in them.  Any output pointer may be NULL. */
vif_status vif_batch_factor_info(const vif_batch *batch, int32_t *batched_factor, int32_t *nbuckets,
                                 int32_t *nbucketed);
void vif_batch_destroy(vif_batch *batch);

/* vif_set_neighbors / vif_get_neighbors -- replace or read the neighbour table
 * (n x mv int32, row i holds min(i,mv) indices < i in ascending order, padded
 * with -1). */
vif_status vif_set_neighbors(vif_ctx *ctx, const int32_t *N);
vif_status vif_get_neighbors(const vif_ctx *ctx, int32_t *N);

/* vif_get_factors -- the residual Vecchia factors of the last vif_nll call:
 * Acoef (n x mv, row i = A_i on N(i), zero padded; B_{i,N(i)} = -A_i) and D (n),
 * Eq. D_A_Vecchia.  Either pointer may be NULL. */
vif_status vif_get_factors(const vif_ctx *ctx, double *Acoef, double *D);

/* vif_get_stats -- counters of the last neighbour search: number of queries whose
 * float32 filter result needed a float64 rescore at the boundary, and number that
 * fell back to a float64 brute-force scan. */
vif_status vif_get_knn_stats(const vif_ctx *ctx, int64_t *n_rescored, int64_t *n_fallback);

/* vif_get_stage_times -- device time (ms, CUDA events on the context's stream) of
 * the stages of the last vif_nll call of a context built with stage_timing = 1:
 *   [0] Sigma_m, its Cholesky factor and inverse            [1] A = L_m^{-1} Sigma_mn
 *   [2] residual Vecchia factors and rows of [F z]          [3] Gram [F z]^T [F z]
 *   [4] capacitance Cholesky and the scalar likelihood
 * ms: host array of at least VIF_NSTAGES doubles. */
#define VIF_NSTAGES 5
vif_status vif_get_stage_times(const vif_ctx *ctx, double *ms);

/* vif_nll_noalloc -- the float64 negative log-likelihood of vif_nll (same value,
 * same neighbour-table format), for callers that cannot allocate device memory:
 * code inside a framework that owns the GPU's memory (its caching allocator has
 * already reserved the free HBM, so a raw cudaMalloc fails or fragments it),
 * plug-ins whose host forbids device allocations after start-up, and
 * latency-critical loops that cannot pay for the device-wide synchronisation of
 * cudaMalloc/cudaFree.  It needs no context and calls no allocating routine.
 * The paper has no counterpart to this entry point; it is an interface addition.
 *   X (n x d), Z (m x d), N (n x mv int32, rows as for vif_set_neighbors), y (n):
 *   DEVICE (or managed) pointers, checked with cudaPointerGetAttributes: any other
 *   pointer is refused with VIF_ERR_ARG before work is enqueued.  The element types
 *   (float64, int32) cannot be checked from a pointer and are the caller's duty.
 *   theta: as for vif_nll, with the same checks (VIF_ERR_ARG for non-finite or
 *   non-positive values).  stream: cudaStream_t (NULL = legacy default).
 *   nll_out: HOST double, written when the call returns VIF_OK.  Errors map as for
 *   vif_nll (VIF_ERR_NOT_PD, VIF_ERR_STATE for an invalid neighbour table,
 *   VIF_ERR_TIMEOUT for a device wait that gave up).
 * All intermediates live in one static device array of VIF_NOALLOC_SCRATCH_BYTES
 * inside the library; every GPU that loads the library holds that memory until
 * the process exits.  A problem whose intermediates do not fit (roughly
 * n (m_pad + f_pad + m_v + d + 2) * 8 bytes, m_pad = m rounded up to 32, f_pad = m+1
 * rounded up to 64) is rejected with VIF_ERR_ARG and a message in
 * vif_last_error(NULL).  The first call on a device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture.  All calls share the array, which keeps the last call's contents:
 * calls that overlap on the GPU (several streams or threads at once) race on it. */
#define VIF_NOALLOC_SCRATCH_BYTES (32u << 20)
vif_status vif_nll_noalloc(const double *X, int64_t n, int32_t d, const double *Z, int32_t m,
                           const int32_t *N, int32_t mv, const vif_cov *theta, const double *y,
                           void *stream, double *nll_out);

/* vif_get_factor_tuning -- the float32 factor stage's path and the autotuner's timings:
 * *path = 1 (CUDA cores) or 2 (tensor cores) as used by vif_nll now, 0 while not yet tuned;
 * ms[0], ms[1] (host, nullable): the CUDA-core and tensor-core times of the tuning run (0 if
 * not timed).  VIF_ERR_ARG for a NULL context or path. */
vif_status vif_get_factor_tuning(const vif_ctx *ctx, int32_t *path, double *ms);

/* vif_last_error -- text of the last error on this context ("" if none), valid
 * until the next call on the context; with ctx == NULL, the message of the last
 * failed vif_build in this process. */
const char *vif_last_error(const vif_ctx *ctx);

/* vif_destroy -- free the context and its device buffers (NULL is ignored). */
void vif_destroy(vif_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VIF_H */
