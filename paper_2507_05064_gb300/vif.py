"""Thin ctypes binding of libvif (include/vif.h): argument marshalling only.

Arrays may be numpy arrays (host) or torch CUDA tensors (device); the library
detects which.  Every computation runs in the CUDA library; if libvif.so is
missing this module raises on import of the library, it never falls back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvif.so")

VIF_OK, VIF_ERR_ARG, VIF_ERR_CUDA, VIF_ERR_NOMEM, VIF_ERR_NOT_PD, VIF_ERR_TIMEOUT, \
    VIF_ERR_NOT_CONVERGED, VIF_ERR_STATE = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_NOMEM", "ERR_NOT_PD", "ERR_TIMEOUT",
                "ERR_NOT_CONVERGED", "ERR_STATE"]
FP64, MIXED = 0, 1
PRECOND_VIFDU, PRECOND_VIFDU_LEARNED, PRECOND_FITC = 0, 1, 2
GAUSSIAN, BERNOULLI_LOGIT = 0, 1

# every symbol include/vif.h declares
EXPORTS = ["vif_build", "vif_nll", "vif_predict", "vif_laplace_mode", "vif_laplace_nll", "vif_laplace_nll_grad",
           "vif_laplace_predict",
           "vif_tridiag_log_quadrature", "vif_batch_create", "vif_batch_run",
           "vif_batch_info", "vif_batch_set_shape", "vif_batch_factor_info", "vif_batch_destroy", "vif_mlp_bytes", "vif_mlp_init", "vif_mlp_set_params",
           "vif_mlp_get_params", "vif_mlp_forward", "vif_mlp_backward", "vif_mlp_features", "vif_mlp_train", "vif_set_neighbors", "vif_get_neighbors",
           "vif_get_factors", "vif_get_knn_stats", "vif_get_stage_times", "vif_get_factor_tuning", "vif_nll_noalloc",
           "vif_last_error", "vif_destroy"]
NOALLOC_SCRATCH_BYTES = 32 << 20


class VifCov(C.Structure):
    _fields_ = [("kind", C.c_int32), ("variance", C.c_double), ("lengthscale", C.POINTER(C.c_double)),
                ("n_ls", C.c_int32), ("nugget", C.c_double)]


class VifOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("likelihood", C.c_int32), ("no_neighbor_search", C.c_int32),
                ("stage_timing", C.c_int32), ("factor_path", C.c_int32), ("reserved", C.c_int32 * 3)]


class LaplaceOpts(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("max_pcg", C.c_int32), ("max_newton", C.c_int32),
                ("precond", C.c_int32), ("wait_polls", C.c_int32), ("mlp_weights", C.c_void_p)]


class LaplaceNllStats(C.Structure):
    _fields_ = [("nll", C.c_double), ("neg_log_lik", C.c_double), ("quad", C.c_double),
                ("logdet_sigma", C.c_double), ("logdet_precond", C.c_double), ("slq_term", C.c_double),
                ("logdet", C.c_double), ("logdet_exact_norm", C.c_double), ("newton_iters", C.c_int32),
                ("pcg_iters_mode", C.c_int32), ("pcg_iters_slq", C.c_int32), ("reserved", C.c_int32),
                ("ms_mode", C.c_double), ("ms_slq", C.c_double)]


class LaplaceGradStats(C.Structure):
    _fields_ = [("nll", LaplaceNllStats), ("pcg_iters_v", C.c_int32), ("reserved", C.c_int32),
                ("ms_grad", C.c_double)]


class LaplaceStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("pcg_iters_total", C.c_int32), ("final_rel_res", C.c_double),
                ("ms_pcg", C.c_double), ("ms_total", C.c_double), ("objective", C.c_double)]


class MlpTrainOpts(C.Structure):
    _fields_ = [("steps_per_system", C.c_int32), ("probes", C.c_int32), ("max_newton", C.c_int32),
                ("lr", C.c_float), ("seed", C.c_uint64)]


class MlpTrainStats(C.Structure):
    _fields_ = [("systems", C.c_int32), ("loss_first", C.c_double), ("loss_last", C.c_double)]


MLP_NIN, MLP_NH = 10, 64
MLP_NPARAM = MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1
NSTAGES = 5
STAGES = ["sigma_m_chol_inv", "lowrank_A", "vecchia_factor", "gram_FtF", "capacitance_nll"]


class VifError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libvif.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvif.so not found at {LIB_PATH}: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
        L.vif_build.argtypes = [vp, i64, i32, vp, i32, i32, C.POINTER(VifCov), C.POINTER(VifOpts), vp,
                                C.POINTER(vp)]
        L.vif_nll.argtypes = [vp, C.POINTER(VifCov), vp, dp, dp]
        L.vif_predict.argtypes = [vp, C.POINTER(VifCov), vp, vp, i64, i32, vp, vp]
        L.vif_laplace_mode.argtypes = [vp, C.POINTER(VifCov), vp, C.POINTER(LaplaceOpts), vp,
                                       C.POINTER(LaplaceStats)]
        L.vif_laplace_nll.argtypes = [vp, C.POINTER(VifCov), vp, C.POINTER(LaplaceOpts), i32, vp, C.c_double,
                                      i32, dp, vp, vp, C.POINTER(LaplaceNllStats)]
        L.vif_laplace_nll_grad.argtypes = [vp, C.POINTER(VifCov), vp, C.POINTER(LaplaceOpts), i32, vp, C.c_double,
                                           i32, dp, vp, vp, vp, C.POINTER(LaplaceGradStats)]
        L.vif_tridiag_log_quadrature.argtypes = [vp, vp, i32, dp]
        L.vif_laplace_predict.argtypes = [vp, C.POINTER(VifCov), vp, C.POINTER(LaplaceOpts), vp, i64, i32, vp,
                                          C.c_double, i32, vp, vp, C.POINTER(LaplaceStats)]
        L.vif_set_neighbors.argtypes = [vp, vp]
        L.vif_get_neighbors.argtypes = [vp, vp]
        L.vif_get_factors.argtypes = [vp, vp, vp]
        L.vif_get_knn_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
        L.vif_get_stage_times.argtypes = [vp, dp]
        L.vif_get_factor_tuning.argtypes = [vp, C.POINTER(i32), dp]
        L.vif_nll_noalloc.argtypes = [vp, i64, i32, vp, i32, vp, i32, C.POINTER(VifCov), vp, vp, dp]
        L.vif_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(VifCov), C.POINTER(vp), vp, C.POINTER(vp)]
        L.vif_batch_run.argtypes = [vp, dp]
        L.vif_batch_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), dp]
        L.vif_batch_set_shape.argtypes = [vp, i32, i32, i32]
        L.vif_batch_factor_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.vif_batch_destroy.argtypes = [vp]
        L.vif_batch_destroy.restype = None
        L.vif_mlp_bytes.argtypes = []
        L.vif_mlp_bytes.restype = C.c_size_t
        L.vif_mlp_init.argtypes = [vp, C.c_uint64, vp]
        L.vif_mlp_set_params.argtypes = [vp, vp, vp]
        L.vif_mlp_get_params.argtypes = [vp, vp]
        L.vif_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        L.vif_mlp_backward.argtypes = [vp, vp, vp, i64, vp, vp]
        L.vif_mlp_features.argtypes = [vp, vp, vp]
        L.vif_mlp_train.argtypes = [vp, C.POINTER(VifCov), vp, C.POINTER(MlpTrainOpts), vp,
                                    C.POINTER(MlpTrainStats)]
        L.vif_last_error.argtypes = [vp]
        L.vif_last_error.restype = C.c_char_p
        L.vif_destroy.argtypes = [vp]
        L.vif_destroy.restype = None
        for name in EXPORTS:
            if name not in ("vif_last_error", "vif_destroy", "vif_batch_destroy", "vif_mlp_bytes"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    """Pointer of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _f64(a):
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float64 and a.is_contiguous()
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def make_cov(theta) -> tuple[VifCov, np.ndarray]:
    ls = np.ascontiguousarray(np.atleast_1d(np.asarray(theta.lengthscale, dtype=np.float64)))
    cv = VifCov(int(theta.kind), float(theta.variance), ls.ctypes.data_as(C.POINTER(C.c_double)),
                int(ls.size), float(theta.nugget))
    return cv, ls


def nll_noalloc(X, Z, N, mv: int, theta, y, stream: int = 0) -> float:
    """vif_nll_noalloc: the float64 likelihood without any device allocation.
    X (n, d) and Z (m, d) float64, N (n, mv) int32 and y (n,) float64 must be contiguous
    CUDA tensors; see include/vif.h for who needs this.  Anything else raises
    VifError(VIF_ERR_ARG) before the library is called."""
    L = lib()
    n = int(X.shape[0]) if getattr(X, "ndim", 0) == 2 else -1
    d = int(X.shape[1]) if n >= 0 else -1
    m = 0 if Z is None else int(Z.shape[0])
    _check_device(X, "float64", (n, d), "X")
    _check_device(y, "float64", (n,), "y")
    if m:
        _check_device(Z, "float64", (m, d), "Z")
    if mv:
        _check_device(N, "int32", (n, int(mv)), "N")
    cv, ls = make_cov(theta)
    out = C.c_double()
    st = L.vif_nll_noalloc(_ptr(X), n, d, _ptr(Z) if m else None, m, _ptr(N) if mv else None, int(mv),
                           C.byref(cv), _ptr(y), C.c_void_p(stream), C.byref(out))
    if st != VIF_OK:
        raise VifError(st, L.vif_last_error(None).decode())
    return out.value


def _check_device(t, dtype: str, shape, name: str) -> None:
    """A contiguous CUDA tensor of the given dtype and shape, else VifError(VIF_ERR_ARG)."""
    ok = (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch." + dtype
          and tuple(t.shape) == tuple(shape))
    if not ok:
        desc = (f"{type(t).__name__} {getattr(t, 'dtype', None)} {tuple(getattr(t, 'shape', ()))}"
                f"{' on ' + str(t.device) if hasattr(t, 'device') else ''}")
        raise VifError(VIF_ERR_ARG, f"{name} must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}, "
                                    f"got {desc}")


class Network:
    """The learned correction's network in a device buffer (vif_mlp_*); needs torch."""

    def __init__(self, seed: int = 0, params=None):
        import torch
        L = lib()
        self.buf = torch.zeros(int(L.vif_mlp_bytes()), dtype=torch.uint8, device="cuda")
        if params is None:
            st = L.vif_mlp_init(_ptr(self.buf), int(seed), None)
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            st = L.vif_mlp_set_params(_ptr(self.buf), _ptr(p), None)
        if st != VIF_OK:
            raise VifError(st, "network initialisation failed")

    def params(self) -> np.ndarray:
        out = np.empty(MLP_NPARAM, dtype=np.float32)
        if lib().vif_mlp_get_params(_ptr(self.buf), _ptr(out)) != VIF_OK:
            raise VifError(VIF_ERR_CUDA, "reading the parameters failed")
        return out

    def forward(self, feats):
        import torch
        F = torch.as_tensor(np.ascontiguousarray(feats, dtype=np.float32)).cuda()
        c = torch.empty(F.shape[0], dtype=torch.float32, device="cuda")
        if lib().vif_mlp_forward(_ptr(self.buf), _ptr(F), F.shape[0], _ptr(c), None) != VIF_OK:
            raise VifError(VIF_ERR_CUDA, "forward failed")
        return c.cpu().numpy()

    def backward(self, feats, gc):
        import torch
        F = torch.as_tensor(np.ascontiguousarray(feats, dtype=np.float32)).cuda()
        g = torch.as_tensor(np.ascontiguousarray(gc, dtype=np.float32)).cuda()
        out = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
        if lib().vif_mlp_backward(_ptr(self.buf), _ptr(F), _ptr(g), F.shape[0], _ptr(out), None) != VIF_OK:
            raise VifError(VIF_ERR_CUDA, "backward failed")
        return out.cpu().numpy()


class Batch:
    """Likelihoods of many contexts per CUDA graph replay (vif_batch_*)."""

    def __init__(self, contexts, thetas, ys, stream: int = 0):
        L = lib()
        n = len(contexts)
        self._covs = [make_cov(t) for t in thetas]
        arr = (VifCov * n)(*[c for c, _ in self._covs])
        hs = (C.c_void_p * n)(*[c.h for c in contexts])
        yp = (C.c_void_p * n)(*[_ptr(y).value for y in ys])
        h = C.c_void_p()
        st = L.vif_batch_create(hs, n, arr, yp, C.c_void_p(stream), C.byref(h))
        if st != VIF_OK:
            raise VifError(st, L.vif_last_error(None).decode())
        self.h, self.n, self._keep = h, n, (contexts, ys)

    def run(self) -> np.ndarray:
        out = np.empty(self.n)
        st = lib().vif_batch_run(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
        if st != VIF_OK:
            raise VifError(st, lib().vif_last_error(None).decode())
        return out

    def info(self):
        b, sd, ms = C.c_int32(), C.c_int32(), C.c_double()
        lib().vif_batch_info(self.h, C.byref(b), C.byref(sd), C.byref(ms))
        bf, nb, nbk = C.c_int32(), C.c_int32(), C.c_int32()
        lib().vif_batch_factor_info(self.h, C.byref(bf), C.byref(nb), C.byref(nbk))
        return {"branches": b.value, "split_div": sd.value, "best_replay_ms": ms.value,
                "batched_factor": bf.value, "factor_buckets": nb.value, "bucketed_problems": nbk.value}

    def set_shape(self, branches: int, split_div: int = 1, batched_factor: int = 0):
        st = lib().vif_batch_set_shape(self.h, branches, split_div, int(batched_factor))
        if st != VIF_OK:
            raise VifError(st, "vif_batch_set_shape failed")

    def close(self):
        if getattr(self, "h", None):
            lib().vif_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tridiag_log_quadrature(diag, offdiag) -> float:
    """e_1^T log(T) e_1 of a symmetric tridiagonal T (host computation in the library)."""
    d = np.ascontiguousarray(diag, dtype=np.float64)
    e = np.ascontiguousarray(offdiag, dtype=np.float64)
    out = C.c_double()
    st = lib().vif_tridiag_log_quadrature(_ptr(d), _ptr(e) if e.size else None, int(d.size), C.byref(out))
    if st != VIF_OK:
        raise VifError(st, "vif_tridiag_log_quadrature")
    return out.value


class Context:
    """One built VIF problem: data, inducing points and neighbour sets (vif_build)."""

    def __init__(self, X, Z, mv: int, theta, precision: int = FP64, likelihood: int = GAUSSIAN,
                 stream: int = 0, neighbor_search: bool = True, stage_timing: bool = False,
                 factor_path: int = 0):
        L = lib()
        X = _f64(X)
        Z = _f64(Z) if Z is not None and Z.shape[0] > 0 else None
        self.n, self.d = int(X.shape[0]), int(X.shape[1])
        self.m = 0 if Z is None else int(Z.shape[0])
        self.mv = int(mv)
        self.precision = precision
        cv, ls = make_cov(theta)
        opts = VifOpts(precision, likelihood, 0 if neighbor_search else 1, 1 if stage_timing else 0,
                       int(factor_path), (C.c_int32 * 3)())
        h = C.c_void_p()
        st = L.vif_build(_ptr(X), self.n, self.d, _ptr(Z), self.m, self.mv, C.byref(cv), C.byref(opts),
                         C.c_void_p(stream), C.byref(h))
        if st != VIF_OK:
            raise VifError(st, L.vif_last_error(None).decode())
        self.h = h
        self._keep = (X, Z)

    def _check(self, st):
        if st != VIF_OK:
            raise VifError(st, lib().vif_last_error(self.h).decode())

    def nll(self, theta, y, grad: bool = False):
        """NLL, or (NLL, gradient wrt (sigma1^2, lambda..., sigma^2)) when grad=True."""
        cv, ls = make_cov(theta)
        out = C.c_double()
        y = _f64(y)
        g = np.empty(ls.size + 2) if grad else None
        gp = g.ctypes.data_as(C.POINTER(C.c_double)) if grad else None
        self._check(lib().vif_nll(self.h, C.byref(cv), _ptr(y), C.byref(out), gp))
        return (out.value, g) if grad else out.value

    def predict(self, theta, y, Xp, latent: bool = False):
        cv, ls = make_cov(theta)
        Xp = _f64(Xp)
        npred = int(Xp.shape[0])
        mean = np.empty(npred)
        var = np.empty(npred)
        self._check(lib().vif_predict(self.h, C.byref(cv), _ptr(_f64(y)), _ptr(Xp), npred, int(latent),
                                      _ptr(mean), _ptr(var)))
        return mean, var

    def laplace_mode(self, theta, y, rel_tol=1e-6, max_pcg=1000, max_newton=50, precond=0,
                     mlp_weights=None, allow_not_converged=False, wait_polls=0):
        """Laplace mode for Bernoulli-logit responses y; returns (mode, stats dict).
        wait_polls > 0 bounds every wait of the triangular solves (see include/vif.h)."""
        cv, ls = make_cov(theta)
        wp = None if mlp_weights is None else _ptr(getattr(mlp_weights, "buf", mlp_weights)).value
        opts = LaplaceOpts(float(rel_tol), int(max_pcg), int(max_newton), int(precond), int(wait_polls), wp)
        st = LaplaceStats()
        mode = np.empty(self.n)
        rc = lib().vif_laplace_mode(self.h, C.byref(cv), _ptr(_f64(y)), C.byref(opts), _ptr(mode), C.byref(st))
        if not (rc == VIF_OK or (allow_not_converged and rc == VIF_ERR_NOT_CONVERGED)):
            self._check(rc)
        stats = {k: getattr(st, k) for k, _ in LaplaceStats._fields_}
        stats["status"] = rc
        return mode, stats

    def laplace_nll(self, theta, y, eps, slq_tol=1e-2, slq_max_iter=1000, rel_tol=1e-6, max_pcg=1000,
                    max_newton=50, precond=0, mlp_weights=None, allow_not_converged=False):
        """VIF-Laplace NLL (Eq. log_det_VIFLA) with the SLQ log-determinant of Eq. slq_v1;
        eps: (nprobe, m + 2n) standard normal numbers (host or device).  Returns
        (nll, stats dict with per-probe 'q' and 'zPz')."""
        cv, ls = make_cov(theta)
        wp = None if mlp_weights is None else _ptr(getattr(mlp_weights, "buf", mlp_weights)).value
        opts = LaplaceOpts(float(rel_tol), int(max_pcg), int(max_newton), int(precond), 0, wp)
        e = _f64(eps)
        nprobe = int(e.shape[0])
        q = np.zeros(nprobe)
        zpz = np.zeros(nprobe)
        out = C.c_double()
        st = LaplaceNllStats()
        rc = lib().vif_laplace_nll(self.h, C.byref(cv), _ptr(_f64(y)), C.byref(opts), nprobe, _ptr(e),
                                   float(slq_tol), int(slq_max_iter), C.byref(out), _ptr(q), _ptr(zpz),
                                   C.byref(st))
        if not (rc == VIF_OK or (allow_not_converged and rc == VIF_ERR_NOT_CONVERGED)):
            self._check(rc)
        stats = {k: getattr(st, k) for k, _ in LaplaceNllStats._fields_}
        stats["q"], stats["zPz"], stats["status"] = q, zpz, rc
        return out.value, stats

    def laplace_nll_grad(self, theta, y, eps, slq_tol=1e-2, slq_max_iter=1000, rel_tol=1e-6, max_pcg=1000,
                         max_newton=50, precond=0, allow_not_converged=False):
        """VIF-Laplace NLL (as laplace_nll; precond 0 = VIFDU, 2 = FITC) and its gradient in
        (sigma1^2, lambda...) by stochastic trace estimation with the preconditioner control variate
        (Sec. 4.1, App. B, App. D).
        Returns (nll, grad, stats dict with 'probe_terms' (nprobe, q, 2) = (s_ik, c_ik) and 'trace'
        (q, 4) = (plain mean, c_k, tau_k, T_k))."""
        cv, ls = make_cov(theta)
        opts = LaplaceOpts(float(rel_tol), int(max_pcg), int(max_newton), int(precond), 0, None)
        e = _f64(eps)
        nprobe = int(e.shape[0])
        q = 1 + int(cv.n_ls)
        grad = np.zeros(q)
        terms = np.zeros((nprobe, q, 2))
        trace = np.zeros((q, 4))
        out = C.c_double()
        st = LaplaceGradStats()
        rc = lib().vif_laplace_nll_grad(self.h, C.byref(cv), _ptr(_f64(y)), C.byref(opts), nprobe, _ptr(e),
                                        float(slq_tol), int(slq_max_iter), C.byref(out), _ptr(grad), _ptr(terms),
                                        _ptr(trace), C.byref(st))
        if not (rc == VIF_OK or (allow_not_converged and rc == VIF_ERR_NOT_CONVERGED)):
            self._check(rc)
        stats = {k: getattr(st.nll, k) for k, _ in LaplaceNllStats._fields_}
        stats.update(pcg_iters_v=st.pcg_iters_v, ms_grad=st.ms_grad, probe_terms=terms, trace=trace, status=rc)
        return out.value, grad, stats

    def laplace_predict(self, theta, y, Xp, eps=None, cg_tol=1e-6, cg_max_iter=1000, rel_tol=1e-6,
                        max_pcg=1000, max_newton=50, precond=0, allow_not_converged=False):
        """Latent predictive means (Prop. 3.1) and, with eps (nsample x (m + 2n) normals),
        variances by Alg. 1 (SBPV).  Returns (mean, var or None, stats)."""
        cv, ls = make_cov(theta)
        opts = LaplaceOpts(float(rel_tol), int(max_pcg), int(max_newton), int(precond), 0, None)
        Xp = _f64(Xp)
        npred = int(Xp.shape[0])
        mean = np.empty(npred)
        var = np.empty(npred) if eps is not None else None
        e = _f64(eps) if eps is not None else None
        st = LaplaceStats()
        rc = lib().vif_laplace_predict(self.h, C.byref(cv), _ptr(_f64(y)), C.byref(opts), _ptr(Xp), npred,
                                       int(e.shape[0]) if e is not None else 0, _ptr(e), float(cg_tol),
                                       int(cg_max_iter), _ptr(mean), _ptr(var), C.byref(st))
        if not (rc == VIF_OK or (allow_not_converged and rc == VIF_ERR_NOT_CONVERGED)):
            self._check(rc)
        stats = {k: getattr(st, k) for k, _ in LaplaceStats._fields_}
        stats["status"] = rc
        return mean, var, stats

    def mlp_features(self, W) -> np.ndarray:
        F = np.empty((self.n, MLP_NIN), dtype=np.float32)
        self._check(lib().vif_mlp_features(self.h, _ptr(_f64(W)), _ptr(F)))
        return F

    def mlp_train(self, theta, y, net, steps_per_system=10, probes=8, max_newton=4, lr=1e-3, seed=1):
        cv, ls = make_cov(theta)
        o = MlpTrainOpts(int(steps_per_system), int(probes), int(max_newton), float(lr), int(seed))
        st = MlpTrainStats()
        self._check(lib().vif_mlp_train(self.h, C.byref(cv), _ptr(_f64(y)), C.byref(o), _ptr(net.buf),
                                        C.byref(st)))
        return {"systems": st.systems, "loss_first": st.loss_first, "loss_last": st.loss_last}

    def neighbors(self) -> np.ndarray:
        N = np.empty((self.n, max(self.mv, 0)), dtype=np.int32)
        if self.mv:
            self._check(lib().vif_get_neighbors(self.h, _ptr(N)))
        return N

    def set_neighbors(self, N) -> None:
        N = np.ascontiguousarray(N, dtype=np.int32)
        assert N.shape == (self.n, self.mv)
        self._check(lib().vif_set_neighbors(self.h, _ptr(N)))

    def factors(self):
        Ac = np.zeros((self.n, self.mv))
        D = np.empty(self.n)
        self._check(lib().vif_get_factors(self.h, _ptr(Ac) if self.mv else None, _ptr(D)))
        return Ac, D

    def knn_stats(self):
        a, b = C.c_int64(), C.c_int64()
        self._check(lib().vif_get_knn_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def factor_tuning(self) -> dict:
        """The float32 factor stage's path (1 CUDA cores, 2 tensor cores, 0 not yet tuned)
        and the autotuner's timings in ms."""
        p = C.c_int32()
        ms = (C.c_double * 2)()
        self._check(lib().vif_get_factor_tuning(self.h, C.byref(p), ms))
        return {"path": p.value, "ms_cuda_cores": ms[0], "ms_tensor_cores": ms[1]}

    def stage_times(self) -> dict:
        ms = (C.c_double * NSTAGES)()
        self._check(lib().vif_get_stage_times(self.h, ms))
        return dict(zip(STAGES, list(ms)))

    def close(self):
        if getattr(self, "h", None):
            lib().vif_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
