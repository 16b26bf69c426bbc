// vif_nll_noalloc: the float64 likelihood of vif_nll for callers that cannot
// allocate device memory.  Every intermediate lives in one file-scope static
// device array instead of context buffers obtained from cudaMalloc.
//
// Who needs this: code that runs inside a framework which owns the device's
// memory (its caching allocator has already reserved the free HBM, so a raw
// cudaMalloc fails or fragments the pool), plug-ins whose host forbids device
// allocations after start-up, and latency-critical loops that cannot pay for
// the implicit device-wide synchronisation of cudaMalloc/cudaFree.
//
// The array is part of the library image: every GPU that loads the library
// holds VIF_NOALLOC_SCRATCH_BYTES of it until the process exits.  All calls
// share it and it keeps the last call's contents, so calls that overlap on the
// GPU (several streams or host threads at once) race on it.  Host code cannot
// use the symbol's name as a device address: the first call on each device
// looks the address up with cudaGetSymbolAddress while that device is current,
// so that first call should come before any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "vif_internal.cuh"

using namespace vif;

namespace {

constexpr size_t kScratchBytes = (size_t)VIF_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Carves the scratch array into the buffers of one call (256-byte aligned).
struct Carve {
  uintptr_t base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

struct Layout {
  double *hyp, *Xs, *Zs, *Sm, *Linv, *LinvT, *A, *F, *Acoef, *Dv, *logD, *part, *G, *red, *dscal, *trw;
  int* status;
  size_t bytes;
};

Layout layout(uintptr_t base, int64_t n, int d, int m, int mv, int mpad, int fpad, int nsplit) {
  Carve c{base};
  Layout L;
  const int nt = fpad / 64;
  L.hyp = c.take<double>(32);
  L.Xs = c.take<double>((size_t)n * d);
  L.Zs = c.take<double>((size_t)std::max(m, 1) * d);
  L.Sm = c.take<double>((size_t)mpad * mpad);
  L.Linv = c.take<double>((size_t)mpad * mpad);
  L.LinvT = c.take<double>((size_t)mpad * mpad);
  L.A = c.take<double>((size_t)n * mpad);
  L.F = c.take<double>((size_t)n * fpad);
  L.Acoef = c.take<double>((size_t)n * std::max(mv, 1));
  L.Dv = c.take<double>((size_t)n);
  L.logD = c.take<double>((size_t)n);
  L.part = c.take<double>((size_t)nsplit * (nt * (nt + 1) / 2) * 64 * 64);
  L.G = c.take<double>((size_t)(m + 1) * fpad);
  L.red = c.take<double>(256);
  L.dscal = c.take<double>(16);
  L.trw = c.take<double>(trtri_work_doubles(m + 1));
  L.status = c.take<int>(16);
  L.bytes = c.off;
  return L;
}

vif_status fail(vif_status st, const char* msg) {
  vif_internal_set_global_error(msg);
  return st;
}

#define NA_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      char b_[256];                                                                   \
      snprintf(b_, sizeof(b_), "vif_nll_noalloc: %s: %s", #call, cudaGetErrorString(e_)); \
      return fail(VIF_ERR_CUDA, b_);                                                  \
    }                                                                                 \
  } while (0)

}  // namespace

extern "C" vif_status vif_nll_noalloc(const double* X, int64_t n, int32_t d, const double* Z, int32_t m,
                                      const int32_t* N, int32_t mv, const vif_cov* theta, const double* y,
                                      void* stream, double* nll_out) {
  if (!X || !y || !nll_out || !theta || n < 1 || d < 1 || d > 16 || m < 0 || m > 2048 || mv < 0 || mv > 48 ||
      (m > 0 && !Z) || (mv > 0 && !N))
    return fail(VIF_ERR_ARG, "vif_nll_noalloc: invalid arguments");
  char why[200];
  if (!cov_valid(theta, d, why, sizeof(why))) {
    char b[256];
    snprintf(b, sizeof(b), "vif_nll_noalloc: %s", why);
    return fail(VIF_ERR_ARG, b);
  }
  // the kernels read these arrays directly: a host pointer would become an illegal
  // device access, so anything cudaPointerGetAttributes does not report as device or
  // managed memory is refused before any work is enqueued
  if (!is_device_ptr(X) || !is_device_ptr(y) || (m > 0 && !is_device_ptr(Z)) || (mv > 0 && !is_device_ptr(N)))
    return fail(VIF_ERR_ARG, "vif_nll_noalloc: X, Z, N and y must be device (or managed) pointers");
  const int mpad = std::max(32, ((m + 31) / 32) * 32);
  const int fpad = ((m + 1 + 63) / 64) * 64;
  const int nsplit = gram_nsplit(n, fpad);
  const Layout need = layout(0, n, d, m, mv, mpad, fpad, nsplit);
  if (need.bytes > kScratchBytes) {
    char b[256];
    snprintf(b, sizeof(b), "vif_nll_noalloc: problem needs %zu bytes of scratch, the maximum is %zu",
             need.bytes, kScratchBytes);
    return fail(VIF_ERR_ARG, b);
  }
  void* base = nullptr;
  NA_CK(scratch_address(&base));
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = layout((uintptr_t)base, n, d, m, mv, mpad, fpad, nsplit);

  const CovParams cp = cov_params(theta);
  double h[32];
  for (int t = 0; t < 16; ++t) {
    h[t] = (t < d) ? 1.0 / theta->lengthscale[theta->n_ls == 1 ? 0 : t] : 0.0;
    h[16 + t] = 0.0;   // no centring of the coordinates here
  }
  // only the status words must start at zero; every other buffer is fully written
  NA_CK(cudaMemsetAsync(L.status, 0, 16 * sizeof(int), s));
  NA_CK(cudaMemcpyAsync(L.hyp, h, sizeof(h), cudaMemcpyHostToDevice, s));
  NA_CK(scale_coords(X, n, d, L.hyp, L.hyp + 16, L.Xs, nullptr, s));
  if (m > 0) {
    NA_CK(scale_coords(Z, m, d, L.hyp, L.hyp + 16, L.Zs, nullptr, s));
    NA_CK(build_sigma_m(L.Zs, m, d, cp, L.Sm, mpad, s));
    NA_CK(dense_cholesky(L.Sm, m, mpad, L.status, ST_NOTPD_SIGMAM, s));
    NA_CK(dense_trtri_lower(L.Sm, L.Linv, m, mpad, L.trw, s));
    NA_CK(linv_transpose<double>(L.Linv, m, mpad, L.LinvT, mpad, s));
  }
  NA_CK(lowrank_A<double>(L.Xs, L.Zs, L.LinvT, mpad, L.A, n, d, m, mpad, cp.kind, cp.var, s));
  NA_CK(vecchia_factor<double>(L.A, L.Xs, N, nullptr, y, n, d, m, mpad, mv, fpad, cp, L.F, L.Acoef, L.Dv,
                               L.logD, L.status, s));
  NA_CK(gram_FtF<double>(L.F, n, fpad, m, L.part, nsplit, L.G, fpad, s));
  NA_CK(reduce_sum(L.logD, n, L.red, L.dscal, s));
  NA_CK(dense_cholesky(L.G, m + 1, fpad, L.status, ST_NOTPD_CAP, s));
  NA_CK(nll_finish(L.G, fpad, m, L.dscal, n, L.dscal + 1, s));
  int st[4];
  double val = 0.0;
  NA_CK(cudaMemcpyAsync(st, L.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaMemcpyAsync(&val, L.dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (st[0] != ST_OK) {
    const vif_status e = status_error(st, why, sizeof(why));
    char b[256];
    snprintf(b, sizeof(b), "vif_nll_noalloc: %s", why);
    return fail(e, b);
  }
  *nll_out = val;
  return VIF_OK;
}
