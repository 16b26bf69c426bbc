// Learned diagonal correction of the VIFDU preconditioner (not part of the paper).
//
// A two-layer tanh network maps 10 local features of point i (Laplace weight W_i,
// residual variance D_i, the Vecchia coefficients that touch i, the largest and mean
// residual correlation with its neighbours) to c_i =
// 4 tanh(o_i / 4); the preconditioner then uses W'_i = W_i exp(c_i) in
// P = B^T W' B + Sigma_dagger^{-1} (the CG system keeps W).  c = 0 is the plain
// VIFDU preconditioner, and a zero output layer gives exactly that, so an
// untrained network falls back to the method without it.
//
// Training minimises the Hutchinson estimate of ||P^{-1} A - I||_F^2 with
// A = W + Sigma_dagger^{-1}: for Rademacher probes z, u = P^{-1} A z, r = u - z,
//   dL/dd_j = -2 (B P^{-1} r)_j (B u)_j,   dL/dc_j = dL/dd_j * d_j,  d = W',
// back-propagated through the network and applied with Adam.  Weights are kept
// as float32 master copies plus the float16 copy the kernels read; all network
// arithmetic accumulates in float32.
#include <cuda_fp16.h>

#include "vif_internal.cuh"

namespace vif {

constexpr int NIN = VIF_MLP_NIN, NH = VIF_MLP_NH;
constexpr int NP = VIF_MLP_NPARAM;
constexpr int NPP = (NP + 63) / 64 * 64;
// offsets (floats) of the packed parameters
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;

struct NetView {
  float* master;
  float* m;
  float* v;
  float* step;
  __half* w16;
};
__host__ __device__ inline NetView net_view(void* p) {
  float* f = reinterpret_cast<float*>(p);
  NetView nv;
  nv.master = f;
  nv.m = f + NPP;
  nv.v = f + 2 * NPP;
  nv.step = f + 3 * NPP;
  nv.w16 = reinterpret_cast<__half*>(f + 3 * NPP + 64);
  return nv;
}
size_t mlp_bytes() { return (size_t)(3 * NPP + 64) * sizeof(float) + (size_t)NPP * sizeof(__half); }

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void mlp_init_kernel(void* net, uint64_t seed) {
  NetView nv = net_view(net);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPP; k += gridDim.x * blockDim.x) {
    float w = 0.f;
    double u = (double)(splitmix64(seed * 0x100000001B3ull + (uint64_t)k) >> 11) * (1.0 / 9007199254740992.0);
    if (k >= OW1 && k < OB1) w = (float)((2.0 * u - 1.0) * sqrt(6.0 / (NIN + NH)));
    if (k >= OW2 && k < OB2) w = (float)((2.0 * u - 1.0) * sqrt(6.0 / (2 * NH)));
    if (k >= NP) w = 0.f;
    nv.master[k] = w;
    nv.m[k] = 0.f;
    nv.v[k] = 0.f;
    nv.w16[k] = __float2half_rn(w);
  }
  if (blockIdx.x == 0 && threadIdx.x < 64) nv.step[threadIdx.x] = 0.f;
}

// master := given float32 parameters; the float16 copy follows; Adam state reset.
__global__ void mlp_set_kernel(void* net, const float* p) {
  NetView nv = net_view(net);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPP; k += gridDim.x * blockDim.x) {
    float w = (k < NP) ? p[k] : 0.f;
    nv.master[k] = w;
    nv.m[k] = 0.f;
    nv.v[k] = 0.f;
    nv.w16[k] = __float2half_rn(w);
  }
  if (blockIdx.x == 0 && threadIdx.x < 64) nv.step[threadIdx.x] = 0.f;
}

// ---------------------------------------------------------------------------
// Features (10 per point, fixed affine normalisation)
// ---------------------------------------------------------------------------
__global__ void mlp_features_kernel(const double* __restrict__ W, const double* __restrict__ D,
                                    const double* __restrict__ Acoef, const float* __restrict__ rho,
                                    const int32_t* __restrict__ N,
                                    const int32_t* __restrict__ ch_ptr, const int32_t* __restrict__ ch_row,
                                    const int32_t* __restrict__ ch_slot, int64_t n, int mv, float* F) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double wi = W[i], di = D[i];
  const int q = (int)(i < mv ? i : mv);
  double s_own = 0.0, mW = 0.0;
  for (int k = 0; k < q; ++k) {
    const double a = Acoef[(size_t)i * mv + k];
    s_own += a * a;
    mW += W[N[(size_t)i * mv + k]];
  }
  double s_ch = 0.0, s_chw = 0.0;
  if (mv > 0)
    for (int p = ch_ptr[i]; p < ch_ptr[i + 1]; ++p) {
      const int j = ch_row[p];
      const double a = Acoef[(size_t)j * mv + ch_slot[p]];
      s_ch += a * a;
      s_chw += W[j] * a * a;
    }
  float* f = F + (size_t)i * NIN;
  f[0] = (float)((log(wi) + 3.0) * 0.5);
  f[1] = (float)((log(di) + 3.0) * 0.5);
  f[2] = (float)log1p(wi * di);
  f[3] = (float)((double)q / (mv > 0 ? mv : 1));
  f[4] = (float)s_own;
  f[5] = (float)s_ch;
  f[6] = (float)(q > 0 ? log(mW / q / wi) : 0.0);
  f[7] = (float)log1p(s_chw / wi);
  f[8] = rho ? rho[2 * i] : 0.f;
  f[9] = rho ? rho[2 * i + 1] : 0.f;
}

// ---------------------------------------------------------------------------
// Forward: one thread per point, weights in shared memory (float)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_weights(const __half* w16, float* sw) {
  for (int k = threadIdx.x; k < NP; k += blockDim.x) sw[k] = __half2float(w16[k]);
  __syncthreads();
}

template <typename OutT>
__global__ void mlp_forward_kernel(const __half* __restrict__ w16, const float* __restrict__ F, int64_t n,
                                   OutT* c) {
  extern __shared__ float sw[];
  load_weights(w16, sw);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float f[NIN];
#pragma unroll
  for (int t = 0; t < NIN; ++t) f[t] = F[(size_t)i * NIN + t];
  float h1[NH];
#pragma unroll
  for (int a = 0; a < NH; ++a) {
    float s = sw[OB1 + a];
#pragma unroll
    for (int t = 0; t < NIN; ++t) s += sw[OW1 + a * NIN + t] * f[t];
    h1[a] = tanhf(s);
  }
  float o = sw[OB3];
  for (int a = 0; a < NH; ++a) {
    float s = sw[OB2 + a];
#pragma unroll
    for (int b = 0; b < NH; ++b) s += sw[OW2 + a * NH + b] * h1[b];
    o += sw[OW3 + a] * tanhf(s);
  }
  c[i] = (OutT)(4.f * tanhf(0.25f * o));
}

// ---------------------------------------------------------------------------
// Backward: gradient of sum_i gc_i c_i.  Blocks of 64 threads take tiles of 64
// points; activations go through shared memory and thread a accumulates row a of
// dW2 and dW1 and the a-th bias / output weight over the tiles it sees.
// ---------------------------------------------------------------------------
constexpr int BT = 64;
constexpr int BLD = NH + 1;

__global__ __launch_bounds__(BT) void mlp_backward_kernel(const __half* __restrict__ w16, const float* __restrict__ F,
                                                          const float* __restrict__ gc, int64_t n, float* partial) {
  extern __shared__ float smem[];
  float* sw = smem;                       // NP
  float* sh1 = sw + NPP;                  // BT x BLD
  float* sh2 = sh1 + BT * BLD;
  float* sda2 = sh2 + BT * BLD;
  float* sda1 = sda2 + BT * BLD;
  float* sF = sda1 + BT * BLD;            // BT x NIN
  float* sdo = sF + BT * NIN;             // BT
  load_weights(w16, sw);
  const int t = threadIdx.x;
  float gW2[NH], gW1[NIN];
#pragma unroll
  for (int b = 0; b < NH; ++b) gW2[b] = 0.f;
#pragma unroll
  for (int b = 0; b < NIN; ++b) gW1[b] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
  const int64_t ntile = (n + BT - 1) / BT;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t i = tile * BT + t;
    const bool valid = i < n;
    // forward of point i, keeping activations
    float f[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) {
      f[k] = valid ? F[(size_t)i * NIN + k] : 0.f;
      sF[t * NIN + k] = f[k];
    }
    for (int a = 0; a < NH; ++a) {
      float s = sw[OB1 + a];
#pragma unroll
      for (int k = 0; k < NIN; ++k) s += sw[OW1 + a * NIN + k] * f[k];
      sh1[t * BLD + a] = tanhf(s);
    }
    float o = sw[OB3];
    for (int a = 0; a < NH; ++a) {
      float s = sw[OB2 + a];
      for (int b = 0; b < NH; ++b) s += sw[OW2 + a * NH + b] * sh1[t * BLD + b];
      const float h2 = tanhf(s);
      sh2[t * BLD + a] = h2;
      o += sw[OW3 + a] * h2;
    }
    const float th = tanhf(0.25f * o);
    const float dout = valid ? gc[i] * (1.f - th * th) : 0.f;
    sdo[t] = dout;
    for (int a = 0; a < NH; ++a) {
      const float h2 = sh2[t * BLD + a];
      sda2[t * BLD + a] = dout * sw[OW3 + a] * (1.f - h2 * h2);
    }
    for (int b = 0; b < NH; ++b) {
      float s = 0.f;
      for (int a = 0; a < NH; ++a) s += sw[OW2 + a * NH + b] * sda2[t * BLD + a];
      const float h1 = sh1[t * BLD + b];
      sda1[t * BLD + b] = s * (1.f - h1 * h1);
    }
    __syncthreads();
    // thread t accumulates row a = t
    const int a = t;
    for (int p = 0; p < BT; ++p) {
      const float d2 = sda2[p * BLD + a];
      const float d1 = sda1[p * BLD + a];
#pragma unroll
      for (int b = 0; b < NH; ++b) gW2[b] += d2 * sh1[p * BLD + b];
#pragma unroll
      for (int k = 0; k < NIN; ++k) gW1[k] += d1 * sF[p * NIN + k];
      gb2 += d2;
      gb1 += d1;
      gw3 += sdo[p] * sh2[p * BLD + a];
      if (a == 0) gb3 += sdo[p];
    }
    __syncthreads();
  }
  float* out = partial + (size_t)blockIdx.x * NPP;
  const int a = t;
#pragma unroll
  for (int b = 0; b < NH; ++b) out[OW2 + a * NH + b] = gW2[b];
#pragma unroll
  for (int k = 0; k < NIN; ++k) out[OW1 + a * NIN + k] = gW1[k];
  out[OB1 + a] = gb1;
  out[OB2 + a] = gb2;
  out[OW3 + a] = gw3;
  if (a == 0) out[OB3] = gb3;
}

__global__ void mlp_reduce_kernel(const float* partial, int nb, float* grad) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NP) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(size_t)b * NPP + k];
  grad[k] = (float)s;
}

__global__ void mlp_adam_kernel(void* net, const float* grad, float lr, float b1, float b2, float eps) {
  NetView nv = net_view(net);
  const float t = nv.step[0] + 1.f;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NP) {
    const float g = grad[k];
    const float m = b1 * nv.m[k] + (1.f - b1) * g;
    const float v = b2 * nv.v[k] + (1.f - b2) * g * g;
    nv.m[k] = m;
    nv.v[k] = v;
    const float mh = m / (1.f - powf(b1, t)), vh = v / (1.f - powf(b2, t));
    const float w = nv.master[k] - lr * mh / (sqrtf(vh) + eps);
    nv.master[k] = w;
    nv.w16[k] = __float2half_rn(w);
  }
}
__global__ void mlp_step_kernel(void* net) { net_view(net).step[0] += 1.f; }

// ---------------------------------------------------------------------------
// Loss-gradient pieces
// ---------------------------------------------------------------------------
__global__ void rademacher_kernel(uint64_t seed, int64_t n, double* z) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = (splitmix64(seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(i + 1))) & 1ull) ? 1.0 : -1.0;
}

// gc_i += coeff * (B s)_i (B u)_i d_i,   (B x)_i = x_i - sum_k A_i[k] x_{N_k}
__global__ void lp_grad_kernel(const int32_t* __restrict__ N, const double* __restrict__ Acoef, int64_t n, int mv,
                               const double* __restrict__ s, const double* __restrict__ u,
                               const double* __restrict__ W, const double* __restrict__ corr, double coeff,
                               float* gc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int q = (int)(i < mv ? i : mv);
  double bs = s[i], bu = u[i];
  for (int k = 0; k < q; ++k) {
    const double a = Acoef[(size_t)i * mv + k];
    const int j = N[(size_t)i * mv + k];
    bs -= a * s[j];
    bu -= a * u[j];
  }
  const double d = W[i] * exp(corr[i]);
  gc[i] += (float)(coeff * bs * bu * d);
}

__global__ void zero_f32_kernel(float* x, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.f;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t mlp_init(void* net, uint64_t seed, cudaStream_t s) {
  mlp_init_kernel<<<nblk(NPP, 256), 256, 0, s>>>(net, seed);
  return cudaGetLastError();
}
cudaError_t mlp_set(void* net, const float* p, cudaStream_t s) {
  mlp_set_kernel<<<nblk(NPP, 256), 256, 0, s>>>(net, p);
  return cudaGetLastError();
}
cudaError_t mlp_features(const double* W, const double* D, const double* Acoef, const float* rho, const int32_t* N,
                         const int32_t* ch_ptr, const int32_t* ch_row, const int32_t* ch_slot, int64_t n, int mv,
                         float* F, cudaStream_t s) {
  mlp_features_kernel<<<nblk(n, 256), 256, 0, s>>>(W, D, Acoef, rho, N, ch_ptr, ch_row, ch_slot, n, mv, F);
  return cudaGetLastError();
}
cudaError_t mlp_forward_f32(const void* net, const float* F, int64_t n, float* c, cudaStream_t s) {
  const __half* w16 = net_view(const_cast<void*>(net)).w16;
  mlp_forward_kernel<float><<<nblk(n, 128), 128, NPP * sizeof(float), s>>>(w16, F, n, c);
  return cudaGetLastError();
}
cudaError_t mlp_forward_f64(const void* net, const float* F, int64_t n, double* c, cudaStream_t s) {
  const __half* w16 = net_view(const_cast<void*>(net)).w16;
  mlp_forward_kernel<double><<<nblk(n, 128), 128, NPP * sizeof(float), s>>>(w16, F, n, c);
  return cudaGetLastError();
}
int mlp_backward_blocks(int64_t n) {
  int64_t t = (n + BT - 1) / BT;
  return (int)(t < 304 ? t : 304);
}
cudaError_t mlp_backward(const void* net, const float* F, const float* gc, int64_t n, float* partial, float* grad,
                         cudaStream_t s) {
  const __half* w16 = net_view(const_cast<void*>(net)).w16;
  const int nb = mlp_backward_blocks(n);
  const size_t smem = (size_t)(NPP + 4 * BT * BLD + BT * NIN + BT) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_backward_kernel<<<nb, BT, smem, s>>>(w16, F, gc, n, partial);
  mlp_reduce_kernel<<<nblk(NP, 256), 256, 0, s>>>(partial, nb, grad);
  return cudaGetLastError();
}
cudaError_t mlp_adam(void* net, const float* grad, float lr, cudaStream_t s) {
  mlp_adam_kernel<<<nblk(NP, 256), 256, 0, s>>>(net, grad, lr, 0.9f, 0.999f, 1e-8f);
  mlp_step_kernel<<<1, 1, 0, s>>>(net);
  return cudaGetLastError();
}
cudaError_t mlp_rademacher(uint64_t seed, int64_t n, double* z, cudaStream_t s) {
  rademacher_kernel<<<nblk(n, 256), 256, 0, s>>>(seed, n, z);
  return cudaGetLastError();
}
cudaError_t mlp_lp_grad(const int32_t* N, const double* Acoef, int64_t n, int mv, const double* sv, const double* u,
                        const double* W, const double* corr, double coeff, float* gc, cudaStream_t s) {
  lp_grad_kernel<<<nblk(n, 256), 256, 0, s>>>(N, Acoef, n, mv, sv, u, W, corr, coeff, gc);
  return cudaGetLastError();
}
cudaError_t mlp_zero(float* x, int64_t n, cudaStream_t s) {
  zero_f32_kernel<<<nblk(n, 256), 256, 0, s>>>(x, n);
  return cudaGetLastError();
}
const float* mlp_master(const void* net) { return net_view(const_cast<void*>(net)).master; }

}  // namespace vif
