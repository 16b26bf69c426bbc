// Correlation-based causal neighbour search (Sec. 6, distance d_c; Sec. 2.1
// neighbour rule), as an exact tiled brute force.
//
// For query i and every j < i the ranking key is 1 - |rho_ij| with
//   rho_ij = c_r(i,j) / sqrt(c_r(i,i) c_r(j,j)),  c_r(i,j) = K(s_i,s_j) - a_i . a_j,
// (no nugget; rho := 0 when a residual variance is <= tau), since
// d_c = sqrt(1 - |rho|) orders the same way.  N(i) = the min(i, m_v) smallest
// (key, j) pairs.  The paper's modified cover tree (Alg. 3/4) returns exactly this
// set; a brute force over the n^2/2 pairs is the GPU form of the same answer.
//
// Three stages:
//  1. filter (float32, SIMT): query tiles of 64 stream over earlier key tiles of
//     64 like a causal attention sweep; the 64 x 64 block of a_i . a_j is
//     accumulated over m, the epilogue turns it into keys, and each warp keeps a
//     sorted top-K' list per query in registers (K' = 32 or 64 >= m_v + 8).  For
//     every pair a rigorous bound e_ij on |key32 - key| is formed from the norms
//     of a_i, a_j and a bound on the float32 kernel error; each query also
//     records lowbound = min over all rejected or evicted j of (key32 - e).
//  2. certify (one warp per query): candidates whose interval
//     [key32 - e, key32 + e] proves them inside or outside the top m_v are
//     settled; the ambiguous ones are rescored in float64, and the result is
//     accepted only if every non-candidate is provably worse (lowbound > the
//     worst chosen key).
//  3. fallback: uncertified queries are redone by a float64 brute force.
#include "vif_internal.cuh"

namespace vif {

constexpr int KT = 64;            // query / key tile
constexpr int KC = 32;            // m-chunk of the dot products
constexpr int KMAXD = 16;
#define FINF __int_as_float(0x7f800000)

__device__ __forceinline__ bool lex_less(float ka, int ia, float kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}
__device__ __forceinline__ bool lex_less_d(double ka, int ia, double kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Insert (nk, ni, ne) into a warp-distributed sorted list of 32*E entries
// (lane l holds global positions l*E .. l*E+E-1).  Returns through *ev_key/*ev_e
// the evicted entry (valid on all lanes) if the list was full.
template <int E, typename K>
__device__ __forceinline__ void warp_list_insert(K (&key)[E], int (&idx)[E], float (&ee)[E], int& cnt, K nk,
                                                 int ni, float ne, bool& evicted, K& ev_key, float& ev_e) {
  const int lane = threadIdx.x & 31;
  int below = 0;
#pragma unroll
  for (int s = 0; s < E; ++s) below += (idx[s] >= 0 && (key[s] < nk || (key[s] == nk && idx[s] < ni))) ? 1 : 0;
  const int pos = __reduce_add_sync(0xffffffffu, below);
  evicted = (cnt == 32 * E);
  ev_key = __shfl_sync(0xffffffffu, key[E - 1], 31);
  ev_e = __shfl_sync(0xffffffffu, ee[E - 1], 31);
  K pk = __shfl_up_sync(0xffffffffu, key[E - 1], 1);
  int pi = __shfl_up_sync(0xffffffffu, idx[E - 1], 1);
  float pe = __shfl_up_sync(0xffffffffu, ee[E - 1], 1);
#pragma unroll
  for (int s = E - 1; s >= 0; --s) {
    const int g = lane * E + s;
    K ok;
    int oi;
    float oe;
    if (s > 0) {
      ok = key[s - 1];
      oi = idx[s - 1];
      oe = ee[s - 1];
    } else {
      ok = pk;
      oi = pi;
      oe = pe;
    }
    if (g == pos) {
      key[s] = nk;
      idx[s] = ni;
      ee[s] = ne;
    } else if (g > pos) {
      key[s] = ok;
      idx[s] = oi;
      ee[s] = oe;
    }
  }
  if (!evicted) ++cnt;
}

template <int E>
__global__ __launch_bounds__(256) void knn_filter_kernel(KnnParams p, const float* __restrict__ A32,
                                                         const float* __restrict__ Xs32,
                                                         const float* __restrict__ rs32,
                                                         const float* __restrict__ nrm32, float* cand_key,
                                                         int32_t* cand_idx, float* cand_e, float* lowbound) {
  constexpr int KP = 32 * E;
  const int ntile = (int)((p.n + KT - 1) / KT);
  const int qt = ntile - 1 - (int)blockIdx.x;     // heaviest tiles first
  const int64_t q0 = (int64_t)qt * KT;
  __shared__ __align__(16) float As[KC][KT + 4];
  __shared__ __align__(16) float Bs[KC][KT + 4];
  __shared__ float Sk[KT][KT + 1];
  __shared__ float qx[KT * KMAXD], kx[KT * KMAXD];
  __shared__ float q_rs[KT], q_nrm[KT], k_rs[KT], k_nrm[KT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int w = tid >> 5, lane = tid & 31;
  const int d = p.d;
  for (int e = tid; e < KT * d; e += 256) {
    int64_t qi = q0 + e / d;
    qx[e] = (qi < p.n) ? Xs32[(size_t)q0 * d + e] : 0.f;
  }
  for (int e = tid; e < KT; e += 256) {
    int64_t qi = q0 + e;
    q_rs[e] = (qi < p.n) ? rs32[qi] : 0.f;
    q_nrm[e] = (qi < p.n) ? nrm32[qi] : 0.f;
  }
  float lkey[8][E];
  int lidx[8][E];
  float le[8][E];
  int cnt[8];
  float lowb[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    cnt[a] = 0;
    lowb[a] = FINF;
#pragma unroll
    for (int s = 0; s < E; ++s) {
      lkey[a][s] = FINF;
      lidx[a][s] = -1;
      le[a][s] = 0.f;
    }
  }
  const float u32 = 5.9604645e-8f;
  const float grow = 1.0f + 8.0f * u32;
  for (int kt = 0; kt <= qt; ++kt) {
    const int64_t k0 = (int64_t)kt * KT;
    // two-level summation: each 32-term chunk is summed on its own and then added
    // to the running total, which bounds the float32 error by (32 + m/32 + 2) u
    // times sum |a_ik a_jk| instead of m u.
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int c0 = 0; c0 < p.m; c0 += KC) {
      float part[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) part[u][v] = 0.f;
      __syncthreads();
      for (int e = tid; e < KT * KC; e += 256) {
        int r = e / KC, kk = e % KC;
        int64_t qi = q0 + r, kj = k0 + r;
        As[kk][r] = (qi < p.n) ? A32[(size_t)qi * p.mpad + c0 + kk] : 0.f;
        Bs[kk][r] = (kj < p.n) ? A32[(size_t)kj * p.mpad + c0 + kk] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
        float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) part[u][v] += av[u] * bv[v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += part[u][v];
    }
    __syncthreads();
    for (int e = tid; e < KT * d; e += 256) {
      int64_t kj = k0 + e / d;
      kx[e] = (kj < p.n) ? Xs32[(size_t)k0 * d + e] : 0.f;
    }
    for (int e = tid; e < KT; e += 256) {
      int64_t kj = k0 + e;
      k_rs[e] = (kj < p.n) ? rs32[kj] : 0.f;
      k_nrm[e] = (kj < p.n) ? nrm32[kj] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int ql = ty * 4 + u, kl = tx * 4 + v;
        const int64_t qi = q0 + ql, kj = k0 + kl;
        float key = FINF;
        if (qi < p.n && kj < qi) {
          float rq = q_rs[ql], rk = k_rs[kl];
          if (rq == 0.f || rk == 0.f) {
            key = 1.0f;
          } else {
            float K = cov_r2<float>(sqdist(qx + ql * d, kx + kl * d, d), p.kind, (float)p.var);
            float rho = fabsf((K - acc[u][v]) * rq * rk);
            key = 1.0f - fminf(rho, 1.0f);
          }
        }
        Sk[ql][kl] = key;
      }
    __syncthreads();
    // ---- per-query selection: warp w owns queries w*8 .. w*8+7
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ql = w * 8 + a;
      const float rq = q_rs[ql], nq = q_nrm[ql];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kl = lane + 32 * h;
        const float key = Sk[ql][kl];
        const int j = (int)(k0 + kl);
        const bool valid = key < FINF;
        float e = 0.f;
        if (valid && rq != 0.f && k_rs[kl] != 0.f)
          e = (p.gamma * nq * k_nrm[kl] + p.epsK) * rq * k_rs[kl] * grow + 8.0f * u32;
        float thr_k = __shfl_sync(0xffffffffu, lkey[a][E - 1], 31);
        int thr_i = __shfl_sync(0xffffffffu, lidx[a][E - 1], 31);
        bool full = (cnt[a] == KP);
        bool pass = valid && (!full || lex_less(key, j, thr_k, thr_i));
        if (valid && !pass) lowb[a] = fminf(lowb[a], key - e);
        unsigned bal = __ballot_sync(0xffffffffu, pass);
        while (bal) {
          const int src = __ffs(bal) - 1;
          bal &= bal - 1;
          const float nk = __shfl_sync(0xffffffffu, key, src);
          const int ni = __shfl_sync(0xffffffffu, j, src);
          const float ne = __shfl_sync(0xffffffffu, e, src);
          thr_k = __shfl_sync(0xffffffffu, lkey[a][E - 1], 31);
          thr_i = __shfl_sync(0xffffffffu, lidx[a][E - 1], 31);
          if (cnt[a] == KP && !lex_less(nk, ni, thr_k, thr_i)) {
            lowb[a] = fminf(lowb[a], nk - ne);
            continue;
          }
          bool ev;
          float evk, eve;
          warp_list_insert<E, float>(lkey[a], lidx[a], le[a], cnt[a], nk, ni, ne, ev, evk, eve);
          if (ev) lowb[a] = fminf(lowb[a], evk - eve);
        }
      }
    }
  }
  // ---- write lists
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t qi = q0 + w * 8 + a;
    float lb = lowb[a];
    for (int o = 16; o > 0; o >>= 1) lb = fminf(lb, __shfl_xor_sync(0xffffffffu, lb, o));
    if (qi < p.n) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        size_t g = (size_t)qi * KP + lane * E + s;
        cand_key[g] = lkey[a][s];
        cand_idx[g] = lidx[a][s];
        cand_e[g] = le[a][s];
      }
      if (lane == 0) lowbound[qi] = lb;
    }
  }
}

// float64 key of one pair, warp-cooperative (all lanes return the same value).
__device__ double key64_warp(const KnnParams& p, const double* A64, const double* Xs64, const double* cii,
                             int64_t i, int64_t j) {
  const int lane = threadIdx.x & 31;
  double dot = 0.0;
  for (int k = lane; k < p.m; k += 32) dot += A64[(size_t)i * p.mpad + k] * A64[(size_t)j * p.mpad + k];
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  double ci = cii[i], cj = cii[j];
  if (ci <= p.tau_v || cj <= p.tau_v) return 1.0;
  double K = cov_r2<double>(sqdist(Xs64 + (size_t)i * p.d, Xs64 + (size_t)j * p.d, p.d), p.kind, p.var);
  double rho = fabs(K - dot) / sqrt(ci * cj);
  return 1.0 - fmin(rho, 1.0);
}

template <int E>
__global__ __launch_bounds__(256) void knn_certify_kernel(KnnParams p, const double* __restrict__ A64,
                                                          const double* __restrict__ Xs64,
                                                          const double* __restrict__ cii, const float* cand_key,
                                                          const int32_t* cand_idx, const float* cand_e,
                                                          const float* lowbound, int32_t* N, int* counters,
                                                          int32_t* fallback_list) {
  constexpr int KP = 32 * E;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= p.n) return;
  const int mv = p.mv;
  if (i <= mv) {
    for (int t = lane; t < mv; t += 32) N[(size_t)i * mv + t] = (t < i) ? t : -1;
    return;
  }
  float key[E], e[E], lo[E], hi[E];
  int idx[E];
#pragma unroll
  for (int s = 0; s < E; ++s) {
    size_t g = (size_t)i * KP + lane * E + s;
    key[s] = cand_key[g];
    idx[s] = cand_idx[g];
    e[s] = cand_e[g];
    lo[s] = key[s] - e[s];
    hi[s] = key[s] + e[s];
  }
  const float lb = lowbound[i];
  bool sure_in[E], amb[E];
  int nin_l = 0;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    int c_le = 0, c_lt = 0;
    for (int g = 0; g < KP; ++g) {
      float glo = __shfl_sync(0xffffffffu, lo[g % E], g / E);
      float ghi = __shfl_sync(0xffffffffu, hi[g % E], g / E);
      int gid = __shfl_sync(0xffffffffu, idx[g % E], g / E);
      if (gid < 0) continue;
      if (g != lane * E + s && glo <= hi[s]) ++c_le;
      if (ghi < lo[s]) ++c_lt;
    }
    const bool valid = idx[s] >= 0;
    sure_in[s] = valid && (c_le <= mv - 1) && (lb > hi[s]);
    const bool sure_out = !valid || (c_lt >= mv);
    amb[s] = !sure_in[s] && !sure_out;
    nin_l += sure_in[s] ? 1 : 0;
  }
  const int nin = __reduce_add_sync(0xffffffffu, nin_l);
  bool chosen[E];
#pragma unroll
  for (int s = 0; s < E; ++s) chosen[s] = sure_in[s];
  if (nin < mv) {
    double k64[E];
#pragma unroll
    for (int s = 0; s < E; ++s) k64[s] = 2.0;
    // rescore ambiguous candidates in float64
#pragma unroll
    for (int s = 0; s < E; ++s) {
      unsigned bal = __ballot_sync(0xffffffffu, amb[s]);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1;
        const int j = __shfl_sync(0xffffffffu, idx[s], src);
        double kv = key64_warp(p, A64, Xs64, cii, i, j);
        if (lane == src) k64[s] = kv;
      }
    }
    const int need = mv - nin;
    double kmax = -1.0;
#pragma unroll
    for (int s = 0; s < E; ++s) {
      int rank = 0;
      for (int g = 0; g < KP; ++g) {
        double gk = __shfl_sync(0xffffffffu, k64[g % E], g / E);
        int gid = __shfl_sync(0xffffffffu, idx[g % E], g / E);
        bool gamb = __shfl_sync(0xffffffffu, amb[g % E] ? 1 : 0, g / E) != 0;
        if (gamb && amb[s] && lex_less_d(gk, gid, k64[s], idx[s])) ++rank;
      }
      if (amb[s] && rank < need) {
        chosen[s] = true;
        kmax = fmax(kmax, k64[s]);
      }
    }
    for (int o = 16; o > 0; o >>= 1) kmax = fmax(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    if (lane == 0) atomicAdd(&counters[0], 1);
    if (!((double)lb > kmax)) {
      if (lane == 0) {
        int pos = atomicAdd(&counters[1], 1);
        fallback_list[pos] = (int32_t)i;
      }
      return;
    }
  }
  // write the chosen indices in ascending order
#pragma unroll
  for (int s = 0; s < E; ++s) {
    int rank = 0;
    for (int g = 0; g < KP; ++g) {
      int gid = __shfl_sync(0xffffffffu, idx[g % E], g / E);
      bool gch = __shfl_sync(0xffffffffu, chosen[g % E] ? 1 : 0, g / E) != 0;
      if (gch && gid < idx[s]) ++rank;
    }
    if (chosen[s] && rank < mv) N[(size_t)i * mv + rank] = idx[s];
  }
}

// float64 brute force for one query per CTA: each warp keeps a top-64 list of its
// own j's, then warp 0 merges the eight lists.
__global__ __launch_bounds__(256) void knn_fallback_kernel(KnnParams p, const double* __restrict__ A64,
                                                           const double* __restrict__ Xs64,
                                                           const double* __restrict__ cii, const int32_t* list,
                                                           int32_t* N) {
  constexpr int E = 2, KP = 64;
  const int64_t i = list[blockIdx.x];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double mk[8][KP];
  __shared__ int mi[8][KP];
  double key[E];
  int idx[E];
  float dummy[E];
  int cnt = 0;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    key[s] = 1e300;
    idx[s] = -1;
    dummy[s] = 0.f;
  }
  const double ci = cii[i];
  const double* ai = A64 + (size_t)i * p.mpad;
  for (int64_t jb = (int64_t)w * 32; jb < i; jb += 256) {
    const int64_t j = jb + lane;
    double kj = 1e300;
    if (j < i) {
      double dot = 0.0;
      const double* aj = A64 + (size_t)j * p.mpad;
      for (int k = 0; k < p.m; ++k) dot += ai[k] * aj[k];
      double cj = cii[j];
      if (ci <= p.tau_v || cj <= p.tau_v) {
        kj = 1.0;
      } else {
        double K = cov_r2<double>(sqdist(Xs64 + (size_t)i * p.d, Xs64 + (size_t)j * p.d, p.d), p.kind, p.var);
        kj = 1.0 - fmin(fabs(K - dot) / sqrt(ci * cj), 1.0);
      }
    }
    double thr_k = __shfl_sync(0xffffffffu, key[E - 1], 31);
    int thr_i = __shfl_sync(0xffffffffu, idx[E - 1], 31);
    bool pass = (j < i) && (cnt < KP || lex_less_d(kj, (int)j, thr_k, thr_i));
    unsigned bal = __ballot_sync(0xffffffffu, pass);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      double nk = __shfl_sync(0xffffffffu, kj, src);
      int ni = (int)__shfl_sync(0xffffffffu, (int)j, src);
      thr_k = __shfl_sync(0xffffffffu, key[E - 1], 31);
      thr_i = __shfl_sync(0xffffffffu, idx[E - 1], 31);
      if (cnt == KP && !lex_less_d(nk, ni, thr_k, thr_i)) continue;
      bool ev;
      double evk;
      float eve;
      warp_list_insert<E, double>(key, idx, dummy, cnt, nk, ni, 0.f, ev, evk, eve);
    }
  }
#pragma unroll
  for (int s = 0; s < E; ++s) {
    mk[w][lane * E + s] = key[s];
    mi[w][lane * E + s] = idx[s];
  }
  __syncthreads();
  if (w != 0) return;
  for (int ww = 1; ww < 8; ++ww) {
    for (int g = 0; g < KP; ++g) {
      double nk = mk[ww][g];
      int ni = mi[ww][g];
      if (ni < 0) continue;
      double thr_k = __shfl_sync(0xffffffffu, key[E - 1], 31);
      int thr_i = __shfl_sync(0xffffffffu, idx[E - 1], 31);
      if (cnt == KP && !lex_less_d(nk, ni, thr_k, thr_i)) continue;
      bool ev;
      double evk;
      float eve;
      warp_list_insert<E, double>(key, idx, dummy, cnt, nk, ni, 0.f, ev, evk, eve);
    }
  }
  // the first mv entries of the merged list, in ascending index order
  const int mv = p.mv;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const int gpos = lane * E + s;
    const bool take = gpos < mv && idx[s] >= 0;
    int rank = 0;
    for (int g = 0; g < KP; ++g) {
      int gid = __shfl_sync(0xffffffffu, idx[g % E], g / E);
      if (g < mv && gid >= 0 && gid < idx[s]) ++rank;
    }
    if (take) N[(size_t)i * mv + rank] = idx[s];
  }
}

cudaError_t knn_causal(const KnnParams& p, const float* A32, const double* A64, const float* Xs32,
                       const double* Xs64, const double* cii, const float* rs32, const float* nrm32,
                       float* cand_key, int32_t* cand_idx, float* cand_e, float* lowbound, int32_t* N,
                       int* counters, int32_t* fallback_list, cudaStream_t s) {
  if (p.mv <= 0 || p.n <= 0) return cudaSuccess;
  if (p.d > KMAXD) return cudaErrorInvalidValue;
  const unsigned ntile = (unsigned)((p.n + KT - 1) / KT);
  const unsigned cgrid = (unsigned)((p.n + 7) / 8);
  cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (p.kprime == 32) {
    knn_filter_kernel<1><<<ntile, 256, 0, s>>>(p, A32, Xs32, rs32, nrm32, cand_key, cand_idx, cand_e, lowbound);
    knn_certify_kernel<1><<<cgrid, 256, 0, s>>>(p, A64, Xs64, cii, cand_key, cand_idx, cand_e, lowbound, N,
                                                counters, fallback_list);
  } else {
    knn_filter_kernel<2><<<ntile, 256, 0, s>>>(p, A32, Xs32, rs32, nrm32, cand_key, cand_idx, cand_e, lowbound);
    knn_certify_kernel<2><<<cgrid, 256, 0, s>>>(p, A64, Xs64, cii, cand_key, cand_idx, cand_e, lowbound, N,
                                                counters, fallback_list);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int h[2];
  e = cudaMemcpyAsync(h, counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (h[1] > 0) {
    knn_fallback_kernel<<<h[1], 256, 0, s>>>(p, A64, Xs64, cii, fallback_list, N);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace vif
