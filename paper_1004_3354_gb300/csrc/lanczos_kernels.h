// Lanczos building blocks shared by the solver drivers (lanczos.cu) and the
// request server (serve.cu): reductions, vector updates, the coefficient
// bookkeeping kernel, CGS2 and the tridiagonal solve.  Internal header; each
// translation unit gets its own copy (anonymous namespace).
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ed_internal.h"
#include "tri_common.h"
#include "vec16.h"

namespace ed {

namespace {

constexpr int kRedThreads = 256;

// ------------------------------------------------ element-level helpers
__device__ __forceinline__ void dmac(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void dmac(float2& a, float2 x, float2 y) { df_mac(a, x, y); }
__device__ __forceinline__ void dmac(float2& a, float x, float y) { df_mac1(a, make_float2(x, 0.f), y); }

__device__ __forceinline__ double to_d(double a) { return a; }
__device__ __forceinline__ double to_d(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ double add_acc(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add_acc(float2 a, float2 b) { return df_add(a, b); }

__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shfl_x(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

template <class A>
__device__ __forceinline__ A block_reduce(A v, A* sh) {
  for (int o = 16; o > 0; o >>= 1) v = add_acc(v, shfl_x(v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    v = (lane < nw) ? sh[lane] : A{};
    for (int o = 16; o > 0; o >>= 1) v = add_acc(v, shfl_x(v, o));
  }
  __syncthreads();
  return v;  // valid in thread 0
}

// accumulator initialised from a stored element
__device__ __forceinline__ double acc_of(double x) { return x; }
__device__ __forceinline__ float2 acc_of(float2 x) { return x; }
__device__ __forceinline__ float2 acc_of(float x) { return make_float2(x, 0.f); }

__device__ __forceinline__ void amac(double& a, const double* cd, const float2*, int k, double x) {
  a = fma(cd[k], x, a);
}
__device__ __forceinline__ void amac(float2& a, const double*, const float2* cf, int k, float2 x) {
  df_mac(a, cf[k], x);
}
__device__ __forceinline__ void amac(float2& a, const double*, const float2* cf, int k, float x) {
  df_mac1(a, cf[k], x);
}

__device__ __forceinline__ double store_v(double a, double*) { return a; }
__device__ __forceinline__ float2 store_v(float2 a, float2*) { return df_norm(a); }
__device__ __forceinline__ float store_v(float2 a, float*) { return __fadd_rn(a.x, a.y); }

template <class V>
struct AccOf;
template <>
struct AccOf<double> { using T = double; };
template <>
struct AccOf<float2> { using T = float2; };
template <>
struct AccOf<float> { using T = float2; };

// ------------------------------------------------ reductions
// partial[b] = sum over this block's elements of x*y (as double)
template <class V>
__global__ void __launch_bounds__(kRedThreads) k_dot(const V* __restrict__ x, const V* __restrict__ y,
                                                     uint64_t n, double* __restrict__ partial) {
  using A = typename AccOf<V>::T;
  __shared__ A sh[32];
  A acc{};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    dmac(acc, x[i], y[i]);
  acc = block_reduce(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = to_d(acc);
}

// Multi-dot of the chunk k0 .. k0 + KB - 1: partial[q * nb + b] = block b's
// share of <V_{k0+q}, w>.
template <class V, int KB>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const V* __restrict__ Vb, uint64_t stride, int k0,
                                                          int nvec, const V* __restrict__ w, uint64_t n,
                                                          double* __restrict__ partial) {
  using A = typename AccOf<V>::T;
  __shared__ A sh[32];
  A acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = A{};
  int kn = min(KB, nvec - k0);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    V wi = w[i];
#pragma unroll
    for (int q = 0; q < KB; ++q)
      if (q < kn) dmac(acc[q], Vb[(uint64_t)(k0 + q) * stride + i], wi);
  }
  for (int q = 0; q < kn; ++q) {
    A r = block_reduce(acc[q], sh);
    if (threadIdx.x == 0) partial[(uint64_t)q * gridDim.x + blockIdx.x] = to_d(r);
  }
}

// The same multi-dot with sixteen-byte loads (every slot, and w, 16-byte
// aligned): (KB + 1) x 16 bytes per thread in flight; the tail of the range
// element by element.
template <class V, int KB>
__global__ void __launch_bounds__(kRedThreads) k_multidot16(const V* __restrict__ Vb, uint64_t stride, int k0,
                                                            int nvec, const V* __restrict__ w, uint64_t n,
                                                            double* __restrict__ partial) {
  using A = typename AccOf<V>::T;
  using W16 = Vec16<V>;
  using VT = typename W16::T;
  constexpr int N = W16::N;
  __shared__ A sh[32];
  A acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = A{};
  const int kn = min(KB, nvec - k0);
  const uint64_t nv = n / N;
  const uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (uint64_t)gridDim.x * blockDim.x;
  const VT* wv = reinterpret_cast<const VT*>(w);
  const V* vk = Vb + (uint64_t)k0 * stride;
  for (uint64_t t = g0; t < nv; t += gs) {
    const VT wq = wv[t];
    VT vq[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q)
      if (q < kn) vq[q] = __ldg(reinterpret_cast<const VT*>(vk + (uint64_t)q * stride) + t);
#pragma unroll
    for (int q = 0; q < KB; ++q)
      if (q < kn) {
#pragma unroll
        for (int i = 0; i < N; ++i) dmac(acc[q], W16::get(vq[q], i), W16::get(wq, i));
      }
  }
  for (uint64_t i = nv * N + g0; i < n; i += gs) {
    const V wi = w[i];
#pragma unroll
    for (int q = 0; q < KB; ++q)
      if (q < kn) dmac(acc[q], vk[(uint64_t)q * stride + i], wi);
  }
  for (int q = 0; q < kn; ++q) {
    A r = block_reduce(acc[q], sh);
    if (threadIdx.x == 0) partial[(uint64_t)q * gridDim.x + blockIdx.x] = to_d(r);
  }
}

// ------------------------------------------------ coefficient bookkeeping
struct Coefs {
  double* alpha;    // [m+1]
  double* beta;     // [m+2], beta[0] = 0
  double* nal_d;    // -alpha
  float2* nal_f;
  double* nbe_d;    // -beta
  float2* nbe_f;
  double* inv_d;    // 1 / beta (0 when beta vanished)
  float2* inv_f;
  double* h_d;      // -h (CGS projections)
  float2* h_f;
  double* scale;    // running max |alpha|, beta
  int* exhausted;   // first step with a vanished beta, -1 if none
  double* out;      // generic scalar output slots
  // three-vector recurrence on unnormalised vectors q_j (v_j = sigma_j q_j):
  // q_{j+1} = ua_j H q_j + ub_j q_j + uc_j q_{j-1}
  double* sigma;
  double* ua_d;
  float2* ua_f;
  double* ub_d;
  float2* ub_f;
  double* uc_d;
  float2* uc_f;
  int* step;        // device step index for graph-replayed steps (slot < 0 / j < 0 read it)
};

enum FinishOp { OP_SUM = 0, OP_ALPHA = 1, OP_BETA = 2, OP_NEGH = 3, OP_NORM_INV = 4, OP_SIGMA0 = 5,
                OP_ALPHA_Q = 6, OP_BETA_Q = 7 };

// Sum nb partials (one output per block of this kernel) and apply `op`.
__global__ void __launch_bounds__(kRedThreads) k_finish(const double* __restrict__ partial, int nb, int op,
                                                        int slot, Coefs c, double thr) {
  __shared__ double sh[32];
  int o = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += partial[(uint64_t)o * nb + i];
  v = block_reduce(v, sh);
  if (threadIdx.x != 0) return;
  if (slot < 0) slot = *c.step + (-slot - 1);  // -1: current step j, -2: j + 1
  switch (op) {
    case OP_SUM: c.out[slot + o] = v; break;
    case OP_ALPHA:
      c.alpha[slot] = v;
      c.nal_d[slot] = -v;
      c.nal_f[slot] = df_from_double(-v);
      *c.scale = fmax(*c.scale, fabs(v));
      break;
    case OP_BETA: {
      double b = sqrt(fmax(v, 0.0));
      double sc = fmax(*c.scale, b);
      *c.scale = sc;
      bool dead = !(b > thr * fmax(sc, 1.0));
      if (dead && *c.exhausted < 0) *c.exhausted = slot;
      c.beta[slot] = dead ? 0.0 : b;
      c.nbe_d[slot] = dead ? 0.0 : -b;
      c.nbe_f[slot] = df_from_double(dead ? 0.0 : -b);
      double inv = dead ? 0.0 : 1.0 / b;
      c.inv_d[slot] = inv;
      c.inv_f[slot] = df_from_double(inv);
      break;
    }
    case OP_NEGH:
      c.h_d[slot + o] = -v;
      c.h_f[slot + o] = df_from_double(-v);
      break;
    case OP_NORM_INV: {
      double b = sqrt(fmax(v, 0.0));
      double inv = b > 0.0 ? 1.0 / b : 0.0;
      c.out[slot] = b;
      c.inv_d[slot] = inv;
      c.inv_f[slot] = df_from_double(inv);
      break;
    }
    case OP_SIGMA0: {  // v = <q_0, q_0>
      double b = sqrt(fmax(v, 0.0));
      c.out[0] = b;
      c.sigma[0] = b > 0.0 ? 1.0 / b : 0.0;
      c.beta[0] = 0.0;
      break;
    }
    case OP_ALPHA_Q: {  // v = <q_j, H q_j>; alpha_j = sigma_j^2 v
      const int j = slot;
      const double sg = c.sigma[j];
      const double a = sg * sg * v;
      c.alpha[j] = a;
      *c.scale = fmax(*c.scale, fabs(a));
      const double ua = sg, ub = -a * sg, uc = (j > 0) ? -c.beta[j] * c.sigma[j - 1] : 0.0;
      c.ua_d[j] = ua;
      c.ua_f[j] = df_from_double(ua);
      c.ub_d[j] = ub;
      c.ub_f[j] = df_from_double(ub);
      c.uc_d[j] = uc;
      c.uc_f[j] = df_from_double(uc);
      break;
    }
    case OP_BETA_Q: {  // v = |q_{j+1}|^2
      double b = sqrt(fmax(v, 0.0));
      double sc = fmax(*c.scale, b);
      *c.scale = sc;
      bool dead = !(b > thr * fmax(sc, 1.0));
      if (dead && *c.exhausted < 0) *c.exhausted = slot;
      c.beta[slot] = dead ? 0.0 : b;
      c.sigma[slot] = dead ? 0.0 : 1.0 / b;
      break;
    }
  }
}

// ------------------------------------------------ vector updates
// w = w - alpha_j v - beta_j vprev  (coefficients read from device memory)
template <class V>
__global__ void k_lz_update(V* __restrict__ w, const V* __restrict__ v, const V* __restrict__ vp, uint64_t n,
                            Coefs c, int j) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    auto a = acc_of(w[i]);
    amac(a, c.nal_d, c.nal_f, j, v[i]);
    if (vp) amac(a, c.nbe_d, c.nbe_f, j, vp[i]);
    w[i] = store_v(a, w);
  }
}

// q_out = ua_j y + ub_j q_j + uc_j q_{j-1} with block partials of |q_out|^2.
// q_out may be the buffer of q_{j-1} (element-wise in place).
template <class V>
__global__ void __launch_bounds__(kRedThreads) k_lz_step(const V* __restrict__ y, const V* __restrict__ qj,
                                                         const V* qjm, V* qout, uint64_t n, Coefs c, int j,
                                                         double* __restrict__ partial) {
  using A = typename AccOf<V>::T;
  __shared__ A sh[32];
  A nacc{};
  if (j < 0) j = *c.step;
  if (j == 0) qjm = nullptr;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    typename AccOf<V>::T a{};
    amac(a, c.ua_d, c.ua_f, j, y[i]);
    amac(a, c.ub_d, c.ub_f, j, qj[i]);
    if (qjm) amac(a, c.uc_d, c.uc_f, j, qjm[i]);
    const V q = store_v(a, qout);
    qout[i] = q;
    if (partial) dmac(nacc, q, q);
  }
  if (partial) {
    nacc = block_reduce(nacc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = to_d(nacc);
  }
}

// Sq[i*ldS + j] = S[i*ldS + j] * sigma[j] (Ritz coefficients on unnormalised q_j)
__global__ void k_scale_ritz(const double* __restrict__ S, const double* __restrict__ sigma, int m, int k, int ldS,
                             double* __restrict__ Sq, float2* __restrict__ Sqf) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * k) return;
  int i = t / m, j = t % m;
  double v = S[(size_t)i * ldS + j] * sigma[j];
  Sq[(size_t)i * ldS + j] = v;
  Sqf[(size_t)i * ldS + j] = df_from_double(v);
}

// w -= sum_k h_k V_k for k in [0, nvec)
template <class V>
__global__ void k_multi_axpy(const V* __restrict__ Vb, uint64_t stride, int nvec, V* __restrict__ w, uint64_t n,
                             Coefs c) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    auto a = acc_of(w[i]);
    for (int k = 0; k < nvec; ++k) amac(a, c.h_d, c.h_f, k, Vb[(uint64_t)k * stride + i]);
    w[i] = store_v(a, w);
  }
}

// The same update with sixteen-byte loads and stores (slots and w 16-byte
// aligned); each element's terms in the order k = 0 .. nvec - 1, as above.
template <class V>
__global__ void k_multi_axpy16(const V* __restrict__ Vb, uint64_t stride, int nvec, V* __restrict__ w, uint64_t n,
                               Coefs c) {
  using A = typename AccOf<V>::T;
  using W16 = Vec16<V>;
  using VT = typename W16::T;
  constexpr int N = W16::N;
  const uint64_t nv = n / N;
  const uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (uint64_t)gridDim.x * blockDim.x;
  VT* wv = reinterpret_cast<VT*>(w);
  for (uint64_t t = g0; t < nv; t += gs) {
    const VT wq = wv[t];
    A a[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = acc_of(W16::get(wq, i));
#pragma unroll 4
    for (int k = 0; k < nvec; ++k) {
      const VT vq = __ldg(reinterpret_cast<const VT*>(Vb + (uint64_t)k * stride) + t);
#pragma unroll
      for (int i = 0; i < N; ++i) amac(a[i], c.h_d, c.h_f, k, W16::get(vq, i));
    }
    VT o;
#pragma unroll
    for (int i = 0; i < N; ++i) W16::set(o, i, store_v(a[i], w));
    wv[t] = o;
  }
  for (uint64_t i = nv * N + g0; i < n; i += gs) {
    auto a = acc_of(w[i]);
    for (int k = 0; k < nvec; ++k) amac(a, c.h_d, c.h_f, k, Vb[(uint64_t)k * stride + i]);
    w[i] = store_v(a, w);
  }
}

// out = w * inv[slot]
template <class V>
__global__ void k_scale(const V* __restrict__ w, V* __restrict__ out, uint64_t n, Coefs c, int slot) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    typename AccOf<V>::T a{};
    amac(a, c.inv_d, c.inv_f, slot, w[i]);
    out[i] = store_v(a, out);
  }
}

// v *= 1 / ||v|| (inv_d[slot] from OP_NORM_INV), in place.  Ritz vectors
// regenerated from a three-vector recurrence need it: once a converged Ritz
// value has a ghost copy (loss of orthogonality in finite precision, early
// with float vectors) sum_j S_j v_j keeps its direction but not unit norm.
template <class V>
__global__ void k_rescale(V* __restrict__ v, uint64_t n, Coefs c, int slot) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    typename AccOf<V>::T a{};
    amac(a, c.inv_d, c.inv_f, slot, v[i]);
    v[i] = store_v(a, v);
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ void set_rand(double& o, float u) { o = (double)u; }
__device__ __forceinline__ void set_rand(float2& o, float u) { o = make_float2(u, 0.f); }
__device__ __forceinline__ void set_rand(float& o, float u) { o = u; }

// Seeded start vector: uniform(-1, 1) from a counter-based hash of (seed, i).
template <class V>
__global__ void k_random(V* __restrict__ v, uint64_t n, uint64_t seed) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t r = mix64(seed * 0x2545f4914f6cdd1dull + i);
    float u = (float)((r >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
    set_rand(v[i], u);
  }
}

// out_i += sum_{j<m} S[i*ldS + j] V_j   for eigenvectors i in [i0, i0 + kn)
template <class V, int KB>
__global__ void k_ritz(const V* __restrict__ Vb, uint64_t stride, int m, const double* __restrict__ Sd,
                       const float2* __restrict__ Sf, int ldS, int i0, int kn, V* __restrict__ out,
                       uint64_t n, int accumulate) {
  using A = typename AccOf<V>::T;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (uint64_t)gridDim.x * blockDim.x) {
    A acc[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) acc[q] = (accumulate && q < kn) ? acc_of(out[(uint64_t)(i0 + q) * n + e]) : A{};
    for (int j = 0; j < m; ++j) {
      V vj = Vb[(uint64_t)j * stride + e];
#pragma unroll
      for (int q = 0; q < KB; ++q)
        if (q < kn) amac(acc[q], Sd, Sf, (i0 + q) * ldS + j, vj);
    }
#pragma unroll
    for (int q = 0; q < KB; ++q)
      if (q < kn) out[(uint64_t)(i0 + q) * n + e] = store_v(acc[q], out);
  }
}

__global__ void k_step_inc(int* step) { *step += 1; }

__global__ void k_copy_f64(const void* __restrict__ a, void* __restrict__ b, uint64_t bytes8) {
  const double* s = (const double*)a;
  double* d = (double*)b;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes8;
       i += (uint64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// ------------------------------------------------ tridiagonal eigensolver
// Eigenvalue blockIdx.x (ascending) by 32-way multisection, one warp per value.
__global__ void k_tri_eig(const double* __restrict__ a, const double* __restrict__ b, int m,
                          double* __restrict__ theta) {
  tri_eig_one(a, b, m, blockIdx.x, theta);
}

// Inverse iteration for eigenvector blockIdx.x (thread 0 of the block).
__global__ void k_tri_vec(const double* __restrict__ a, const double* __restrict__ b, int m,
                          const double* __restrict__ theta, double* __restrict__ S, int ldS,
                          double* __restrict__ work) {
  if (threadIdx.x == 0) tri_vec_one(a, b, m, theta, S, ldS, work, blockIdx.x);
}

__global__ void k_tri_finish(const double* __restrict__ theta, int k, int m, double beta_m, double* __restrict__ S,
                             int ldS, float2* __restrict__ Sf, double* __restrict__ resid) {
  tri_finish_block(theta, k, m, beta_m, S, ldS, Sf, resid);
}

// ------------------------------------------------ host-side driver
template <class V>
struct Work {
  Ctx* ctx;
  cudaStream_t st;
  uint64_t n;
  uint32_t grid;
  double* partial;  // ctx->d_red
  Coefs c;
};

template <class V>
int dot_to(Work<V>& W, const V* x, const V* y, int op, int slot, double thr = 0.0) {
  k_dot<V><<<W.grid, kRedThreads, 0, W.st>>>(x, y, W.n, W.partial);
  k_finish<<<1, kRedThreads, 0, W.st>>>(W.partial, (int)W.grid, op, slot, W.c, thr);
  ED_LAUNCH_CHECK();
  return ED_OK;
}

// CGS2 against basis vectors [0, nvec): twice h = V^T w, w -= V h.  The
// projections are reduced eight at a time, so every chunk runs on the full
// grid whatever the basis size.
template <class V>
int cgs2(Work<V>& W, const V* Vb, uint64_t stride, int nvec, V* w) {
  if (nvec <= 0) return ED_OK;
  constexpr int KB = 8;
  const int nb = (int)std::min<uint64_t>(W.grid, (uint64_t)kRedSlots / KB);
  // sixteen-byte loads when every slot and w start on a 16-byte boundary
  const bool v16 = (stride * sizeof(V)) % 16 == 0 && reinterpret_cast<uintptr_t>(Vb) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(w) % 16 == 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int k0 = 0; k0 < nvec; k0 += KB) {
      if (v16) k_multidot16<V, KB><<<nb, kRedThreads, 0, W.st>>>(Vb, stride, k0, nvec, w, W.n, W.partial);
      else k_multidot<V, KB><<<nb, kRedThreads, 0, W.st>>>(Vb, stride, k0, nvec, w, W.n, W.partial);
      k_finish<<<std::min(KB, nvec - k0), kRedThreads, 0, W.st>>>(W.partial, nb, OP_NEGH, k0, W.c, 0.0);
    }
    if (v16) k_multi_axpy16<V><<<W.grid, 256, 0, W.st>>>(Vb, stride, nvec, w, W.n, W.c);
    else k_multi_axpy<V><<<W.grid, 256, 0, W.st>>>(Vb, stride, nvec, w, W.n, W.c);
    ED_LAUNCH_CHECK();
  }
  return ED_OK;
}

struct DevBuf {
  Ctx* ctx = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  int alloc(Ctx* c, size_t b) {
    ctx = c;
    bytes = b ? b : 1;
    return dev_alloc(c, &p, bytes);
  }
  ~DevBuf() {
    if (p) dev_free(ctx, p, bytes);
  }
};

// Carves typed arrays out of one allocation (256-byte aligned).
struct Carve {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

size_t coef_bytes(int mmax, int k) {
  size_t m2 = (size_t)mmax + 2;
  return 256 * 64 + m2 * 8 * 24 + (size_t)k * m2 * 8 * 10 + 4096;
}

Coefs carve_coefs(Carve& cv, int mmax) {
  Coefs c;
  size_t m2 = (size_t)mmax + 2;
  c.alpha = cv.take<double>(m2);
  c.beta = cv.take<double>(m2);
  c.nal_d = cv.take<double>(m2);
  c.nal_f = cv.take<float2>(m2);
  c.nbe_d = cv.take<double>(m2);
  c.nbe_f = cv.take<float2>(m2);
  c.inv_d = cv.take<double>(m2);
  c.inv_f = cv.take<float2>(m2);
  c.h_d = cv.take<double>(m2);
  c.h_f = cv.take<float2>(m2);
  c.scale = cv.take<double>(1);
  c.exhausted = cv.take<int>(1);
  c.out = cv.take<double>(64);
  c.sigma = cv.take<double>(m2);
  c.ua_d = cv.take<double>(m2);
  c.ua_f = cv.take<float2>(m2);
  c.ub_d = cv.take<double>(m2);
  c.ub_f = cv.take<float2>(m2);
  c.uc_d = cv.take<double>(m2);
  c.uc_f = cv.take<float2>(m2);
  c.step = cv.take<int>(1);
  return c;
}

__global__ void k_init_coefs(Coefs c, int m2) {
  for (int i = threadIdx.x; i < m2; i += blockDim.x) {
    c.alpha[i] = 0;
    c.beta[i] = 0;
    c.nal_d[i] = 0;
    c.nal_f[i] = make_float2(0, 0);
    c.nbe_d[i] = 0;
    c.nbe_f[i] = make_float2(0, 0);
    c.inv_d[i] = 0;
    c.inv_f[i] = make_float2(0, 0);
    c.h_d[i] = 0;
    c.h_f[i] = make_float2(0, 0);
    c.sigma[i] = 0;
    c.ua_d[i] = c.ub_d[i] = c.uc_d[i] = 0;
    c.ua_f[i] = c.ub_f[i] = c.uc_f[i] = make_float2(0, 0);
  }
  if (threadIdx.x == 0) {
    *c.scale = 0.0;
    *c.exhausted = -1;
    *c.step = 0;
  }
}

// Solve the m x m tridiagonal problem for its k lowest pairs.
int tridiag(Ctx* ctx, cudaStream_t st, const Coefs& c, int m, int k, double beta_m, double* theta,
            double* S, float2* Sf, int ldS, double* resid, double* work) {
  k_tri_eig<<<k, 32, 0, st>>>(c.alpha, c.beta, m, theta);
  k_tri_vec<<<k, 32, 0, st>>>(c.alpha, c.beta, m, theta, S, ldS, work);
  k_tri_finish<<<1, 128, 0, st>>>(theta, k, m, beta_m, S, ldS, Sf, resid);
  ED_LAUNCH_CHECK();
  (void)ctx;
  return ED_OK;
}

template <class V>
int lanczos_impl(Sector* s, const ed_lanczos_opts* o, double* evals, void* evecs, ed_lanczos_info* info,
                 cudaStream_t st) {
  auto t_start = std::chrono::steady_clock::now();
  Ctx* ctx = s->ctx;
  const uint64_t n = s->dim;
  const int k = o->k;
  const int reorth = o->reorth ? 1 : 0;
  int mmax = (int)std::min<uint64_t>((uint64_t)o->max_iter, n);
  if (mmax < 1) mmax = 1;
  const int check_every = std::max(1, o->check_every);
  const int kk = std::min<int>(k, (int)n);

  // workspace: basis (mmax + 1 vectors with reorthogonalisation, else 3), w
  size_t eb = sizeof(V);
  int nvec_store = reorth ? (mmax + 1) : 3;
  DevBuf vb, cb, v0b;
  // basis slots padded to 32 elements, so that each starts 16-byte aligned
  const uint64_t ld = pad32(n);
  ED_TRY(vb.alloc(ctx, ((size_t)nvec_store + 1) * ld * eb));
  ED_TRY(cb.alloc(ctx, coef_bytes(mmax, std::max(kk, 1))));
  V* Vbase = static_cast<V*>(vb.p);
  V* w = Vbase + (size_t)nvec_store * ld;
  if (!reorth) ED_TRY(v0b.alloc(ctx, n * eb));
  Carve cv{static_cast<char*>(cb.p)};
  Coefs c = carve_coefs(cv, mmax);
  int ldS = mmax + 1;
  double* theta = cv.take<double>(ED_MAX_K);
  double* resid = cv.take<double>(ED_MAX_K);
  double* Sd = cv.take<double>((size_t)ldS * std::max(kk, 1));
  float2* Sf = cv.take<float2>((size_t)ldS * std::max(kk, 1));
  double* twork = cv.take<double>((size_t)6 * ldS * std::max(kk, 1));

  Work<V> W;
  W.ctx = ctx;
  W.st = st;
  W.n = n;
  W.grid = (uint32_t)std::min<uint64_t>((n + kRedThreads - 1) / kRedThreads, (uint64_t)ctx->num_sms * 8);
  if (W.grid == 0) W.grid = 1;
  W.partial = ctx->d_red;
  W.c = c;
  uint32_t vgrid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 16);
  if (vgrid == 0) vgrid = 1;

  k_init_coefs<<<1, 256, 0, st>>>(c, mmax + 2);
  auto vec = [&](int j) -> V* { return reorth ? Vbase + (size_t)j * ld : Vbase + (size_t)(j % 3) * ld; };

  // start vector
  if (o->v0) {
    ED_TRY_CUDA(cudaMemcpyAsync(w, o->v0, n * eb, cudaMemcpyDeviceToDevice, st));
  } else {
    k_random<V><<<vgrid, 256, 0, st>>>(w, n, o->seed);
  }
  ED_TRY(dot_to(W, (const V*)w, (const V*)w, OP_NORM_INV, 0));
  k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(0), n, c, 0);
  ED_LAUNCH_CHECK();
  if (!reorth) ED_TRY_CUDA(cudaMemcpyAsync(v0b.p, vec(0), n * eb, cudaMemcpyDeviceToDevice, st));

  // one event pair per step to time the H*v launches
  std::vector<cudaEvent_t> evs(2 * (size_t)mmax);
  for (auto& e : evs) ED_TRY_CUDA(cudaEventCreate(&e));
  struct EvGuard {
    std::vector<cudaEvent_t>* v;
    ~EvGuard() {
      for (auto e : *v) cudaEventDestroy(e);
    }
  } evguard{&evs};
  double apply_ms = 0.0;
  int n_timed = 0;

  std::vector<double> h_theta(ED_MAX_K), h_res(ED_MAX_K);
  int m = 0;          // current Krylov dimension
  int n_conv = 0;
  double beta_last = 0.0;
  bool done = false;
  int status = ED_OK;
  int restarts = 0;
  const double thr = 1e-13;
  int j = 0;
  bool exhausted = false;
  while (!done) {
    exhausted = false;
    for (; j < mmax; ++j) {
      V* vj = vec(j);
      V* vjm = (j > 0) ? vec(j - 1) : nullptr;
      ED_TRY_CUDA(cudaEventRecord(evs[2 * j], st));
      ED_TRY(apply_h(s, vj, w, st));
      ED_TRY_CUDA(cudaEventRecord(evs[2 * j + 1], st));
      n_timed = std::max(n_timed, j + 1);
      ED_TRY(dot_to(W, (const V*)vj, (const V*)w, OP_ALPHA, j));
      k_lz_update<V><<<vgrid, 256, 0, st>>>(w, vj, vjm, n, c, j);
      ED_LAUNCH_CHECK();
      if (reorth) ED_TRY(cgs2(W, (const V*)Vbase, ld, j + 1, w));
      ED_TRY(dot_to(W, (const V*)w, (const V*)w, OP_BETA, j + 1, thr));
      k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(j + 1), n, c, j + 1);
      ED_LAUNCH_CHECK();
      m = j + 1;
      bool check = ((m % check_every) == 0) || (m == mmax) || (n <= 4096);
      if (!check) continue;
      // exhausted Krylov space?
      int ex = -1;
      ED_TRY_CUDA(cudaMemcpyAsync(ctx->h_red, c.exhausted, sizeof(int), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      std::memcpy(&ex, ctx->h_red, sizeof(int));
      if (ex >= 0) {
        m = ex;  // T is complete up to here; later steps are discarded
        exhausted = true;
        ++j;
        break;
      }
      int kc = std::min(kk, m);
      ED_TRY(tridiag(ctx, st, c, m, kc, 0.0, theta, Sd, Sf, ldS, resid, twork));
      // residuals use beta_{m}
      ED_TRY_CUDA(cudaMemcpyAsync(ctx->h_red, c.beta + m, sizeof(double), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaMemcpyAsync(ctx->h_red + 1, theta, kc * sizeof(double), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      beta_last = ctx->h_red[0];
      std::memcpy(h_theta.data(), ctx->h_red + 1, kc * sizeof(double));
      // residual = beta_m * |last component|
      std::vector<double> last(kc);
      for (int i = 0; i < kc; ++i)
        ED_TRY_CUDA(cudaMemcpyAsync(&last[i], Sd + (size_t)i * ldS + m - 1, sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      n_conv = 0;
      for (int i = 0; i < kc; ++i) {
        h_res[i] = std::fabs(beta_last * last[i]);
        if (h_res[i] <= o->tol * std::max(1.0, std::fabs(h_theta[i])) && n_conv == i) ++n_conv;
      }
      if (kc >= kk && n_conv >= kk) {
        ++j;
        done = true;
        break;
      }
    }
    if (done) break;
    if (!exhausted && j >= mmax && m >= mmax) {
      status = ED_ERR_NOT_CONVERGED;
      break;
    }
    // Krylov space exhausted at m: finished if it spans the sector or we have
    // k values already; otherwise restart from a fresh orthogonal vector.
    {
      int kc = std::min(kk, m);
      ED_TRY(tridiag(ctx, st, c, m, kc, 0.0, theta, Sd, Sf, ldS, resid, twork));
      ED_TRY_CUDA(cudaMemcpyAsync(ctx->h_red, theta, kc * sizeof(double), cudaMemcpyDeviceToHost, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      std::memcpy(h_theta.data(), ctx->h_red, kc * sizeof(double));
      for (int i = 0; i < kc; ++i) h_res[i] = 0.0;
      n_conv = kc;
      beta_last = 0.0;
      if (!reorth || (uint64_t)m >= n || m >= mmax || kc >= kk) {
        done = true;
        break;
      }
      // new random direction, orthogonalised against V[0..m)
      ++restarts;
      k_random<V><<<vgrid, 256, 0, st>>>(w, n, o->seed + 7919ull * restarts);
      ED_TRY(cgs2(W, (const V*)Vbase, ld, m, w));
      ED_TRY(dot_to(W, (const V*)w, (const V*)w, OP_NORM_INV, 1));
      k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(m), n, c, 1);
      // beta[m] = 0 splits T; reset the exhaustion flag
      double zero = 0.0;
      int neg = -1;
      ED_TRY_CUDA(cudaMemcpyAsync(c.beta + m, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
      ED_TRY_CUDA(cudaMemcpyAsync(c.nbe_d + m, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
      float2 zf = make_float2(0.f, 0.f);
      ED_TRY_CUDA(cudaMemcpyAsync(c.nbe_f + m, &zf, sizeof(float2), cudaMemcpyHostToDevice, st));
      ED_TRY_CUDA(cudaMemcpyAsync(c.exhausted, &neg, sizeof(int), cudaMemcpyHostToDevice, st));
      ED_TRY_CUDA(cudaStreamSynchronize(st));
      j = m;
    }
  }

  int kc = std::min(kk, m);
  for (int i = 0; i < kc; ++i) evals[i] = h_theta[i];
  for (int i = kc; i < k; ++i) evals[i] = NAN;
  if (info) {
    info->iters = m;
    info->n_converged = std::min(n_conv, kc);
    for (int i = 0; i < ED_MAX_K; ++i) info->residual[i] = (i < kc) ? h_res[i] : 0.0;
  }
  if (evecs && kc > 0) {
    // S for the final m
    ED_TRY(tridiag(ctx, st, c, m, kc, 0.0, theta, Sd, Sf, ldS, resid, twork));
    V* out = static_cast<V*>(evecs);
    if (reorth) {
      for (int i0 = 0; i0 < kc; i0 += 8)
        k_ritz<V, 8><<<vgrid, 256, 0, st>>>(Vbase, ld, m, Sd, Sf, ldS, i0, std::min(8, kc - i0), out, n, 0);
      ED_LAUNCH_CHECK();
    } else {
      // second pass: regenerate v_j with the stored alpha, beta and accumulate
      ED_TRY_CUDA(cudaMemsetAsync(out, 0, (size_t)kc * n * eb, st));
      ED_TRY_CUDA(cudaMemcpyAsync(vec(0), v0b.p, n * eb, cudaMemcpyDeviceToDevice, st));
      for (int jj = 0; jj < m; ++jj) {
        for (int i0 = 0; i0 < kc; i0 += 8)
          k_ritz<V, 8><<<vgrid, 256, 0, st>>>(vec(jj), n, 1, Sd + jj, Sf + jj, ldS, i0, std::min(8, kc - i0), out,
                                              n, 1);
        if (jj + 1 == m) break;
        ED_TRY(apply_h(s, vec(jj), w, st));
        k_lz_update<V><<<vgrid, 256, 0, st>>>(w, vec(jj), jj > 0 ? vec(jj - 1) : nullptr, n, c, jj);
        k_scale<V><<<vgrid, 256, 0, st>>>(w, vec(jj + 1), n, c, jj + 1);
        ED_LAUNCH_CHECK();
      }
    }
  }
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  for (int q = 0; q < n_timed; ++q) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, evs[2 * q], evs[2 * q + 1]) == cudaSuccess) apply_ms += ms;
  }
  if (info) info->apply_ms = apply_ms;
  if (info)
    info->total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (status != ED_OK) set_error("Lanczos did not converge in %d steps", mmax);
  return status;
}

}  // namespace

}  // namespace ed
