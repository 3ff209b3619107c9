// Batched Lanczos over many sectors at once: every active sector advances one
// Lanczos step per replay of a single CUDA graph, and each kernel of the step
// (one H*v over all sectors, the dot products, the update, CGS2 full
// reorthogonalisation, the norm and the scaling) is ONE launch over a device
// work list of (sector, chunk of consecutive elements) items (up to 8192
// elements by default; ed_batch_autotune picks the chunk that packs the sectors
// fastest).  The step index lives in
// device memory, so the graph captured once serves every step; sectors that
// converge are switched off in a device flag array and their items return at
// once.  This packs the many small sectors of a model (the 169 sectors of the
// N_s = 12 three-orbital impurity range from 1 to 853,776 states) into launches
// that fill the GPU, where one sector at a time would leave it idle.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "apply_common.h"
#include "tri_common.h"
#include "vec16.h"

struct ed_batch;

namespace ed {

namespace {

// Untuned chunk: the largest power of two from 256 to 8192 that still cuts the
// batch into at least eight items per SM (at N_s = 12, all 169 sectors: 8192,
// 2.4 ms per FP64 step against 3.3 ms with 1024-element items).
uint32_t default_chunk(const std::vector<uint64_t>& dims, int sms) {
  const uint64_t want = 8ull * (uint64_t)std::max(sms, 1);
  for (uint32_t c = 8192; c > 256; c >>= 1) {
    uint64_t items = 0;
    for (uint64_t d : dims) items += (d + c - 1) / c;
    if (items >= want) return c;
  }
  return 256;
}
constexpr int kBT = 256;           // threads per block
constexpr int kKB = 8;             // basis vectors per multi-dot register group

struct JobDev {
  SectorView S;
  const uint32_t* ub;
  const uint32_t* db;
  uint64_t off;   // element offset inside every vector slot
  uint64_t dim;
  uint32_t item0, item1;
  uint64_t seed_mix;  // start-vector hash term of the job (the same for a job alone or among others)
};

struct BatchDev {
  const JobDev* jobs;
  const uint2* items;  // {job, first element}
  uint32_t n_items;
  uint32_t chunk;      // elements per item
  int n_jobs;
  uint64_t tot;        // elements per vector slot
  int* active;         // [n_jobs]
  int* step;           // current step j
  int ms;              // coefficient row length per job (max_iter + 2)
  double* alpha;       // [job][ms]
  double* beta;
  double* nal_d;
  float2* nal_f;
  double* nbe_d;
  float2* nbe_f;
  double* inv_d;
  float2* inv_f;
  double* h_d;         // [job][ms] negated CGS projections
  float2* h_f;
  double* scale;       // [job]
  int* exhausted;      // [job]
  double* partial;     // [ms][n_items]
  double thr;
};

template <class V>
struct BAcc;
template <>
struct BAcc<double> { using T = double; };
template <>
struct BAcc<float2> { using T = float2; };
template <>
struct BAcc<float> { using T = float2; };

__device__ __forceinline__ void bmac(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void bmac(float2& a, float2 x, float2 y) { df_mac(a, x, y); }
__device__ __forceinline__ void bmac(float2& a, float x, float y) { df_mac1(a, make_float2(x, 0.f), y); }
__device__ __forceinline__ double badd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 badd(float2 a, float2 b) { return df_add(a, b); }
__device__ __forceinline__ double bshfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 bshfl(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double bd(double a) { return a; }
__device__ __forceinline__ double bd(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ double bacc_of(double x) { return x; }
__device__ __forceinline__ float2 bacc_of(float2 x) { return x; }
__device__ __forceinline__ float2 bacc_of(float x) { return make_float2(x, 0.f); }
__device__ __forceinline__ void bcmac(double& a, const double* cd, const float2*, size_t k, double x) {
  a = fma(cd[k], x, a);
}
__device__ __forceinline__ void bcmac(float2& a, const double*, const float2* cf, size_t k, float2 x) {
  df_mac(a, cf[k], x);
}
__device__ __forceinline__ void bcmac(float2& a, const double*, const float2* cf, size_t k, float x) {
  df_mac1(a, cf[k], x);
}
__device__ __forceinline__ double bstore(double a, double*) { return a; }
__device__ __forceinline__ float2 bstore(float2 a, float2*) { return df_norm(a); }
__device__ __forceinline__ float bstore(float2 a, float*) { return __fadd_rn(a.x, a.y); }

template <class A>
__device__ __forceinline__ A bblock_sum(A v) {
  __shared__ A sh[kBT / 32];
  for (int o = 16; o > 0; o >>= 1) v = badd(v, bshfl(v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < kBT / 32) ? sh[lane] : A{};
    for (int o = 16; o > 0; o >>= 1) v = badd(v, bshfl(v, o));
  }
  return v;
}

// ---------------------------------------------------------------- step kernels
// w = H V_j for every active sector.
template <class P>
__global__ void __launch_bounds__(kBT) k_b_apply(BatchDev B, const typename P::V* __restrict__ Vb,
                                                 typename P::V* __restrict__ w) {
  using V = typename P::V;
  const int j = *B.step;
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    if (!B.active[item.x]) continue;
    const JobDev& J = B.jobs[item.x];
    const V* x = Vb + (uint64_t)j * B.tot + J.off;
    V* y = w + J.off;
    const uint32_t Dd = J.S.D_dn;
    const uint64_t e1 = min((uint64_t)item.y + B.chunk, J.dim);
    for (uint64_t e = item.y + threadIdx.x; e < e1; e += kBT) {
      const uint32_t u = (uint32_t)(e / Dd), d = (uint32_t)(e % Dd);
      const V* xr = x + (uint64_t)u * Dd;
      auto xrow = [xr](uint32_t q) { return xr[q]; };
      y[e] = element<P>(J.S, x, u, J.ub[u], d, J.db[d], row_e<P>(J.S, u), xrow);
    }
  }
}

// partial[slot * n_items + it] = <a, b> over the item, a/b selected by mode:
// 0: <V_j, w>   1: <w, w>
template <class V>
__global__ void __launch_bounds__(kBT) k_b_dot(BatchDev B, const V* __restrict__ Vb, const V* __restrict__ w,
                                               int mode) {
  using A = typename BAcc<V>::T;
  const int j = *B.step;
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    if (!B.active[item.x]) continue;  // k_b_finish reads no partial of a converged sector
    A acc{};
    const JobDev& J = B.jobs[item.x];
    const uint64_t e1 = min((uint64_t)item.y + B.chunk, J.dim);
    const V* a = (mode == 0) ? Vb + (uint64_t)j * B.tot + J.off : w + J.off;
    const V* b = w + J.off;
    for (uint64_t e = item.y + threadIdx.x; e < e1; e += kBT) bmac(acc, a[e], b[e]);
    acc = bblock_sum(acc);
    if (threadIdx.x == 0) B.partial[it] = bd(acc);
  }
}

// The CGS2 kernels read sixteen-byte vectors (vec16.h).  Vector slots and
// sector offsets are padded to 32 elements and work items start at multiples
// of the chunk, so every item starts 16-byte aligned.

// Block sums of up to kKB accumulators with one barrier: each warp reduces
// every accumulator (butterfly), then warp q reduces accumulator q over the
// warps in the same butterfly order as bblock_sum; lane 0 of warp q stores it.
template <class A>
__device__ __forceinline__ void bblock_sum_group(A (&acc)[kKB], int nq, double* out, uint64_t stride) {
  __shared__ A sh[kKB][kBT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // the previous group's readers are done with sh
#pragma unroll
  for (int q = 0; q < kKB; ++q) {
    A v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v = badd(v, bshfl(v, o));
    if (lane == 0) sh[q][w] = v;
  }
  __syncthreads();
  static_assert(kBT / 32 >= kKB, "one warp per accumulator");
  if (w < nq) {
    A v = (lane < kBT / 32) ? sh[w][lane] : A{};
    for (int o = 16; o > 0; o >>= 1) v = badd(v, bshfl(v, o));
    if (lane == 0) out[(uint64_t)w * stride] = bd(v);
  }
}

// partial[k * n_items + it] = <V_k, w>, k <= j.  Sixteen-byte loads keep
// (kKB + 1) x 16 bytes per thread in flight; the item's ragged tail (fewer
// than one vector) is read element by element.
template <class V>
__global__ void __launch_bounds__(kBT) k_b_multidot(BatchDev B, const V* __restrict__ Vb, const V* __restrict__ w) {
  using A = typename BAcc<V>::T;
  using W16 = Vec16<V>;
  using VT = typename W16::T;
  constexpr int N = W16::N;
  const int j = *B.step;
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    if (!B.active[item.x]) continue;  // k_b_finish reads no partial of a converged sector
    const JobDev& J = B.jobs[item.x];
    const uint64_t e0 = J.off + item.y;
    const uint64_t n = min((uint64_t)item.y + B.chunk, J.dim) - item.y;
    const uint64_t nv = n / N;
    const VT* wv = reinterpret_cast<const VT*>(w + e0);
    for (int k0 = 0; k0 <= j; k0 += kKB) {
      const int nq = min(kKB, j + 1 - k0);
      A acc[kKB];
#pragma unroll
      for (int q = 0; q < kKB; ++q) acc[q] = A{};
      {
        const V* vk = Vb + (uint64_t)k0 * B.tot + e0;
        for (uint64_t t = threadIdx.x; t < nv; t += kBT) {
          const VT wq = wv[t];
          VT vq[kKB];
#pragma unroll
          for (int q = 0; q < kKB; ++q)
            if (q < nq) vq[q] = __ldg(reinterpret_cast<const VT*>(vk + (uint64_t)q * B.tot) + t);
#pragma unroll
          for (int q = 0; q < kKB; ++q)
            if (q < nq) {
#pragma unroll
              for (int i = 0; i < N; ++i) bmac(acc[q], W16::get(vq[q], i), W16::get(wq, i));
            }
        }
        for (uint64_t e = nv * N + threadIdx.x; e < n; e += kBT) {
          const V we = w[e0 + e];
#pragma unroll
          for (int q = 0; q < kKB; ++q)
            if (q < nq) bmac(acc[q], vk[(uint64_t)q * B.tot + e], we);
        }
      }
      bblock_sum_group(acc, nq, B.partial + (uint64_t)k0 * B.n_items + it, B.n_items);
    }
  }
}

enum { BF_ALPHA = 0, BF_BETA = 1, BF_NEGH = 2, BF_NORM0 = 3 };

// One block per (job, k): sum the job's item partials of row k and store.
__global__ void __launch_bounds__(kBT) k_b_finish(BatchDev B, int op) {
  const int job = blockIdx.x, k = blockIdx.y;
  const int j = *B.step;
  if (!B.active[job]) return;
  if (op == BF_NEGH && k > j) return;
  const JobDev& J = B.jobs[job];
  const int row = (op == BF_NEGH) ? k : 0;
  double v = 0.0;
  for (uint32_t it = J.item0 + threadIdx.x; it < J.item1; it += kBT) v += B.partial[(uint64_t)row * B.n_items + it];
  v = bblock_sum(v);
  if (threadIdx.x != 0) return;
  const size_t base = (size_t)job * B.ms;
  switch (op) {
    case BF_ALPHA:
      B.alpha[base + j] = v;
      B.nal_d[base + j] = -v;
      B.nal_f[base + j] = df_from_double(-v);
      B.scale[job] = fmax(B.scale[job], fabs(v));
      break;
    case BF_BETA: {
      const double b = sqrt(fmax(v, 0.0));
      const double sc = fmax(B.scale[job], b);
      B.scale[job] = sc;
      const bool dead = !(b > B.thr * fmax(sc, 1.0));
      if (dead && B.exhausted[job] < 0) B.exhausted[job] = j + 1;
      B.beta[base + j + 1] = dead ? 0.0 : b;
      B.nbe_d[base + j + 1] = dead ? 0.0 : -b;
      B.nbe_f[base + j + 1] = df_from_double(dead ? 0.0 : -b);
      const double inv = dead ? 0.0 : 1.0 / b;
      B.inv_d[base + j + 1] = inv;
      B.inv_f[base + j + 1] = df_from_double(inv);
      break;
    }
    case BF_NEGH:
      B.h_d[base + k] = -v;
      B.h_f[base + k] = df_from_double(-v);
      break;
    case BF_NORM0: {
      const double b = sqrt(fmax(v, 0.0));
      const double inv = b > 0.0 ? 1.0 / b : 0.0;
      B.inv_d[base] = inv;
      B.inv_f[base] = df_from_double(inv);
      B.beta[base] = 0.0;
      break;
    }
  }
}

// mode 0: w += nal_j V_j + nbe_j V_{j-1}
// mode 2: V_{j+1} = inv_{j+1} w        mode 3: V_0 = inv_0 w
template <class V>
__global__ void __launch_bounds__(kBT) k_b_axpy(BatchDev B, V* __restrict__ Vb, V* __restrict__ w, int mode) {
  using A = typename BAcc<V>::T;
  const int j = *B.step;
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    if (!B.active[item.x]) continue;
    const JobDev& J = B.jobs[item.x];
    const size_t base = (size_t)item.x * B.ms;
    const uint64_t e1 = min((uint64_t)item.y + B.chunk, J.dim);
    for (uint64_t e = item.y + threadIdx.x; e < e1; e += kBT) {
      const uint64_t g = J.off + e;
      if (mode == 0) {
        A a = bacc_of(w[g]);
        bcmac(a, B.nal_d, B.nal_f, base + j, Vb[(uint64_t)j * B.tot + g]);
        if (j > 0) bcmac(a, B.nbe_d, B.nbe_f, base + j, Vb[(uint64_t)(j - 1) * B.tot + g]);
        w[g] = bstore(a, w);
      } else {
        const int s = (mode == 2) ? j + 1 : 0;
        A a{};
        bcmac(a, B.inv_d, B.inv_f, base + s, w[g]);
        Vb[(uint64_t)s * B.tot + g] = bstore(a, Vb);
      }
    }
  }
}

// CGS2 update w += sum_{k<=j} h_k V_k for every active sector: sixteen-byte
// loads of w and of each V_k, each element's terms in the order k = 0..j
// (the ragged tail of an item element by element).
template <class V>
__global__ void __launch_bounds__(kBT) k_b_cgs_update(BatchDev B, const V* __restrict__ Vb, V* __restrict__ w) {
  using A = typename BAcc<V>::T;
  using W16 = Vec16<V>;
  using VT = typename W16::T;
  constexpr int N = W16::N;
  const int j = *B.step;
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    if (!B.active[item.x]) continue;
    const JobDev& J = B.jobs[item.x];
    const size_t base = (size_t)item.x * B.ms;
    const uint64_t e0 = J.off + item.y;
    const uint64_t n = min((uint64_t)item.y + B.chunk, J.dim) - item.y;
    const uint64_t nv = n / N;
    VT* wv = reinterpret_cast<VT*>(w + e0);
    const V* v0 = Vb + e0;
    for (uint64_t t = threadIdx.x; t < nv; t += kBT) {
      const VT wq = wv[t];
      A a[N];
#pragma unroll
      for (int i = 0; i < N; ++i) a[i] = bacc_of(W16::get(wq, i));
#pragma unroll 4
      for (int k = 0; k <= j; ++k) {
        const VT vq = __ldg(reinterpret_cast<const VT*>(v0 + (uint64_t)k * B.tot) + t);
#pragma unroll
        for (int i = 0; i < N; ++i) bcmac(a[i], B.h_d, B.h_f, base + k, W16::get(vq, i));
      }
      VT o;
#pragma unroll
      for (int i = 0; i < N; ++i) W16::set(o, i, bstore(a[i], w));
      wv[t] = o;
    }
    for (uint64_t e = nv * N + threadIdx.x; e < n; e += kBT) {
      A a = bacc_of(w[e0 + e]);
      for (int k = 0; k <= j; ++k) bcmac(a, B.h_d, B.h_f, base + k, v0[(uint64_t)k * B.tot + e]);
      w[e0 + e] = bstore(a, w);
    }
  }
}

__global__ void k_b_step_inc(int* step) { *step += 1; }

__device__ __forceinline__ uint64_t bmix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ void bset(double& o, float u) { o = (double)u; }
__device__ __forceinline__ void bset(float2& o, float u) { o = make_float2(u, 0.f); }
__device__ __forceinline__ void bset(float& o, float u) { o = u; }

// Seeded start vectors of every sector (uniform(-1, 1) per element and sector).
template <class V>
__global__ void k_b_random(BatchDev B, V* __restrict__ w, uint64_t seed) {
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    const JobDev& J = B.jobs[item.x];
    const uint64_t e1 = min((uint64_t)item.y + B.chunk, J.dim);
    for (uint64_t e = item.y + threadIdx.x; e < e1; e += kBT) {
      const uint64_t r = bmix(seed * 0x2545f4914f6cdd1dull + J.seed_mix + e);
      bset(w[J.off + e], (float)((r >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f);
    }
  }
}

// Ritz vectors of every job: out_q[i * dim + e] = sum_{j < m_q} S[q][i][j] V_j[e]
// for i < min(k_q, m_q); jobs whose output pointer is NULL are skipped.
__device__ __forceinline__ void rmac(double& a, double s, float2, double v) { a = fma(s, v, a); }
__device__ __forceinline__ void rmac(float2& a, double, float2 s, float2 v) { df_mac(a, s, v); }
__device__ __forceinline__ void rmac(float2& a, double, float2 s, float v) { df_mac1(a, s, v); }
__device__ __forceinline__ double rout(double a, double*) { return a; }
__device__ __forceinline__ float2 rout(float2 a, float2*) { return df_norm(a); }
__device__ __forceinline__ float rout(float2 a, float*) { return __fadd_rn(a.x, a.y); }

template <class V>
__global__ void k_b_ritz(BatchDev B, const V* __restrict__ Vb, const double* __restrict__ S,
                         const float2* __restrict__ Sf, const int* __restrict__ mj, const int* __restrict__ kj,
                         int kmax, V* const* __restrict__ outs) {
  using A = typename BAcc<V>::T;
  for (uint32_t it = blockIdx.x; it < B.n_items; it += gridDim.x) {
    const uint2 item = B.items[it];
    V* out = outs[item.x];
    if (!out) continue;
    const JobDev& J = B.jobs[item.x];
    const int m = mj[item.x], kq = min(kj[item.x], m);
    const uint64_t e1 = min((uint64_t)item.y + B.chunk, J.dim);
    for (uint64_t e = item.y + threadIdx.x; e < e1; e += kBT)
      for (int i = 0; i < kq; ++i) {
        const size_t row = ((size_t)item.x * kmax + i) * B.ms;
        A acc{};
        for (int j = 0; j < m; ++j) rmac(acc, S[row + j], Sf[row + j], Vb[(uint64_t)j * B.tot + J.off + e]);
        out[(uint64_t)i * J.dim + e] = rout(acc, out);
      }
  }
}

// --------------------------------------------------- batched tridiagonal solve
__global__ void k_bt_eig(const double* __restrict__ alpha, const double* __restrict__ beta, int ms,
                         const int* __restrict__ mj, const int* __restrict__ kj, int kmax, double* __restrict__ theta) {
  const int i = blockIdx.x, job = blockIdx.y;
  if (i >= kj[job] || i >= mj[job]) return;
  tri_eig_one(alpha + (size_t)job * ms, beta + (size_t)job * ms, mj[job], i, theta + (size_t)job * kmax);
}

__global__ void k_bt_vec(const double* __restrict__ alpha, const double* __restrict__ beta, int ms,
                         const int* __restrict__ mj, const int* __restrict__ kj, int kmax, const double* __restrict__ theta,
                         double* __restrict__ S, double* __restrict__ work) {
  const int i = blockIdx.x, job = blockIdx.y;
  if (threadIdx.x != 0 || i >= kj[job] || i >= mj[job]) return;
  const int ldS = ms;
  tri_vec_one(alpha + (size_t)job * ms, beta + (size_t)job * ms, mj[job], theta + (size_t)job * kmax,
              S + (size_t)job * kmax * ldS, ldS, work + (size_t)job * kmax * 6 * ldS, i);
}

__global__ void k_bt_finish(const double* __restrict__ beta, int ms, const int* __restrict__ mj,
                            const int* __restrict__ kj, int kmax, const double* __restrict__ theta,
                            double* __restrict__ S, float2* __restrict__ Sf, double* __restrict__ resid) {
  const int job = blockIdx.x;
  const int m = mj[job], k = min(kj[job], mj[job]);
  if (m < 1 || k < 1) return;
  const int ldS = ms;
  tri_finish_block(theta + (size_t)job * kmax, k, m, beta[(size_t)job * ms + m], S + (size_t)job * kmax * ldS, ldS,
                   Sf + (size_t)job * kmax * ldS, resid + (size_t)job * kmax);
}

}  // namespace

struct Batch {
  Ctx* ctx = nullptr;
  int prec = 0;
  int n_jobs = 0;
  std::vector<std::unique_ptr<Sector>> sectors;
  std::vector<JobDev> hjobs;
  std::vector<uint2> hitems;
  uint64_t tot = 0;
  uint32_t chunk = 0;
  JobDev* djobs = nullptr;
  uint2* ditems = nullptr;   // owned separately: rebuilt when the chunk changes
  size_t ditems_bytes = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  cudaStream_t stream = nullptr;
  template <class T>
  int alloc(T** p, size_t n) {
    int st = dev_alloc(ctx, reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
    if (st == ED_OK) allocs.push_back({(void*)*p, std::max<size_t>(n, 1) * sizeof(T)});
    return st;
  }
  // Cut every sector into items of `c` elements and upload the list.
  int set_chunk(uint32_t c) {
    hitems.clear();
    for (size_t q = 0; q < hjobs.size(); ++q) {
      hjobs[q].item0 = (uint32_t)hitems.size();
      for (uint64_t e = 0; e < hjobs[q].dim; e += c) hitems.push_back(make_uint2((unsigned)q, (unsigned)e));
      hjobs[q].item1 = (uint32_t)hitems.size();
    }
    if (ditems) dev_free(ctx, ditems, ditems_bytes);
    ditems = nullptr;
    ditems_bytes = std::max<size_t>(hitems.size(), 1) * sizeof(uint2);
    int st = dev_alloc(ctx, reinterpret_cast<void**>(&ditems), ditems_bytes);
    if (st != ED_OK) {
      ditems_bytes = 0;
      return st;
    }
    ED_TRY_CUDA(cudaMemcpy(djobs, hjobs.data(), sizeof(JobDev) * hjobs.size(), cudaMemcpyHostToDevice));
    ED_TRY_CUDA(cudaMemcpy(ditems, hitems.data(), sizeof(uint2) * hitems.size(), cudaMemcpyHostToDevice));
    chunk = c;
    return ED_OK;
  }
  void release() {
    for (auto& a : allocs) dev_free(ctx, a.first, a.second);
    allocs.clear();
    if (ditems) dev_free(ctx, ditems, ditems_bytes);
    ditems = nullptr;
    for (auto& s : sectors) free_sector(s.get());
    sectors.clear();
    if (stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

namespace {

struct RunBufs {
  Batch* b;
  std::vector<std::pair<void*, size_t>> allocs;
  template <class T>
  int alloc(T** p, size_t n) {
    int st = dev_alloc(b->ctx, reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
    if (st == ED_OK) allocs.push_back({(void*)*p, std::max<size_t>(n, 1) * sizeof(T)});
    return st;
  }
  ~RunBufs() {
    for (auto& a : allocs) dev_free(b->ctx, a.first, a.second);
  }
};

// With ritz != NULL (one device pointer per job, NULL to skip a job) the k
// lowest Ritz vectors of each job are written there, k consecutive vectors of
// the job's dimension in the batch's format.
template <class P>
int batch_run(Batch* bt, const ed_lanczos_opts* o, double* evals, int* iters, ed_batch_info* info,
              cudaStream_t user, void* const* ritz = nullptr, int* conv = nullptr) {
  using V = typename P::V;
  auto t0 = std::chrono::steady_clock::now();
  Ctx* ctx = bt->ctx;
  const int J = bt->n_jobs;
  const int k = o->k;
  uint64_t maxdim = 0;
  for (auto& jb : bt->hjobs) maxdim = std::max(maxdim, jb.dim);
  const int mmax = (int)std::min<uint64_t>((uint64_t)o->max_iter, maxdim);
  const int ms = mmax + 2;
  const int check_every = std::max(1, o->check_every);
  cudaStream_t st = bt->stream;
  RunBufs R{bt, {}};
  V* Vb = nullptr;
  V* w = nullptr;
  ED_TRY(R.alloc(&Vb, (size_t)(mmax + 1) * bt->tot));
  ED_TRY(R.alloc(&w, bt->tot));
  BatchDev B{};
  B.jobs = bt->djobs;
  B.items = bt->ditems;
  B.n_items = (uint32_t)bt->hitems.size();
  B.chunk = bt->chunk;
  B.n_jobs = J;
  B.tot = bt->tot;
  B.ms = ms;
  B.thr = 1e-13;
  ED_TRY(R.alloc(&B.active, J));
  ED_TRY(R.alloc(&B.step, 1));
  ED_TRY(R.alloc(&B.alpha, (size_t)J * ms));
  ED_TRY(R.alloc(&B.beta, (size_t)J * ms));
  ED_TRY(R.alloc(&B.nal_d, (size_t)J * ms));
  ED_TRY(R.alloc(&B.nal_f, (size_t)J * ms));
  ED_TRY(R.alloc(&B.nbe_d, (size_t)J * ms));
  ED_TRY(R.alloc(&B.nbe_f, (size_t)J * ms));
  ED_TRY(R.alloc(&B.inv_d, (size_t)J * ms));
  ED_TRY(R.alloc(&B.inv_f, (size_t)J * ms));
  ED_TRY(R.alloc(&B.h_d, (size_t)J * ms));
  ED_TRY(R.alloc(&B.h_f, (size_t)J * ms));
  ED_TRY(R.alloc(&B.scale, J));
  ED_TRY(R.alloc(&B.exhausted, J));
  ED_TRY(R.alloc(&B.partial, (size_t)ms * B.n_items));
  // tridiagonal workspace
  const int kmax = std::max(1, k);
  double *theta = nullptr, *S = nullptr, *work = nullptr, *resid = nullptr;
  float2* Sf = nullptr;
  int *dm = nullptr, *dk = nullptr;
  ED_TRY(R.alloc(&theta, (size_t)J * kmax));
  ED_TRY(R.alloc(&resid, (size_t)J * kmax));
  ED_TRY(R.alloc(&S, (size_t)J * kmax * ms));
  ED_TRY(R.alloc(&Sf, (size_t)J * kmax * ms));
  ED_TRY(R.alloc(&work, (size_t)J * kmax * 6 * ms));
  ED_TRY(R.alloc(&dm, J));
  ED_TRY(R.alloc(&dk, J));

  ED_TRY_CUDA(cudaMemsetAsync(B.alpha, 0, sizeof(double) * J * ms, st));
  ED_TRY_CUDA(cudaMemsetAsync(B.beta, 0, sizeof(double) * J * ms, st));
  ED_TRY_CUDA(cudaMemsetAsync(B.nbe_d, 0, sizeof(double) * J * ms, st));
  ED_TRY_CUDA(cudaMemsetAsync(B.nbe_f, 0, sizeof(float2) * J * ms, st));
  ED_TRY_CUDA(cudaMemsetAsync(B.scale, 0, sizeof(double) * J, st));
  ED_TRY_CUDA(cudaMemsetAsync(B.exhausted, 0xff, sizeof(int) * J, st));  // -1
  ED_TRY_CUDA(cudaMemsetAsync(B.step, 0, sizeof(int), st));
  std::vector<int> h_active(J, 1), h_k(J), h_m(J, 0), done(J, 0), h_ex(J, -1);
  for (int q = 0; q < J; ++q) h_k[q] = (int)std::min<uint64_t>((uint64_t)k, bt->hjobs[q].dim);
  ED_TRY_CUDA(cudaMemcpyAsync(B.active, h_active.data(), sizeof(int) * J, cudaMemcpyHostToDevice, st));
  ED_TRY_CUDA(cudaMemcpyAsync(dk, h_k.data(), sizeof(int) * J, cudaMemcpyHostToDevice, st));

  const uint32_t grid = (uint32_t)std::min<uint64_t>(B.n_items, (uint64_t)ctx->num_sms * 8);
  const dim3 fgrid(J, 1), hgrid(J, ms);
  // start vectors: random, normalised per sector
  k_b_random<V><<<grid, kBT, 0, st>>>(B, w, o->seed);
  k_b_dot<V><<<grid, kBT, 0, st>>>(B, Vb, w, 1);
  k_b_finish<<<fgrid, kBT, 0, st>>>(B, BF_NORM0);
  k_b_axpy<V><<<grid, kBT, 0, st>>>(B, Vb, w, 3);
  ED_LAUNCH_CHECK();

  // one Lanczos step for all active sectors, captured once
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ED_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  k_b_apply<P><<<grid, kBT, 0, st>>>(B, Vb, w);
  k_b_dot<V><<<grid, kBT, 0, st>>>(B, Vb, w, 0);
  k_b_finish<<<fgrid, kBT, 0, st>>>(B, BF_ALPHA);
  k_b_axpy<V><<<grid, kBT, 0, st>>>(B, Vb, w, 0);
  for (int pass = 0; pass < 2; ++pass) {
    k_b_multidot<V><<<grid, kBT, 0, st>>>(B, Vb, w);
    k_b_finish<<<hgrid, kBT, 0, st>>>(B, BF_NEGH);
    k_b_cgs_update<V><<<grid, kBT, 0, st>>>(B, Vb, w);
  }
  k_b_dot<V><<<grid, kBT, 0, st>>>(B, Vb, w, 1);
  k_b_finish<<<fgrid, kBT, 0, st>>>(B, BF_BETA);
  k_b_axpy<V><<<grid, kBT, 0, st>>>(B, Vb, w, 2);
  k_b_step_inc<<<1, 1, 0, st>>>(B.step);
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(ce));
    return ED_ERR_CUDA;
  }
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    set_error("graph instantiation failed: %s", cudaGetErrorString(ce));
    return ED_ERR_CUDA;
  }
  struct ExecGuard {
    cudaGraphExec_t e;
    ~ExecGuard() { cudaGraphExecDestroy(e); }
  } eg{exec};

  std::vector<double> h_theta((size_t)J * kmax), h_res((size_t)J * kmax), h_bm(J);
  int steps = 0, replays = 0;
  for (int jstep = 0; jstep < mmax; ++jstep) {
    ED_TRY_CUDA(cudaGraphLaunch(exec, st));
    ++replays;
    steps = jstep + 1;
    const bool check = (steps % check_every == 0) || steps == mmax;
    if (!check) continue;
    ED_TRY_CUDA(cudaMemcpyAsync(h_ex.data(), B.exhausted, sizeof(int) * J, cudaMemcpyDeviceToHost, st));
    ED_TRY_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < J; ++q) {
      if (done[q]) continue;
      h_m[q] = (h_ex[q] >= 0) ? h_ex[q] : steps;
    }
    ED_TRY_CUDA(cudaMemcpyAsync(dm, h_m.data(), sizeof(int) * J, cudaMemcpyHostToDevice, st));
    k_bt_eig<<<dim3(kmax, J), 32, 0, st>>>(B.alpha, B.beta, ms, dm, dk, kmax, theta);
    k_bt_vec<<<dim3(kmax, J), 32, 0, st>>>(B.alpha, B.beta, ms, dm, dk, kmax, theta, S, work);
    k_bt_finish<<<J, 128, 0, st>>>(B.beta, ms, dm, dk, kmax, theta, S, Sf, resid);
    ED_LAUNCH_CHECK();
    ED_TRY_CUDA(cudaMemcpyAsync(h_theta.data(), theta, sizeof(double) * J * kmax, cudaMemcpyDeviceToHost, st));
    ED_TRY_CUDA(cudaMemcpyAsync(h_res.data(), resid, sizeof(double) * J * kmax, cudaMemcpyDeviceToHost, st));
    ED_TRY_CUDA(cudaStreamSynchronize(st));
    bool all = true;
    for (int q = 0; q < J; ++q) {
      if (done[q]) continue;
      const int kc = std::min(h_k[q], h_m[q]);
      bool conv = h_ex[q] >= 0;  // Krylov space exhausted: the T spectrum is exact
      if (!conv && kc >= h_k[q]) {
        conv = true;
        for (int i = 0; i < kc; ++i)
          if (h_res[(size_t)q * kmax + i] > o->tol * std::max(1.0, std::fabs(h_theta[(size_t)q * kmax + i]))) conv = false;
      }
      if (conv) {
        done[q] = 1;
        h_active[q] = 0;
        if (iters) iters[q] = h_m[q];
        for (int i = 0; i < k; ++i)
          evals[(size_t)q * k + i] = (i < kc) ? h_theta[(size_t)q * kmax + i] : NAN;
      } else {
        all = false;
      }
    }
    ED_TRY_CUDA(cudaMemcpyAsync(B.active, h_active.data(), sizeof(int) * J, cudaMemcpyHostToDevice, st));
    if (all) break;
  }
  int status = ED_OK;
  for (int q = 0; q < J; ++q)
    if (!done[q]) {
      status = ED_ERR_NOT_CONVERGED;
      const int kc = std::min(h_k[q], h_m[q]);
      if (iters) iters[q] = h_m[q];
      for (int i = 0; i < k; ++i) evals[(size_t)q * k + i] = (i < kc) ? h_theta[(size_t)q * kmax + i] : NAN;
    }
  if (conv)
    for (int q = 0; q < J; ++q) conv[q] = done[q];
  if (ritz) {
    V** douts = nullptr;
    ED_TRY(R.alloc(&douts, J));
    ED_TRY_CUDA(cudaMemcpyAsync(douts, ritz, sizeof(void*) * J, cudaMemcpyHostToDevice, st));
    k_b_ritz<V><<<grid, kBT, 0, st>>>(B, Vb, S, Sf, dm, dk, kmax, douts);
    ED_LAUNCH_CHECK();
  }
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->steps = steps;
    info->graph_replays = replays;
    info->n_sectors = J;
    info->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  (void)user;
  if (status != ED_OK) set_error("batched Lanczos: some sectors did not converge in %d steps", mmax);
  return status;
}

}  // namespace

}  // namespace ed

using namespace ed;

struct ed_batch {
  Batch b;
};

extern "C" int ed_batch_create(ed_ctx* ctx, const ed_model* model, int n_sectors, const int* n_up, const int* n_dn,
                               int prec, ed_batch** out) {
  if (!ctx || !model || !n_up || !n_dn || !out) ED_INVALID("NULL argument");
  if (n_sectors < 1) ED_INVALID("n_sectors must be >= 1");
  *out = nullptr;
  Ctx* c = ctx_of(ctx);
  std::unique_ptr<ed_batch> h(new ed_batch());
  Batch& b = h->b;
  b.ctx = c;
  b.prec = prec;
  b.n_jobs = n_sectors;
  ED_TRY_CUDA(cudaSetDevice(c->device));
  uint64_t off = 0;
  for (int q = 0; q < n_sectors; ++q) {
    std::unique_ptr<Sector> s(new Sector());
    int st = build_sector(c, model, n_up[q], n_dn[q], prec, s.get());
    if (st != ED_OK) {
      free_sector(s.get());
      b.release();
      return st;
    }
    JobDev jd{};
    jd.S = s->view();
    jd.ub = s->up.basis;
    jd.db = s->dn.basis;
    jd.off = off;
    jd.dim = s->dim;
    jd.seed_mix = (uint64_t)q * 0x9e3779b97f4a7c15ull;
    b.hjobs.push_back(jd);
    off += (s->dim + 31) & ~(uint64_t)31;
    b.sectors.push_back(std::move(s));
  }
  b.tot = off;
  int st = b.alloc(&b.djobs, b.hjobs.size());
  if (st == ED_OK) {
    std::vector<uint64_t> dims;
    for (const auto& j : b.hjobs) dims.push_back(j.dim);
    st = b.set_chunk(default_chunk(dims, c->num_sms));
  }
  if (st != ED_OK) {
    b.release();
    return st;
  }
  if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess) {
    b.release();
    set_error("batch set-up copy failed");
    return ED_ERR_CUDA;
  }
  *out = h.release();
  return ED_OK;
}

extern "C" int ed_batch_destroy(ed_batch* h) {
  if (!h) return ED_OK;
  cudaSetDevice(h->b.ctx->device);
  h->b.release();
  delete h;
  return ED_OK;
}

namespace ed {
namespace {
int batch_dispatch(Batch* b, const ed_lanczos_opts* opts, double* evals, int* iters, ed_batch_info* info,
                   cudaStream_t user, void* const* ritz = nullptr, int* conv = nullptr) {
  switch (b->prec) {
    case ED_PREC_FP64: return batch_run<PolF64>(b, opts, evals, iters, info, user, ritz, conv);
    case ED_PREC_DF64: return batch_run<PolDF>(b, opts, evals, iters, info, user, ritz, conv);
    default: return batch_run<PolF32>(b, opts, evals, iters, info, user, ritz, conv);
  }
}
bool chunk_ok(int c) { return c >= 64 && c <= 65536 && (c & (c - 1)) == 0; }
}  // namespace

// Sectors of different models solved together (the request server's packs of
// small requests): n jobs, job q the sector (n_up[q], n_dn[q]) of *models[q],
// all advanced by the same graph-replayed steps over one work list of `chunk`
// elements per item.  A job's arithmetic depends only on its own sector, the
// chunk and the seed, not on the other jobs, so its result is the same alone
// or in any pack.  evals: n * k (NaN past a job's dimension); iters, conv
// (1 where the job met tol or exhausted its Krylov space): n each; ritz: one
// device pointer per job for its k Ritz vectors (or NULL).  The batch's tables
// and vectors are made in ctx and released before returning.
int batch_solve_pack(Ctx* ctx, int prec, int n, const ed_model* const* models, const int* n_up, const int* n_dn,
                     const ed_lanczos_opts* o, uint32_t chunk, double* evals, int* iters, int* conv,
                     void* const* ritz) {
  Batch b;
  b.ctx = ctx;
  b.prec = prec;
  b.n_jobs = n;
  struct Rel {
    Batch* b;
    ~Rel() { b->release(); }
  } rel{&b};
  uint64_t off = 0;
  for (int q = 0; q < n; ++q) {
    std::unique_ptr<Sector> s(new Sector());
    int st = build_sector(ctx, models[q], n_up[q], n_dn[q], prec, s.get());
    if (st != ED_OK) {
      free_sector(s.get());
      return st;
    }
    JobDev jd{};
    jd.S = s->view();
    jd.ub = s->up.basis;
    jd.db = s->dn.basis;
    jd.off = off;
    jd.dim = s->dim;
    jd.seed_mix = 0;  // every job starts as it would alone
    b.hjobs.push_back(jd);
    off += (s->dim + 31) & ~(uint64_t)31;
    b.sectors.push_back(std::move(s));
  }
  b.tot = off;
  ED_TRY(b.alloc(&b.djobs, b.hjobs.size()));
  ED_TRY(b.set_chunk(chunk));
  ED_TRY_CUDA(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
  return batch_dispatch(&b, o, evals, iters, nullptr, b.stream, ritz, conv);
}
}  // namespace ed

extern "C" int ed_batch_set_chunk(ed_batch* h, int chunk) {
  if (!h) ED_INVALID("NULL argument");
  if (!chunk_ok(chunk)) ED_INVALID("chunk %d is not a power of two in 64..65536", chunk);
  ED_TRY_CUDA(cudaSetDevice(h->b.ctx->device));
  ED_TRY_CUDA(cudaStreamSynchronize(h->b.stream));
  return h->b.set_chunk((uint32_t)chunk);
}

extern "C" int ed_batch_autotune(ed_batch* h, int steps, ed_batch_tune_result* out, void* stream) {
  if (!h || !out) ED_INVALID("NULL argument");
  steps = std::max(2, std::min(steps, 64));
  Batch* b = &h->b;
  ED_TRY_CUDA(cudaSetDevice(b->ctx->device));
  std::memset(out, 0, sizeof(*out));
  out->chosen = -1;
  const int cand[] = {256, 512, 1024, 2048, 4096, 8192, 16384, 32768};
  // a few graph-replayed Lanczos steps of every sector (never converging)
  ed_lanczos_opts o{};
  o.k = 1;
  o.tol = 1e-300;
  o.max_iter = steps;
  o.check_every = steps;
  o.seed = 1;
  o.reorth = 1;
  std::vector<double> ev(b->n_jobs);
  double best = 0.0;
  for (int c : cand) {
    const int i = out->n_candidates++;
    out->chunk[i] = c;
    out->ms_per_step[i] = -1.0;
    ED_TRY(b->set_chunk((uint32_t)c));
    ed_batch_info info{};
    const int st = batch_dispatch(b, &o, ev.data(), nullptr, &info, as_stream(stream));
    if (st != ED_OK && st != ED_ERR_NOT_CONVERGED) return st;
    ED_TRY_CUDA(cudaStreamSynchronize(b->stream));
    out->ms_per_step[i] = info.total_ms / std::max(1, info.steps);
    if (out->chosen < 0 || out->ms_per_step[i] < best) {
      best = out->ms_per_step[i];
      out->chosen = i;
    }
  }
  set_error("");
  return b->set_chunk((uint32_t)out->chunk[out->chosen]);
}

extern "C" int ed_batch_lanczos(ed_batch* h, const ed_lanczos_opts* opts, double* evals, int* iters,
                                ed_batch_info* info, void* stream) {
  if (!h || !opts || !evals) ED_INVALID("NULL argument");
  if (opts->k < 1 || opts->k > 16) ED_INVALID("k=%d outside 1..16 for the batched solver", opts->k);
  if (opts->max_iter < 1 || !(opts->tol > 0.0)) ED_INVALID("bad max_iter / tol");
  if (!opts->reorth) ED_INVALID("the batched solver always reorthogonalises (set reorth = 1)");
  Batch* b = &h->b;
  ED_TRY_CUDA(cudaSetDevice(b->ctx->device));
  cudaStream_t user = as_stream(stream);
  // order the batch's private stream after the caller's stream and back
  cudaEvent_t ev;
  ED_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(b->stream, ev, 0);
  const int st = batch_dispatch(b, opts, evals, iters, info, user);
  cudaEventRecord(ev, b->stream);
  cudaStreamWaitEvent(user, ev, 0);
  cudaEventDestroy(ev);
  return st;
}
