// ed_dot_noalloc: the dot product of ed_dot without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns every device allocation (a fixed arena handed out
// by another runtime), processes that must not grow their footprint once a
// long solve is under way, or callers with no ed_ctx (whose creation
// allocates).  This entry point needs neither: its per-block partial sums live
// in a file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
#include <mutex>

#include "ed_internal.h"

namespace ed {

namespace {

constexpr uint64_t kNoAllocSlots = 65536;  // partial sums, one per tile
constexpr uint64_t kNoAllocTile = 4096;    // elements reduced by one block
constexpr int kNoAllocThreads = 256;
constexpr int kMaxDevices = 64;

// slots [0, kNoAllocSlots): tile partials; slot kNoAllocSlots: the result
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots + 32];

double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once per device).
int scratch_for_current_device(double** out) {
  int dev = 0;
  ED_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) ED_INVALID("device ordinal %d outside 0..%d", dev, kMaxDevices - 1);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error("cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
      return ED_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return ED_OK;
}

__device__ __forceinline__ void nmac(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void nmac(float2& a, float2 x, float2 y) { df_mac(a, x, y); }
__device__ __forceinline__ void nmac(float2& a, float x, float y) { df_mac1(a, make_float2(x, 0.f), y); }
__device__ __forceinline__ double nadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 nadd(float2 a, float2 b) { return df_add(a, b); }
__device__ __forceinline__ double nshfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 nshfl(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double nd(double a) { return a; }
__device__ __forceinline__ double nd(float2 a) { return (double)a.x + (double)a.y; }

template <class V>
struct NAcc;
template <>
struct NAcc<double> { using T = double; };
template <>
struct NAcc<float2> { using T = float2; };
template <>
struct NAcc<float> { using T = float2; };

// Block b reduces elements [b * tile, (b + 1) * tile) into partial[b]; the
// accumulation is the one ed_dot uses (double for FP64, double-float otherwise).
template <class V>
__global__ void __launch_bounds__(kNoAllocThreads) k_dot_tiles(const V* __restrict__ x, const V* __restrict__ y,
                                                              uint64_t n, double* __restrict__ partial) {
  using A = typename NAcc<V>::T;
  __shared__ A sh[kNoAllocThreads / 32];
  A acc{};
  const uint64_t b0 = (uint64_t)blockIdx.x * kNoAllocTile;
  const uint64_t b1 = b0 + kNoAllocTile < n ? b0 + kNoAllocTile : n;
  for (uint64_t i = b0 + threadIdx.x; i < b1; i += kNoAllocThreads) nmac(acc, x[i], y[i]);
  for (int o = 16; o > 0; o >>= 1) acc = nadd(acc, nshfl(acc, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    A v = threadIdx.x < kNoAllocThreads / 32 ? sh[threadIdx.x] : A{};
    for (int o = 16; o > 0; o >>= 1) v = nadd(v, nshfl(v, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = nd(v);
  }
}

// One block sums the nb partials into result.
__global__ void __launch_bounds__(kNoAllocThreads) k_dot_tiles_final(const double* __restrict__ partial, uint64_t nb,
                                                                    double* __restrict__ result) {
  __shared__ double sh[kNoAllocThreads / 32];
  double v = 0.0;
  for (uint64_t i = threadIdx.x; i < nb; i += kNoAllocThreads) v += partial[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < kNoAllocThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) *result = w;
  }
}

}  // namespace

}  // namespace ed

using namespace ed;

extern "C" int ed_dot_noalloc(const void* x, const void* y, uint64_t n, int prec, double* result, void* stream) {
  if (!x || !y || !result) ED_INVALID("NULL argument");
  if (prec != ED_PREC_FP64 && prec != ED_PREC_DF64 && prec != ED_PREC_FP32) ED_INVALID("unknown precision %d", prec);
  const uint64_t max_n = kNoAllocSlots * kNoAllocTile;
  if (n > max_n)
    ED_INVALID("n = %llu exceeds the %llu-element limit of the fixed no-alloc scratch (%llu tiles of %llu)",
               (unsigned long long)n, (unsigned long long)max_n, (unsigned long long)kNoAllocSlots,
               (unsigned long long)kNoAllocTile);
  if (n == 0) {
    *result = 0.0;
    return ED_OK;
  }
  double* scratch = nullptr;
  ED_TRY(scratch_for_current_device(&scratch));
  cudaStream_t st = as_stream(stream);
  const uint64_t nb = (n + kNoAllocTile - 1) / kNoAllocTile;
  switch (prec) {
    case ED_PREC_FP64:
      k_dot_tiles<double><<<(unsigned)nb, kNoAllocThreads, 0, st>>>((const double*)x, (const double*)y, n, scratch);
      break;
    case ED_PREC_DF64:
      k_dot_tiles<float2><<<(unsigned)nb, kNoAllocThreads, 0, st>>>((const float2*)x, (const float2*)y, n, scratch);
      break;
    default:
      k_dot_tiles<float><<<(unsigned)nb, kNoAllocThreads, 0, st>>>((const float*)x, (const float*)y, n, scratch);
  }
  ED_LAUNCH_CHECK();
  k_dot_tiles_final<<<1, kNoAllocThreads, 0, st>>>(scratch, nb, scratch + kNoAllocSlots);
  ED_LAUNCH_CHECK();
  ED_TRY_CUDA(cudaMemcpyAsync(result, scratch + kNoAllocSlots, sizeof(double), cudaMemcpyDeviceToHost, st));
  ED_TRY_CUDA(cudaStreamSynchronize(st));
  return ED_OK;
}
