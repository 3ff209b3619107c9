// Sixteen-byte vectors of vector elements for the streaming kernels of the
// Lanczos recurrence: four FP32, two double-float or two FP64 elements per
// load or store.  Callers use them only where every vector slot starts on a
// 16-byte boundary, and read the ragged tail of a range element by element.
#pragma once

#include <cuda_runtime.h>

namespace ed {

template <class V>
struct Vec16;

template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int N = 4;
  __device__ static __forceinline__ float get(const T& v, int i) { return (&v.x)[i]; }
  __device__ static __forceinline__ void set(T& v, int i, float x) { (&v.x)[i] = x; }
};

template <>
struct Vec16<float2> {
  using T = float4;
  static constexpr int N = 2;
  __device__ static __forceinline__ float2 get(const T& v, int i) {
    return i ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
  }
  __device__ static __forceinline__ void set(T& v, int i, float2 x) {
    if (i) v.z = x.x, v.w = x.y;
    else v.x = x.x, v.y = x.y;
  }
};

template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int N = 2;
  __device__ static __forceinline__ double get(const T& v, int i) { return (&v.x)[i]; }
  __device__ static __forceinline__ void set(T& v, int i, double x) { (&v.x)[i] = x; }
};

// Basis slots padded to a multiple of 32 elements start 16-byte aligned.
inline uint64_t pad32(uint64_t n) { return (n + 31) & ~(uint64_t)31; }

}  // namespace ed
