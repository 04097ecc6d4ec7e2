// Device-side helpers shared by the RA-FEAST kernels (sm_103a).
//
// Complex values are stored as interleaved (re, im) pairs of T = float or
// double; one pair is float2 / double2. The inner-solve state is laid out
// row-major: row r, subspace column i, shift j at complex offset
// r * ldc + i * NC + j, so one lane owns all NC shifts of a column i (a
// "chunk") and can combine them into the quadrature sum without atomics.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rafeast {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };
template <typename T> using c2 = typename C2<T>::t;

template <typename T> __device__ __forceinline__ c2<T> mk(T re, T im) {
  c2<T> v; v.x = re; v.y = im; return v;
}
template <typename T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T> __device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a*b + c
template <typename T> __device__ __forceinline__ c2<T> cfma(c2<T> a, c2<T> b, c2<T> c) {
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// real s * a + c
template <typename T> __device__ __forceinline__ c2<T> crfma(T s, c2<T> a, c2<T> c) {
  return mk<T>(fma(s, a.x, c.x), fma(s, a.y, c.y));
}

// ---- chunk loads / stores: NC consecutive complex values ------------------
// float: 16-byte vector accesses when NC is even (offsets are then 16-byte
// aligned because every row stride and chunk offset is a multiple of 2
// complex values), else 8-byte accesses. double: one 16-byte access each.
template <int NC>
__device__ __forceinline__ void ld_chunk(const float* __restrict__ p, float2 (&v)[NC]) {
  if constexpr (NC % 2 == 0) {
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) {
      float4 t = __ldg(reinterpret_cast<const float4*>(p) + k);
      v[2 * k] = make_float2(t.x, t.y);
      v[2 * k + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) v[k] = __ldg(reinterpret_cast<const float2*>(p) + k);
  }
}
template <int NC>
__device__ __forceinline__ void ld_chunk(const double* __restrict__ p, double2 (&v)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) v[k] = __ldg(reinterpret_cast<const double2*>(p) + k);
}
// plain (coherent) loads for data written earlier by the same kernel family
template <int NC>
__device__ __forceinline__ void ldcg_chunk(const float* p, float2 (&v)[NC]) {
  if constexpr (NC % 2 == 0) {
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) {
      float4 t = __ldcg(reinterpret_cast<const float4*>(p) + k);
      v[2 * k] = make_float2(t.x, t.y);
      v[2 * k + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) v[k] = __ldcg(reinterpret_cast<const float2*>(p) + k);
  }
}
template <int NC>
__device__ __forceinline__ void ldcg_chunk(const double* p, double2 (&v)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) v[k] = __ldcg(reinterpret_cast<const double2*>(p) + k);
}
template <int NC>
__device__ __forceinline__ void st_chunk(float* p, const float2 (&v)[NC]) {
  if constexpr (NC % 2 == 0) {
#pragma unroll
    for (int k = 0; k < NC / 2; ++k)
      reinterpret_cast<float4*>(p)[k] = make_float4(v[2 * k].x, v[2 * k].y, v[2 * k + 1].x, v[2 * k + 1].y);
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) reinterpret_cast<float2*>(p)[k] = v[k];
  }
}
template <int NC>
__device__ __forceinline__ void st_chunk(double* p, const double2 (&v)[NC]) {
#pragma unroll
  for (int k = 0; k < NC; ++k) reinterpret_cast<double2*>(p)[k] = v[k];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace rafeast
