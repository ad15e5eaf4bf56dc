// Device helpers shared by the sparse-coding kernels (k_omp.cu, k_omp_tm.cu).
// Internal to the library.
#pragma once

#include <stdint.h>

namespace dlk {
namespace omp {

constexpr unsigned FULL = 0xffffffffu;

// Read-only load that does not allocate in L1: each signal's correlations and
// samples are read once, and keeping them out of L1 leaves it to the Gram rows
// every step reads (measured: OMP 2.4% faster than plain loads).
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Bits of the argmax key that carry the element index t within a lane.
template <int NT>
constexpr int tbits() {
  return NT <= 1 ? 0 : NT <= 2 ? 1 : NT <= 4 ? 2 : NT <= 8 ? 3 : NT <= 16 ? 4 : 5;
}

template <int NT>
__device__ __forceinline__ float elem(const float2 (&a)[NT / 2], int t) {
  return (t & 1) ? a[t >> 1].y : a[t >> 1].x;
}

// Three-input maximum (one instruction on the sm_100 family); NaN inputs are
// ignored unless all three are NaN.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Maximum of N values (compile-time N) by a tree of three-input maxima.
template <int N>
__device__ __forceinline__ float max_tree(const float (&v)[N]) {
  if constexpr (N == 1) {
    return v[0];
  } else if constexpr (N == 2) {
    return fmaxf(v[0], v[1]);
  } else {
    constexpr int M = (N + 2) / 3;
    float w[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const int a = 3 * j;
      if (a + 2 < N)
        w[j] = fmax3(v[a], v[a + 1], v[a + 2 < N ? a + 2 : 0]);
      else if (a + 1 < N)
        w[j] = fmaxf(v[a], v[a + 1 < N ? a + 1 : 0]);
      else
        w[j] = v[a];
    }
    return max_tree<M>(w);
  }
}

// Argmax key of element t: |alpha| with the low TB mantissa bits replaced by
// (NT-1-t).  The float maximum of the keys gives the largest |alpha| and, among
// values equal to within 2^-(23-TB) relative, the lowest t; NaN (masked)
// elements are ignored.  Returns max(0, keys).
template <int NT>
__device__ __forceinline__ float keys_max(const float2 (&a)[NT / 2], unsigned vmask) {
  float k[NT + 1];
#pragma unroll
  for (int t = 0; t < NT; ++t)
    k[t] = __uint_as_float((__float_as_uint(elem<NT>(a, t)) & vmask) | (unsigned)(NT - 1 - t));
  k[NT] = 0.f;
  return max_tree<NT + 1>(k);
}

}  // namespace omp
}  // namespace dlk
