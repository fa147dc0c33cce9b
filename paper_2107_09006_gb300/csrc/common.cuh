// Shared device helpers: launch shapes, warp/block reductions, bf16 conversion.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"

namespace lsq {

constexpr int kThreads = 256;       // threads of every block-wide kernel
constexpr int kWarps = kThreads / 32;
constexpr int kT = 32;              // tile edge of the block-envelope storage

// Bounds-checked build (-DLS_DEBUG_BOUNDS, the library libls_schwarz_dbg.so): the gather,
// scatter and local-solve kernels check their indices and copy ranges; an index out of
// range is not used: the kernel writes kErrBounds into the error slot it was given and
// skips the access, and the host returns LS_ERR_INVALID.  In the product build every
// check is a constant true.
#ifdef LS_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif

__device__ __forceinline__ bool in_range(int64_t i, int64_t n, double* err) {
  if constexpr (!kDebugBounds) {
    return true;
  } else {
    if (i >= 0 && i < n) return true;
    if (err) *err = kErrBounds;
    return false;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum: every thread gets the same value.  red must hold kWarps
// entries and is reused after the call returns.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) s += red[k];
  __syncthreads();
  return s;
}

// Sum of a partials array of length P, identical in every block that calls it.
__device__ __forceinline__ double reduce_partials(const double* __restrict__ part, int P, double* red) {
  double s = 0.0;
  for (int k = threadIdx.x; k < P; k += blockDim.x) s += part[k];
  return block_sum(s, red);
}

template <class T> struct Arith;
template <> struct Arith<double> { using type = double; };
template <> struct Arith<float> { using type = float; };
template <> struct Arith<__nv_bfloat16> { using type = float; };

__device__ __forceinline__ double to_arith(double x, double) { return x; }
__device__ __forceinline__ float to_arith(float x, float) { return x; }
__device__ __forceinline__ float to_arith(__nv_bfloat16 x, float) { return __bfloat162float(x); }

}  // namespace lsq
