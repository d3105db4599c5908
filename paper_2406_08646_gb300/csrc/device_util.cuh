// Device helpers shared by the kernels of libgbs.so: the global timer,
// L2-coherent loads, deterministic block reductions and rounded FMAs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace gbs {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// L2-coherent loads for values written by other CTAs inside the same launch.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) {
  return __ldcg(p);
}

// Deterministic block reduction of NV values: fixed xor-shuffle tree inside a
// warp, then warp sums added in warp order by thread 0.  Result valid in
// thread 0 only.  `scratch` holds NV * 32 values.  Ends with __syncthreads.
template <typename T, int NV>
__device__ __forceinline__ void block_reduce(T (&v)[NV], T *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T x = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL_MASK, x, off);
    if (lane == 0) scratch[k * 32 + warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T s = scratch[k * 32];
      for (int w = 1; w < nwarps; ++w) s += scratch[k * 32 + w];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Fused multiply-add, correctly rounded once.
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace gbs
