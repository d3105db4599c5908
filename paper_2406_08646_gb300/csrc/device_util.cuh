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

// Sum of one value over a warp with an xor butterfly: every lane gets the
// same bits (each step adds the same two partial sums, in either order).
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL_MASK, x, off);
  return x;
}

// Deterministic block reduction of NV values: a butterfly inside each warp,
// then warp 0 reduces the 32 warp sums (absent warps count 0) with the same
// butterfly.  Result valid in thread 0 (in fact in every lane of warp 0).
// `scratch` holds NV * 32 values.  Ends with __syncthreads.
template <typename T, int NV>
__device__ __forceinline__ void block_reduce(T (&v)[NV], T *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const T x = warp_sum(v[k]);
    if (lane == 0) scratch[k * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nwarps ? scratch[k * 32 + lane] : T(0));
  }
  __syncthreads();
}

// Block-wide sums that EVERY thread receives, with one barrier: after it,
// each warp reduces the warp sums itself with the same butterfly, so all
// threads hold bitwise identical totals.  scratch holds two halves of
// NV * 32 values used alternately (half = 0, 1, 0, ...): a half is rewritten
// two calls later, after the intervening call's barrier, which no thread
// passes before every thread has finished reading it.
template <typename T, int NV>
__device__ __forceinline__ void block_allreduce(T (&v)[NV], T *scratch, int half) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  T *s = scratch + half * NV * 32;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const T x = warp_sum(v[k]);
    if (lane == 0) s[k * 32 + warp] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nwarps ? s[k * 32 + lane] : T(0));
}

// Fused multiply-add, correctly rounded once.
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace gbs
