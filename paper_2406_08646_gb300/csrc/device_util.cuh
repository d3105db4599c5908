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

// Deterministic block reduction of NV values, result in warp 0 (thread 0).
// Every thread stores its values in `scratch` (NV * blockDim.x values, one
// row per value); after one barrier, lane l of warp 0 adds the values of
// threads l, l + 32, l + 64, ... into four running sums taken in turn, which
// it combines, and a butterfly over warp 0 adds the lanes.  A fixed order, so
// the result is reproducible bit for bit.  FP64 is slow on this part (a
// warp-wide FP64 instruction takes 16 clocks of an SM's FP64 pipe), so the
// reduction uses about nthreads / 32 + 8 warp-wide adds per value instead of
// a butterfly in every warp.  Ends with __syncthreads (scratch reuse).
template <typename T>
__device__ __forceinline__ T block_sum_lanes(const T *s, int nt) {
  const int lane = threadIdx.x & 31;
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int j = lane;
  for (; j + 96 < nt; j += 128) {
    a0 += s[j];
    a1 += s[j + 32];
    a2 += s[j + 64];
    a3 += s[j + 96];
  }
  if (j < nt) a0 += s[j];
  if (j + 32 < nt) a1 += s[j + 32];
  if (j + 64 < nt) a2 += s[j + 64];
  return warp_sum((a0 + a1) + (a2 + a3));
}

template <typename T, int NV>
__device__ __forceinline__ void block_reduce(T (&v)[NV], T *scratch) {
  const int nt = blockDim.x;
#pragma unroll
  for (int k = 0; k < NV; ++k) scratch[k * nt + threadIdx.x] = v[k];
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = block_sum_lanes<T>(scratch + k * nt, nt);
  }
  __syncthreads();
}

// A hint to bring bytes [p, p + n) into L2: one bulk prefetch, which holds
// no registers and has no completion to wait for, so a warp can put a whole
// run of data in flight before its first load of it.  The bulk prefetch
// wants a 16-byte aligned start and a length in whole 16-byte units: the
// range is shrunk to the aligned units inside it (and to 64 KB), which
// keeps every prefetched byte inside [p, p + n).
__device__ __forceinline__ void prefetch_l2(const void *p, size_t n) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t s = (a + 15) & ~(uintptr_t)15;
  uintptr_t e = (a + n) & ~(uintptr_t)15;
  if (e > s + 65536) e = s + 65536;
  if (e > s)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s))
                 : "memory");
}

template <typename T>
__device__ __forceinline__ void prefetch_rows(const T *v, int r0, int r1) {
  if (r1 > r0) prefetch_l2(v + r0, (size_t)(r1 - r0) * sizeof(T));
}

// Fused multiply-add, correctly rounded once.
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace gbs
