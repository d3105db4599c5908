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

// A flag published to, and read by, other CTAs of the same launch: the
// store releases (at GPU scope) everything the storing thread has ordered
// before it; the load acquires.
__device__ __forceinline__ void st_release(int32_t *p, int32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sum of one value over a warp with an xor butterfly: every lane gets the
// same bits (each step adds the same two partial sums, in either order).
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL_MASK, x, off);
  return x;
}

// Sums over the 32 lanes of NV <= 4 values at once: at distance 16 (and 8
// when NV > 2) each lane keeps half of the values, sends the other half to
// its partner and adds what it receives, so later steps work on fewer values
// per lane; a butterfly over the remaining distances completes the sums.
// Value k ends in lane 16 k (NV = 2) or 8 k (NV > 2) and is broadcast from
// there.  5 or 6 warp-wide adds for the NV values together, against 5 NV
// for one butterfly per value (an FP64 warp instruction holds a
// sub-partition's FP64 pipe for 64 clocks on this part).  A fixed order.
template <typename T, int NV>
__device__ __forceinline__ void warp_sums(T (&t)[NV]) {
  static_assert(NV >= 1 && NV <= 4, "warp_sums: 1 to 4 values");
  const int lane = threadIdx.x & 31;
  if constexpr (NV == 1) {
    t[0] = warp_sum(t[0]);
  } else if constexpr (NV == 2) {
    const bool hi = lane & 16;
    T u = (hi ? t[1] : t[0]) + __shfl_xor_sync(FULL_MASK, hi ? t[0] : t[1], 16);
#pragma unroll
    for (int d = 8; d > 0; d >>= 1) u += __shfl_xor_sync(FULL_MASK, u, d);
    t[0] = __shfl_sync(FULL_MASK, u, 0);
    t[1] = __shfl_sync(FULL_MASK, u, 16);
  } else {
    const T t3 = NV == 4 ? t[NV - 1] : T(0);
    const bool h16 = lane & 16, h8 = lane & 8;
    // lanes < 16 keep values 0, 1; lanes >= 16 keep values 2, 3
    const T a = (h16 ? t[2] : t[0]) + __shfl_xor_sync(FULL_MASK, h16 ? t[0] : t[2], 16);
    const T b = (h16 ? t3 : t[1]) + __shfl_xor_sync(FULL_MASK, h16 ? t[1] : t3, 16);
    // bit 3 clear keeps the first of them, set the second
    T u = (h8 ? b : a) + __shfl_xor_sync(FULL_MASK, h8 ? a : b, 8);
#pragma unroll
    for (int d = 4; d > 0; d >>= 1) u += __shfl_xor_sync(FULL_MASK, u, d);
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = __shfl_sync(FULL_MASK, u, 8 * k);
  }
}

// Deterministic block sums of NV <= 4 values per thread, spread over the
// SM's four sub-partitions (whose FP64 pipes work in parallel): every thread
// stores its values (row k of s holds value k of all nt threads); after a
// barrier, warp 4k + q -- on sub-partition q -- adds quarter q of row k,
// two values per lane at a time, and leaves 32 lane partials in p; after a
// second barrier warp 0 adds the four quarters' partials lane by lane and
// warp_sums adds the lanes.  About nt / 128 + 3 + 6 / NV warp-wide adds per
// value on the critical path, against nt / 32 + 8 for one warp doing it all.
// Totals in warp 0.  nt = blockDim.x must be a multiple of 128 and at least
// 256 (the kernels here run 512 or 1024 threads); s holds NV nt values, p
// 128 NV.  s is free once the second barrier is passed; p is read by warp 0
// only, so a later call (whose first barrier warp 0 must reach) cannot
// overwrite it early.
template <typename T, int NV>
__device__ __forceinline__ void block_sums(T (&v)[NV], T *s, T *p) {
  const int nt = blockDim.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k * nt + threadIdx.x] = v[k];
  __syncthreads();
  if (w < 4 * NV) {
    const int len = nt >> 2;
    const T *q = s + (w >> 2) * nt + (w & 3) * len;
    T a0 = q[lane], a1 = q[lane + 32];
    for (int j = lane + 64; j < len; j += 64) {
      a0 += q[j];
      a1 += q[j + 32];
    }
    p[w * 32 + lane] = a0 + a1;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const T *r = p + 128 * k + lane;
      v[k] = (r[0] + r[32]) + (r[64] + r[96]);
    }
    warp_sums<T, NV>(v);
  }
}

// The phase kernels' block reduction: block_sums with s and p in one
// scratch array of NV (nt + 128) values (s first, then p).
constexpr int BLOCK_SUMS_EXTRA = 512;  // p: 128 values per reduced value, up to 4
template <typename T, int NV>
__device__ __forceinline__ void block_reduce(T (&v)[NV], T *scratch) {
  block_sums<T, NV>(v, scratch, scratch + NV * blockDim.x);
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

// IEEE-754 tests on the bits, on the integer pipe: a single thread's scalar
// step (a reduction's fin) waits on every FP64 instruction it issues, and on
// GB300 each holds an FP64 pipe for 64 clocks however few lanes are active.
__device__ __forceinline__ bool finite64(double x) {  // not Inf, not NaN
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool positive64(double x) {  // x > 0.0 (false for NaN)
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool nan64(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}

// Fused multiply-add, correctly rounded once.
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace gbs
