// Device helpers shared by the kernels of libgbs.so: memory-order primitives,
// bounded grid barrier, deterministic block reductions and the staged CSR row
// product used by SpMV and by the fused CG phases.
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

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p,
                                                    unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_s32(const int32_t *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// L2-coherent loads for values written by other CTAs inside the same launch.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) {
  return __ldcg(p);
}

// Grid-wide barrier for a cooperative (co-resident) launch.  Monotonic 64-bit
// arrival counter: the k-th barrier completes when the counter reaches k * G.
// Every wait is bounded by timeout_ns; on expiry the CTA records
// GBS_ERR_TIMEOUT in *err and returns false, and any CTA that later finds *err
// set returns false at once, so no wait can outlive the timeout.
struct GridBarrier {
  unsigned long long *ctr;
  int32_t *err;
  unsigned long long target;
  int64_t timeout_ns;
  unsigned extra;  // phantom participants (testing the timeout path); normally 0

  __device__ bool sync() {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      target += gridDim.x + extra;
      int ok = 1;
      __threadfence();
      red_release_add_u64(ctr, 1ull);
      if (ld_relaxed_s32(err) != 0) {
        ok = 0;
      } else {
        const uint64_t t0 = global_ns();
        unsigned spins = 0;
        while (ld_acquire_u64(ctr) < target) {
          if ((++spins & 63u) == 0) {
            if (ld_relaxed_s32(err) != 0) {
              ok = 0;
              break;
            }
            if ((int64_t)(global_ns() - t0) > timeout_ns) {
              atomicCAS(err, 0, GBS_ERR_TIMEOUT);
              ok = 0;
              break;
            }
          }
        }
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
};

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

// Rounded product and sum with no fused multiply-add, so a row sum reproduces
// "s = s + a*x" evaluated left to right in the value type.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// Staged CSR product for one work block of rows [r0, r1) (r1 - r0 <= blockDim.x).
// The block's nonzeros are streamed with coalesced loads in chunks of `cap`;
// each product val*x[col] is written to shared memory `prod`, then the thread
// owning row r0 + threadIdx.x sums its row's products in CSR order starting
// from 0.  Returns that row sum (0 for threads without a row).  The matrix is
// read through the read-only path; x is read with plain loads because inside a
// persistent kernel it is written by other CTAs between grid barriers.
template <typename T>
__device__ __forceinline__ T staged_row_product(const int32_t *__restrict__ row_ptr,
                                                const int32_t *__restrict__ col,
                                                const T *__restrict__ val, const T *x,
                                                int32_t r0, int32_t r1, T *prod, int cap) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int32_t a = __ldg(row_ptr + r0), e = __ldg(row_ptr + r1);
  const int32_t r = r0 + tid;
  const bool has = r < r1;
  const int32_t rs = has ? __ldg(row_ptr + r) : 0;
  const int32_t re = has ? __ldg(row_ptr + r + 1) : 0;
  T acc = T(0);
  for (int32_t c0 = a; c0 < e; c0 += cap) {
    const int n = min(e - c0, cap);
    const int32_t *cc = col + c0;
    const T *vv = val + c0;
    int k = tid;
    for (; k + 3 * nt < n; k += 4 * nt) {
      const int32_t j0 = __ldg(cc + k), j1 = __ldg(cc + k + nt);
      const int32_t j2 = __ldg(cc + k + 2 * nt), j3 = __ldg(cc + k + 3 * nt);
      const T a0 = __ldg(vv + k), a1 = __ldg(vv + k + nt);
      const T a2 = __ldg(vv + k + 2 * nt), a3 = __ldg(vv + k + 3 * nt);
      const T x0 = x[j0], x1 = x[j1], x2 = x[j2], x3 = x[j3];
      prod[k] = mul_rn(a0, x0);
      prod[k + nt] = mul_rn(a1, x1);
      prod[k + 2 * nt] = mul_rn(a2, x2);
      prod[k + 3 * nt] = mul_rn(a3, x3);
    }
    for (; k < n; k += nt) prod[k] = mul_rn(__ldg(vv + k), x[__ldg(cc + k)]);
    __syncthreads();
    const int32_t lo = max(rs, c0), hi = min(re, c0 + n);
    for (int32_t q = lo; q < hi; ++q) acc = add_rn(acc, prod[q - c0]);
    __syncthreads();
  }
  return acc;
}

}  // namespace gbs
