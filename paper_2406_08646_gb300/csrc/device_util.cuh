// Device helpers shared by the kernels of libgbs.so: memory-order primitives,
// shared-memory barriers and bulk copies, the bounded grid barrier and
// deterministic block reductions.
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

// ---- shared-memory mbarrier + bulk (TMA) copies ---------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Make barrier initialisation visible to the async proxy (bulk copies).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Order this thread's generic-proxy accesses (shared and global) before its
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes: multiple
// of 16; both addresses 16-byte aligned).  The matrix stream is marked
// evict-first in L2 so it does not push out the vectors gathered by SpMV.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
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
      fence_proxy_async();
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

// Fused multiply-add, correctly rounded once.
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

}  // namespace gbs
