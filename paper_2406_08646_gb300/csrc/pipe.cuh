// Per-warp streaming pipelines fed by bulk (TMA) copies.
//
// Every warp of a CTA is an independent worker: it walks its own work blocks
// (global warp w takes blocks w, w + W, w + 2W, ... of a block table, W = all
// warps of the grid) through `ns` private shared-memory stages.  Lane 0 issues
// the bulk copies of the next blocks (completing on the stage's mbarrier) while
// the warp computes on the current one, so at any time each warp keeps up to
// ns-1 blocks in flight and the SM overlaps many warps' copies, gathers and
// FP64 work without CTA-wide synchronisation.  Consumers only read a stage;
// after a __syncwarp lane 0 may refill it (no proxy fence needed for that).
//
// Stage layout (bytes, every region 16-byte aligned):
//   H  [16]                    block descriptor {r0, r1, a, e} (lane 0 writes)
//   SpMV blocks:  V [cap x 8] | C [cap x 4] | RP [(R + 8) x 4] | S0 [(R + 8) x 8]
//   update blocks: S0..S4 [(R + 8) x 8 each]
// V, C hold the block's CSR values and columns from a0 = a & ~3, RP its row
// pointers from r0 & ~3, Sk vector slices from r0 rounded down to 16 bytes.
// Only whole 16-byte units inside the block are copied; the few elements or
// rows at either ragged end are read from global memory by the lane that
// needs them, so no copy ever reads outside its array.
#pragma once

#include "device_util.cuh"

namespace gbs {

constexpr int PIPE_MAX_STAGES = 4;
constexpr int UPD_SLICES = 5;

__host__ __device__ constexpr int64_t spmv_stage_bytes(int cap, int R) {
  return 16 + (int64_t)cap * 12 + (int64_t)(R + 8) * 4 + (int64_t)(R + 8) * 8;
}
__host__ __device__ constexpr int64_t upd_stage_bytes(int R) {
  return 16 + (int64_t)UPD_SLICES * (R + 8) * 8;
}

struct BlkDesc {
  int32_t r0, r1, a, e;  // rows [r0, r1), nonzeros [a, e)
};

// A table of work blocks (rows [blk_row0[b], blk_row0[b+1]) of system
// blk_sys[b]; blocks never straddle systems).
struct BlockTable {
  int32_t nblocks;
  const int32_t *row0;  // nblocks + 1
  const int32_t *nz0;   // nblocks + 1: row_ptr[row0[b]]
  const int32_t *sys;   // nblocks
  const int32_t *sys_blk0;   // nsys + 1
  const int32_t *sys_slot0;  // nsys + 1: reduction slot offsets for W workers
};

__device__ __forceinline__ BlkDesc load_desc(const BlockTable &t, int b) {
  BlkDesc d;
  d.r0 = __ldg(t.row0 + b);
  d.r1 = __ldg(t.row0 + b + 1);
  d.a = __ldg(t.nz0 + b);
  d.e = __ldg(t.nz0 + b + 1);
  return d;
}

struct WarpPipe {
  unsigned char *buf;  // this warp's ns stages
  uint64_t *bar;       // this warp's ns barriers
  int ns;
  int cap;             // SpMV stage: nonzeros (multiple of 4)
  int Ra, Re;          // rows per SpMV block / per update block
  int64_t stage_bytes;
  uint32_t parity;
  int32_t *err;
  int64_t timeout_ns;
  uint64_t pol_stream, pol_vec;

  __device__ unsigned char *stage(int s) const { return buf + (size_t)s * stage_bytes; }
  __device__ BlkDesc *H(unsigned char *st) const { return reinterpret_cast<BlkDesc *>(st); }
  // SpMV layout
  __device__ void *V(unsigned char *st) const { return st + 16; }
  __device__ int32_t *C(unsigned char *st) const {
    return reinterpret_cast<int32_t *>(st + 16 + (size_t)cap * 8);
  }
  __device__ int32_t *RP(unsigned char *st) const {
    return reinterpret_cast<int32_t *>(st + 16 + (size_t)cap * 12);
  }
  __device__ void *SA(unsigned char *st) const {
    return st + 16 + (size_t)cap * 12 + (size_t)(Ra + 8) * 4;
  }
  // update layout
  __device__ void *SE(unsigned char *st, int k) const {
    return st + 16 + (size_t)k * (Re + 8) * 8;
  }

  // Lane 0, once per kernel, before any use; the caller then synchronises.
  __device__ void init_barriers() {
    for (int s = 0; s < ns; ++s) mbar_init(bar + s, 1);
    fence_barrier_init();
  }

  // All lanes.  Bounded: on expiry record GBS_ERR_TIMEOUT, then wait once
  // more (bounded) for the copies still in flight, and report failure.
  __device__ bool wait(int s) {
    const uint32_t par = (parity >> s) & 1u;
    parity ^= (1u << s);
    if (mbar_try_wait(bar + s, par)) return true;
    for (int round = 0; round < 2; ++round) {
      const uint64_t t0 = global_ns();
      unsigned spins = 0;
      for (;;) {
        if (mbar_try_wait(bar + s, par)) return round == 0;
        if ((++spins & 15u) == 0 && (int64_t)(global_ns() - t0) > timeout_ns) break;
      }
      atomicCAS(err, 0, GBS_ERR_TIMEOUT);
    }
    return false;
  }
};

// Lane 0: complete the stage's barrier phase with `bytes` of copies to come
// (or at once when there are none).  Returns whether copies must be issued.
__device__ __forceinline__ bool arrive_for(uint64_t *bar, uint32_t bytes) {
  if (bytes == 0) {
    mbar_arrive(bar);
    return false;
  }
  mbar_arrive_expect_tx(bar, bytes);
  return true;
}

// Rows [lo, hi) of a vector slice are bulk-copied in 16-byte units; rows
// outside are read from global memory by slice_get.
template <typename T>
struct SliceRange {
  static constexpr int U = 16 / (int)sizeof(T);
  int r0a, lo, hi;
  __device__ SliceRange(int r0, int r1) {
    r0a = r0 & ~(U - 1);
    lo = min((r0 + U - 1) & ~(U - 1), r1);
    hi = max(r1 & ~(U - 1), lo);
  }
  __device__ uint32_t bytes() const { return (uint32_t)(hi - lo) * (uint32_t)sizeof(T); }
};

template <typename T>
__device__ __forceinline__ void slice_copy(void *dst, const T *src, const SliceRange<T> &q,
                                           uint64_t *bar, uint64_t pol) {
  if (q.hi > q.lo)
    bulk_load(static_cast<T *>(dst) + (q.lo - q.r0a), src + q.lo, q.bytes(), bar, pol);
}

template <typename T>
__device__ __forceinline__ T slice_get(const void *sl, const T *src, const SliceRange<T> &q,
                                       int r) {
  return (r >= q.lo && r < q.hi) ? static_cast<const T *>(sl)[r - q.r0a] : src[r];
}

// CSR value / column range of a block in 4-element units:
// head [a, lo), copied units [lo, hi), tail [hi, e).
struct NzRange {
  int32_t a, e, a0, lo, hi;
  bool fits;
  __device__ NzRange(int32_t a_, int32_t e_, int cap) : a(a_), e(e_) {
    a0 = a & ~3;
    lo = min((a + 3) & ~3, e);
    hi = max(e & ~3, lo);
    fits = (e - a0) <= cap;
  }
};

// Lane 0: bytes and copies of a SpMV block's CSR part (values, columns, row
// pointers).  A block longer than a stage (fits == false) copies nothing; its
// rows are then read with plain loads.
template <typename T>
__device__ __forceinline__ uint32_t csr_bytes(const BlkDesc &d, int cap) {
  const NzRange z(d.a, d.e, cap);
  if (!z.fits) return 0u;
  const SliceRange<int32_t> rq(d.r0, d.r1 + 1);
  return (uint32_t)(z.hi - z.lo) * (uint32_t)(sizeof(T) + 4) + rq.bytes();
}

template <typename T>
__device__ __forceinline__ void csr_copy(const WarpPipe &P, unsigned char *st, const BlkDesc &d,
                                         const int32_t *row_ptr, const int32_t *col,
                                         const T *val, uint64_t *bar) {
  const NzRange z(d.a, d.e, P.cap);
  if (!z.fits) return;
  if (z.hi > z.lo) {
    bulk_load(static_cast<T *>(P.V(st)) + (z.lo - z.a0), val + z.lo,
              (uint32_t)(z.hi - z.lo) * (uint32_t)sizeof(T), bar, P.pol_stream);
    bulk_load(P.C(st) + (z.lo - z.a0), col + z.lo, (uint32_t)(z.hi - z.lo) * 4u, bar,
              P.pol_stream);
  }
  const SliceRange<int32_t> rq(d.r0, d.r1 + 1);
  slice_copy<int32_t>(P.RP(st), row_ptr, rq, bar, P.pol_stream);
}

// Row r: sum over its nonzeros of val * x[col], in CSR order from 0, one
// fused multiply-add per nonzero (the FP64 units of GB300 issue about as many
// operations per second as HBM delivers nonzeros, so the product spends
// exactly one FP64 instruction per nonzero).  Eight gathers of x are issued
// before the FMAs.  STAGED: values, columns and row pointers from the stage
// (ragged ends from global memory); otherwise everything from global memory.
template <typename T, bool STAGED>
__device__ __forceinline__ T row_product(const WarpPipe &P, unsigned char *st, const NzRange &z,
                                         const SliceRange<int32_t> &rq, const int32_t *row_ptr,
                                         const int32_t *col, const T *val, const T *x, int r) {
  int32_t rs, re;
  if (STAGED) {
    rs = slice_get<int32_t>(P.RP(st), row_ptr, rq, r);
    re = slice_get<int32_t>(P.RP(st), row_ptr, rq, r + 1);
  } else {
    rs = __ldg(row_ptr + r);
    re = __ldg(row_ptr + r + 1);
  }
  const T *V = STAGED ? static_cast<const T *>(P.V(st)) : nullptr;
  const int32_t *C = STAGED ? P.C(st) : nullptr;
  T acc = T(0);
  constexpr int UNR = 8;
  for (int32_t q0 = rs; q0 < re; q0 += UNR) {
    T v[UNR], xv[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int32_t g = q0 + u;
      int32_t c = 0;
      v[u] = T(0);
      if (g < re) {
        if (STAGED && g >= z.lo && g < z.hi) {
          c = C[g - z.a0];
          v[u] = V[g - z.a0];
        } else {
          c = __ldg(col + g);
          v[u] = __ldg(val + g);
        }
      }
      xv[u] = (g < re) ? x[c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
      if (q0 + u < re) acc = fma_rn(v[u], xv[u], acc);
  }
  return acc;
}

// All rows of a SpMV block, lane per row (rows r0 + lane, + 32, ...):
// f(r, row_sum).  Uses the stage when the block fits, plain loads otherwise.
template <typename T, class F>
__device__ __forceinline__ void block_rows(const WarpPipe &P, unsigned char *st,
                                           const BlkDesc &d, const int32_t *row_ptr,
                                           const int32_t *col, const T *val, const T *x, F &f) {
  const int lane = threadIdx.x & 31;
  const NzRange z(d.a, d.e, P.cap);
  const SliceRange<int32_t> rq(d.r0, d.r1 + 1);
  if (z.fits) {
    for (int r = d.r0 + lane; r < d.r1; r += 32)
      f(r, row_product<T, true>(P, st, z, rq, row_ptr, col, val, x, r));
  } else {
    for (int r = d.r0 + lane; r < d.r1; r += 32)
      f(r, row_product<T, false>(P, st, z, rq, row_ptr, col, val, x, r));
  }
}

// Drive one warp's pipeline over its wanted blocks of table t.
//   want(b) -> bool            uniform across the warp
//   issue(d, stage, bar)       lane 0: arrive(.expect_tx) + bulk copies
//   work(b, d, stage)          all lanes of the warp
// worker = global warp index, W = number of warps in the grid.
template <class Want, class Issue, class Work>
__device__ __forceinline__ void warp_stream(WarpPipe &P, const BlockTable &t, int worker, int W,
                                            Want &want, Issue &issue, Work &work) {
  const int lane = threadIdx.x & 31;
  auto next = [&](int b) -> int {
    for (; b < t.nblocks; b += W)
      if (want(b)) return b;
    return -1;
  };
  // the stages may have been written by a plain phase (generic proxy) before
  fence_proxy_async();
  __syncwarp();
  int ib = next(worker), cb = ib, is = 0, cs = 0;
  BlkDesc nd{0, 0, 0, 0};
  if (lane == 0 && ib >= 0) nd = load_desc(t, ib);
  auto issue_next = [&]() {
    if (lane == 0) {
      unsigned char *st = P.stage(is);
      *P.H(st) = nd;
      issue(nd, st, P.bar + is);
    }
    ib = next(ib + W);
    if (lane == 0 && ib >= 0) nd = load_desc(t, ib);
    is = (is + 1 == P.ns) ? 0 : is + 1;
  };
  for (int k = 0; k < P.ns - 1 && ib >= 0; ++k) issue_next();
  while (cb >= 0) {
    __syncwarp();  // every lane is done with the stage refilled below
    if (ib >= 0) issue_next();
    P.wait(cs);
    unsigned char *st = P.stage(cs);
    const BlkDesc d = *P.H(st);
    work(cb, d, st);
    cb = next(cb + W);
    cs = (cs + 1 == P.ns) ? 0 : cs + 1;
  }
}

}  // namespace gbs
