// Phase bodies of the Jacobi-PCG solve (Sec. 6.1 CG with device-resident
// scalars and no host round trip; Sec. 7 diagonal preconditioning and batched
// systems; Sec. 2 A7 FP32 inner solve under FP64 refinement).
//
// Each phase is one kernel launch; the iterations run inside a CUDA graph
// whose conditional WHILE node repeats the body (A, B, C) until the device
// clears its condition.  A CTA walks blocks c, c+G, c+2G, ... of the phase's
// block table (rows of one system per block).  Per iteration:
//   A: q = A p fused with the partial p.q
//   B: x += alpha p, r -= alpha q, z = D^-1 r (stored over q), r.z and r.r
//   C: p = z + beta p, and the loop condition
// GB300 issues FP64 FMAs at about the rate HBM delivers nonzeros, so the row
// products spend one FMA per stored nonzero and as few other FP64
// instructions as possible (see csr_rows).
//
// Reductions are deterministic: a CTA reduces its rows of a system in a fixed
// tree and writes one slot per (system, CTA); the CTA whose slot arrives last
// (atomic arrival counter per system) sums the system's slots in slot order
// and updates that system's scalars (alpha, beta, norms, status) in device
// memory, where the next phase reads them.  Converged systems are frozen
// (their blocks are skipped).
//
// Refined mode (per-system state machine, M_* modes): an FP32 PCG on FP32
// copies of A and D^-1 with FP32 vectors and FP32 reductions solves
// A d = r / ||r||; between inner solves the same A/B/C phases run the FP64
// outer step: x += s d (phase C), r = b - A x and ||r|| (phase A), and the
// inner restart r32 = RN(r / s), d = 0 (phase B).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

enum { M_INNER = 0, M_XUPD = 1, M_START = 2 };
constexpr int SLOT_STRIDE = 4;  // doubles per reduction slot
constexpr int PHASE_TPB = 512;  // threads per CTA of every phase kernel
// Shared scratch of the phase kernels' block reductions (NV <= 4 values per
// thread and the lane partials, device_util.cuh's block_reduce); kernels
// whose reductions carry one value need only RED_SCRATCH1.
constexpr int RED_SCRATCH = 4 * PHASE_TPB + BLOCK_SUMS_EXTRA;
constexpr int RED_SCRATCH1 = PHASE_TPB + BLOCK_SUMS_EXTRA / 4;
static_assert(PHASE_TPB % 128 == 0 && PHASE_TPB >= 256, "block_sums needs 128 k threads");
constexpr int SELL_MIN_CTAS = 4;  // sliced-ELL kernels: 4 CTAs (2048 threads) per SM

// A table of work blocks: rows [row0[b], row0[b+1]) of system sys[b].
struct BlockTable {
  int32_t nblocks;
  const int32_t *row0;       // nblocks + 1
  const int32_t *sys;        // nblocks
  const int32_t *sys_blk0;   // nsys + 1
  const int32_t *sys_slot0;  // nsys + 1: reduction slot offsets for this table's grid
  const int32_t *slice0;     // nblocks + 1: first 32-row slice of each block
  // block ends, where blocks do not tile the rows (the size split's tables,
  // which skip the small systems); null: block b ends where b + 1 starts
  const int32_t *row1, *slice1;
};

__device__ __forceinline__ int blk_row_end(const BlockTable &t, int b) {
  return __ldg((t.row1 ? t.row1 : t.row0 + 1) + b);
}
__device__ __forceinline__ int blk_slice_end(const BlockTable &t, int b) {
  return __ldg((t.slice1 ? t.slice1 : t.slice0 + 1) + b);
}

struct PcgArgs {
  int32_t nsys, ensemble;
  BlockTable ta, te;  // SpMV blocks, update blocks
  int64_t part_e;     // first reduction slot of table te
  int32_t grid_e;     // CTAs of the kernels that walk table te
  const int32_t *row_ptr, *col;
  const double *val;
  const float *val32;
  SellView sv;           // sliced-ELL copy (kernels with L == 0)
  const double *sval;
  const float *sval32;
  int32_t stream_matrix;  // 1: load the sliced copy evict-first (larger than L2 / 2)
  const double *dinv;
  const float *dinv32;
  double *r, *p, *q;
  float *r32, *p32, *q32, *d32;
  double *part;
  unsigned *sys_cnt;
  SysState *st;
  DevCtl *ctl;
  const CallArgs *call;
  const int32_t *order;             // per-CTA solver: its systems, largest first
  int32_t cta_n;                    //   how many (CTA k solves order[k], then takes the
                                    //   next one from DevCtl::queue)
  cudaGraphConditionalHandle cond;  // loop condition of the graph (stepped == 0)
  int32_t stepped;                  // 1: loop trips launched by the host
  int32_t trip;                     // stepped: index of this trip
  double *kv[KRYLOV_NVEC];          // nonsymmetric solvers' work vectors
  SellView tv;                      // sliced-ELL copy of A^T (BiCG), A's slices
  const double *tval;
  int32_t *halo_flags;              // one-kernel CG: iteration each CTA published
  int32_t halo_lo, halo_n;          //   and the window of CTAs it waits for
  int32_t grid_a;                   // CTAs of the kernels that walk table ta
};

// A solve loop on the phase kernels: the start-up kernels, the WHILE body
// (run while any system is active), the closing kernels.  Each kernel walks
// the SpMV block table (A) or, where *_e is set, the update table (E).
struct LoopPlan {
  int npre, nbody, npost;
  void (*pre[2])(PcgArgs);
  bool pre_e[2];
  void (*body[4])(PcgArgs);
  bool body_e[4];
  void (*post[2])(PcgArgs);
  bool post_e[2];
  bool body_coop;  // the body's kernels wait on one another's CTAs: cooperative launch
};

PcgArgs make_args(gbs_mat A, bool per_system, bool refined);
int build_loop_graph(gbs_mat A, const LoopPlan &P, PcgArgs a, cudaGraphExec_t *out);
int run_loop_stepped(const LoopPlan &P, PcgArgs a, int grid_a, int grid_e, int64_t cap,
                     DevCtl *ctl, cudaStream_t s);
int run_loop(gbs_mat A, const LoopPlan &P, int kind, const PcgArgs &a, const double *b,
             double *x, const ksp_opts &o, bool per_system, cudaStream_t s);
bool use_cta_solver(gbs_mat A, bool per_system);
int32_t split_count(gbs_mat A);
// The per-CTA solver's automatic choice: the largest system solved has at
// most CTA_AUTO_WORK nonzeros plus eight per row, or a batch gives every SM
// systems_per_sm CTAs.
bool cta_size_rule(gbs_mat A, bool per_system, int systems_per_sm);
int sm_count(gbs_mat A);
// The plan caps the phase kernels' grids at one or two CTAs per SM: its
// sliced-ELL row kernels run in their 64-register build.
inline bool wide_rows(gbs_mat A) { return A->ctas_per_sm == 1 || A->ctas_per_sm == 2; }

__device__ __forceinline__ int sys_of(const PcgArgs &a, const BlockTable &t, int b) {
  return a.ensemble ? 0 : __ldg(t.sys + b);
}
__device__ __forceinline__ int sys_b0(const PcgArgs &a, const BlockTable &t, int s) {
  return a.ensemble ? 0 : __ldg(t.sys_blk0 + s);
}
__device__ __forceinline__ int sys_nblk(const PcgArgs &a, const BlockTable &t, int s) {
  return a.ensemble ? t.nblocks : __ldg(t.sys_blk0 + s + 1) - __ldg(t.sys_blk0 + s);
}
__device__ __forceinline__ int64_t sys_slot0(const PcgArgs &a, const BlockTable &t, int s) {
  return a.ensemble ? 0 : (int64_t)__ldg(t.sys_slot0 + s);
}

__device__ __forceinline__ void deactivate(const PcgArgs &a, SysState &S, int status) {
  S.status = status;
  S.active = 0;
  atomicSub(&a.ctl->n_active, 1);
}

// Host-stepped loop: trip a.trip runs unless the previous trip stopped it.
__device__ __forceinline__ bool trip_live(const PcgArgs &a) {
  return !a.stepped || ldcg(&a.ctl->stop[a.trip & 1]) == 0;
}

// CTA 0 books the time since the previous phase kernel started to that
// phase and marks the start of phase k (kernels of one solve run in order).
// The two loads go out together and the sum is a fire-and-forget atomic, so
// the stamp costs CTA 0 one L2 round trip.
__device__ __forceinline__ void stamp_phase(const PcgArgs &a, int k) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevCtl *c = a.ctl;
    const int lp = c->last_phase;
    const int64_t st = c->stamp;
    const int64_t t = (int64_t)global_ns();
    atomicAdd(reinterpret_cast<unsigned long long *>(c->phase_ns + lp),
              (unsigned long long)(t - st));
    c->stamp = t;
    c->last_phase = k;
  }
}

// Sums over the warp of a system's ns reduction slots from base on (NV
// values each, SLOT_STRIDE apart): lane l adds slots l, l + 32, l + 64, ...
// in that order, then warp_sums adds the lanes -- a fixed order.  The lane's
// loads for a batch of slots (8 values in registers) are all issued before
// its first add, so the sum over a one-wave grid's slots takes a few L2
// round trips, not one per slot a lane holds.  Every lane ends with the
// totals.
template <int NV>
__device__ __forceinline__ void slot_sums(const double *part, int64_t base, int ns,
                                          double (&tot)[NV]) {
  constexpr int SLOT_BATCH = 8 / NV > 0 ? 8 / NV : 1;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = 0.0;
  for (int i0 = 0; i0 < ns; i0 += 32 * SLOT_BATCH) {
    double v[SLOT_BATCH][NV];
#pragma unroll
    for (int j = 0; j < SLOT_BATCH; ++j) {
      const int i = i0 + lane + 32 * j;
#pragma unroll
      for (int k = 0; k < NV; ++k)
        v[j][k] = i < ns ? ldcg(part + (base + i) * SLOT_STRIDE + k) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < SLOT_BATCH; ++j)
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (i0 + lane + 32 * j < ns) tot[k] += v[j][k];
  }
  warp_sums<double, NV>(tot);
}

// Reduce the CTA's NV partials over its run on system s (last block b of a
// table processed by G CTAs) into the system's slot; the last arriving CTA
// sums all slots in slot order and calls fin(s, totals) on thread 0 -- or,
// when fin also takes a lane index, on every lane of that CTA's warp 0 (a
// fin that needs the warp, e.g. to sum another kernel's slots).  ARRIVE =
// false: only the slot is written (no arrival count, no fin): a later
// kernel's fin sums those slots itself.  f32: FP32 accumulation throughout.
// REDUCED: acc already holds the CTA's totals in warp 0 (no block sums).
//
// Ensemble solves (FP64, !REDUCED) finish wide: thread 0 counts the CTA in,
// every thread learns at a barrier whether it was the last, and the last
// CTA's first four warps sum the slots (wide_sums: one L2 round trip and
// the adds spread over the four FP64 pipes, where warp 0 alone waits on
// several round trips and adds on one pipe).  NE > 0 (wide
// finish only): the last CTA also sums NE values of each of the system's
// slots in table E's region -- partials another kernel wrote without
// arrival -- and fin gets NV + NE totals (the NE are zero on the warp-0
// finish of per-system solves).

// The last CTA's sums, by its first four warps (one per sub-partition, whose
// FP64 pipes work in parallel -- the FP64 adds, not the loads, are what
// these sums wait on): thread i loads slots i, i + 128, ... of the NV-value
// region, a batch of up to 8 / NV slots in flight before the first add,
// adds them in slot order, then does the same over the NE-value region;
// warp_sums adds each warp's lanes, and warp 0 adds the four warps' sums
// with one lane per value.  A fixed order; one L2 round trip a region for up
// to 1024 / N slots.  Totals on every lane of warp 0.  (Measured on the Q1
// 96^3 CG against warp 0 alone, as in per-system solves: 73.6 against 75.4
// us per iteration; issuing both regions' loads before any add, with twelve
// values a thread in flight, gave 75.5.)
constexpr int WIDE_WARPS = 4;
template <int N>
__device__ __forceinline__ void wide_region(const double *part, int64_t base, int ns, int off,
                                            double *v) {
  constexpr int NT = 32 * WIDE_WARPS;
  constexpr int WIDE_BATCH = N == 1 ? 8 : (N == 2 ? 4 : 2);
  for (int i0 = (int)threadIdx.x; i0 < ns; i0 += NT * WIDE_BATCH) {
    double u[WIDE_BATCH][N];
#pragma unroll
    for (int j = 0; j < WIDE_BATCH; ++j)
#pragma unroll
      for (int k = 0; k < N; ++k)
        u[j][k] = i0 + j * NT < ns ? ldcg(part + (base + i0 + j * NT) * SLOT_STRIDE + k) : 0.0;
#pragma unroll
    for (int j = 0; j < WIDE_BATCH; ++j)
      if (i0 + j * NT < ns) {
#pragma unroll
        for (int k = 0; k < N; ++k) v[off + k] += u[j][k];
      }
  }
}

template <int NV, int NE>
__device__ __noinline__ void wide_sums(const double *part, int64_t base, int ns,
                                       int64_t ebase, int ens, double (&tot)[NV + NE]) {
  constexpr int NT = NV + NE;
  static_assert(NT >= 1 && NT <= 4, "wide_sums: 1 to 4 values");
  __shared__ double ws[WIDE_WARPS][NT];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < WIDE_WARPS) {
    double v[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) v[k] = 0.0;
    wide_region<NV>(part, base, ns, 0, v);
    if constexpr (NE > 0) wide_region<NE>(part, ebase, ens, NV, v);
    warp_sums<double, NT>(v);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NT; ++k) ws[w][k] = v[k];
    }
  }
  __syncthreads();
  if (w == 0) {
    const int k = lane < NT ? lane : 0;
    const double t = (ws[0][k] + ws[1][k]) + (ws[2][k] + ws[3][k]);
#pragma unroll
    for (int q = 0; q < NT; ++q) tot[q] = __shfl_sync(FULL_MASK, t, q);
  }
}

template <int NV, bool ARRIVE = true, bool REDUCED = false, int NE = 0, class Fin>
__device__ __forceinline__ void flush(const PcgArgs &a, const BlockTable &t, int64_t part_off,
                                      int s, int b, double (&acc)[NV], double *red, bool f32,
                                      Fin &fin) {
  const int G = gridDim.x;
  if constexpr (REDUCED) {
  } else if (f32) {
    float v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = (float)acc[k];
    block_reduce<float, NV>(v, reinterpret_cast<float *>(red));
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = (double)v[k];
  } else {
    block_reduce<double, NV>(acc, red);
  }
  const int b0 = sys_b0(a, t, s), nb = sys_nblk(a, t, s);
  const int ns = min(nb, G);
  const int slot = (b - b0) % G;
  const int64_t base = part_off + sys_slot0(a, t, s);
  constexpr int NT = NV + NE;
  if constexpr (ARRIVE && !REDUCED) {
    if (a.ensemble && !f32) {  // uniform over the CTA
      __shared__ int last;
      if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) a.part[(base + slot) * SLOT_STRIDE + k] = acc[k];
        __threadfence();
        last = atomicAdd(a.sys_cnt + s, 1u) == (unsigned)(ns - 1);
      }
      __syncthreads();
      if (!last) return;
      double tot[NT];
      wide_sums<NV, NE>(a.part, base, ns, a.part_e + sys_slot0(a, a.te, s),
                        min(sys_nblk(a, a.te, s), a.grid_e), tot);
      if ((threadIdx.x >> 5) != 0) return;
      const int lane = threadIdx.x & 31;
      if (lane == 0) a.sys_cnt[s] = 0u;
      if constexpr (std::is_invocable_v<Fin &, int, double(&)[NT], int>) {
        fin(s, tot, lane);
      } else {
        if (lane == 0) fin(s, tot);
      }
      return;
    }
  }
  // Warp 0 alone finishes: the other warps go on to their next blocks (or
  // exit) at once instead of waiting at a barrier for the fence and the
  // arrival count.  The last CTA's warp 0 reads the slots through L2
  // (ldcg): every writer fenced its slot before counting itself in, so all
  // slots are visible once the count is complete.  No fence after fin: the
  // state it writes is read by later kernels only (a CTA reads a system's
  // state before its own flush, hence before that system's fin), and kernel
  // boundaries order those accesses.
  if ((threadIdx.x >> 5) != 0) return;
  const int lane = threadIdx.x & 31;
  if constexpr (!ARRIVE) {
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) a.part[(base + slot) * SLOT_STRIDE + k] = acc[k];
    }
    return;
  }
  unsigned prev = 0;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) a.part[(base + slot) * SLOT_STRIDE + k] = acc[k];
    __threadfence();
    prev = atomicAdd(a.sys_cnt + s, 1u);
  }
  if (__shfl_sync(FULL_MASK, prev, 0) != (unsigned)(ns - 1)) return;
  // lane l adds slots l, l + 32, ... (each slot's NV values are adjacent),
  // then warp_sums adds the lanes
  double tot[NT];
#pragma unroll
  for (int k = NV; k < NT; ++k) tot[k] = 0.0;
  double (&tv)[NV] = *reinterpret_cast<double(*)[NV]>(tot);
  if (f32) {
    float x[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) x[k] = 0.f;
    for (int i = lane; i < ns; i += 32) {
      const double *sl = a.part + (base + i) * SLOT_STRIDE;
#pragma unroll
      for (int k = 0; k < NV; ++k) x[k] += (float)ldcg(sl + k);
    }
    warp_sums<float, NV>(x);
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = (double)x[k];
  } else {
    slot_sums<NV>(a.part, base, ns, tv);
  }
  if (lane == 0) a.sys_cnt[s] = 0u;
  if constexpr (std::is_invocable_v<Fin &, int, double(&)[NT], int>) {
    fin(s, tot, lane);
  } else {
    if (lane == 0) fin(s, tot);
  }
}

// The CTA's pass over its blocks of table t (b = blockIdx.x, + G, ...).
// want(s) -> 0 skip / 1 FP64 / 2 FP32 reduction (uniform for a system, and
// unchanged until the system's fin runs); work(s, b, r0, r1, acc) processes
// block b, rows [r0, r1).  A CTA meets each system in one run of consecutive visits, so it
// flushes once per system it touches (NV == 0: no reduction).
template <int NV, bool ARRIVE = true, int NE = 0, class Want, class Work, class Fin>
__device__ __forceinline__ void walk(const PcgArgs &a, const BlockTable &t, int64_t part_off,
                                     double *red, Want &want, Work &work, Fin &fin) {
  constexpr int NA = NV > 0 ? NV : 1;
  const int G = gridDim.x;
  int cur_s = -1, cur_b = -1, kind = 0;
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  for (int b = blockIdx.x; b < t.nblocks; b += G) {
    const int s = sys_of(a, t, b);
    const int r0 = __ldg(t.row0 + b), r1 = blk_row_end(t, b);  // issued with want's loads
    if (s != cur_s) {
      if constexpr (NV > 0) {
        if (kind) flush<NV, ARRIVE, false, NE>(a, t, part_off, cur_s, cur_b, acc, red, kind == 2, fin);
      }
      cur_s = s;
      kind = want(s);
#pragma unroll
      for (int k = 0; k < NA; ++k) acc[k] = 0.0;
    }
    if (!kind) continue;
    cur_b = b;
    work(s, b, r0, r1, acc);
  }
  if constexpr (NV > 0) {
    if (kind) flush<NV, ARRIVE, false, NE>(a, t, part_off, cur_s, cur_b, acc, red, kind == 2, fin);
  }
}

// Combine the L row partials of each lane of an L-lane group so that lane li
// ends with the full sum of row li: at distance d each lane keeps half of its
// rows, sends the other half to lane li ^ d and adds what it receives -- L-1
// adds per lane, against L log2(L) for one butterfly per row.  Fixed order.
template <typename T, int L>
__device__ __forceinline__ T transpose_reduce(T (&acc)[L], int li) {
#pragma unroll
  for (int d = L / 2; d >= 1; d >>= 1) {
    const bool hi = (li & d) != 0;
#pragma unroll
    for (int i = 0; i < d; ++i) {
      const T send = hi ? acc[i] : acc[i + d];
      const T keep = hi ? acc[i + d] : acc[i];
      acc[i] = keep + __shfl_xor_sync(FULL_MASK, send, d);
    }
  }
  return acc[0];
}

// Row products of rows [r0, r1): f(r, sum_k a_rk x_k) for each row, every
// product one FMA.  L < 32: each warp takes 32 consecutive rows per pass; a
// group of L lanes owns L of them, lane li walks entries li, li+L, ... of all
// L rows (the trip count is the warp's longest row over L, the same for every
// lane), and transpose_reduce leaves row base+lane in lane `lane`, so f runs
// on every lane with coalesced row indices.  L == 32: one row per warp, xor
// butterfly, f on lane 0.  All lanes reach the shuffles.
template <typename T, int L, class F>
__device__ __forceinline__ void csr_rows(const int32_t *__restrict__ row_ptr,
                                         const int32_t *__restrict__ col,
                                         const T *__restrict__ val, const T *__restrict__ x,
                                         int r0, int r1, F &f) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (L == 32) {
    for (int r = r0 + warp; r < r1; r += nw) {
      const int s = __ldg(row_ptr + r), e = __ldg(row_ptr + r + 1);
      T acc = T(0);
      for (int q = s + lane; q < e; q += 32)
        acc = fma_rn(__ldg(val + q), __ldg(x + __ldg(col + q)), acc);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, off);
      if (lane == 0) f(r, acc);
    }
  } else {
    const int li = lane & (L - 1), g0 = lane - li;
    for (int base = r0 + warp * 32; base < r1; base += nw * 32) {
      const int my = base + lane;
      int s = 0, e = 0;
      if (my < r1) {
        s = __ldg(row_ptr + my);
        e = __ldg(row_ptr + my + 1);
      }
      const int mxw = (int)__reduce_max_sync(FULL_MASK, (unsigned)(e - s));
      int rs[L], len[L];
#pragma unroll
      for (int u = 0; u < L; ++u) {
        rs[u] = __shfl_sync(FULL_MASK, s, g0 + u);
        len[u] = __shfl_sync(FULL_MASK, e - s, g0 + u);
      }
      T acc[L];
#pragma unroll
      for (int u = 0; u < L; ++u) acc[u] = T(0);
      for (int t = 0; t < mxw; t += L) {
        const int k = t + li;
        int c[L];
        T v[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
          const bool ok = k < len[u];
          c[u] = ok ? __ldg(col + rs[u] + k) : -1;
          v[u] = ok ? __ldg(val + rs[u] + k) : T(0);
        }
#pragma unroll
        for (int u = 0; u < L; ++u)
          if (c[u] >= 0) acc[u] = fma_rn(v[u], __ldg(x + c[u]), acc[u]);
      }
      const T sum = transpose_reduce<T, L>(acc, li);
      if (my < r1) f(my, sum);
    }
  }
}

// Element-wise rows [r0, r1) of a vector-update phase, thread by thread.  The
// loads of two rows are issued before either row's stores (the vectors are
// separate arrays, but the compiler cannot know they do not alias), so each
// thread keeps two rows of loads in flight.
template <class Load, class Apply>
__device__ __forceinline__ void rows2(int r0, int r1, Load &load, Apply &apply) {
  const int T = blockDim.x;
  int r = r0 + threadIdx.x;
  for (; r + T < r1; r += 2 * T) {
    const auto u = load(r);
    const auto w = load(r + T);
    apply(r, u);
    apply(r + T, w);
  }
  if (r < r1) apply(r, load(r));
}

template <typename T, int N>
struct Vals {
  T v[N];
};

// How a row product gathers x: GATHER_NC the read-only path (x is not
// written during the kernel), GATHER_CA a plain L1-cached load (coherent for
// values the same CTA wrote before a barrier, and for values other CTAs
// published with a release that this thread's acquire load observed).
enum { GATHER_CA = 0, GATHER_NC = 1 };

template <int GATHER, typename T>
__device__ __forceinline__ T ld_x(const T *p) {
  if constexpr (GATHER == GATHER_NC) return __ldg(p);
  else return __ldca(p);
}

// Read-only load of a matrix entry, evict-first when STREAM.
template <bool STREAM, typename T>
__device__ __forceinline__ T ld_entry(const T *p) {
  if constexpr (STREAM) return __ldcs(p);
  else return __ldg(p);
}

template <typename T>
struct Pair;
template <>
struct Pair<double> {
  typedef double2 type;
};
template <>
struct Pair<float> {
  typedef float2 type;
};

// Row products of the 32-row slices [s0, s1) of the sliced-ELL copy: warp w
// takes slices s0 + w, s0 + w + nw, ...; lane i sums row i of the slice in
// CSR order, one FMA per stored nonzero; padding is skipped.  Entries
// k = 2m, 2m + 1 of a lane's row are adjacent (pair layout, sell.cu), so one
// load fetches two column indices and one 8- or 16-byte load two values; two
// pairs are in flight per step.  With column patterns (S.pat set) no column
// index is read: lane i's k-th column is r + pool[pat[sl] + k], the offsets
// loaded two at a time by one broadcast load, and bit k of its mask says
// whether row i holds it (8 bytes per FP64 entry plus 4 per row).  Without,
// column indices come as 32-bit columns (S.col, padding -1) or, when every
// column is within 2^15 - 1 of its row, as 16-bit offsets col - row (S.off,
// padding SELL_PAD16): 10 bytes per FP64 nonzero instead of 12.  A slice's
// bounds, first row and pattern are loaded before its entries, so no
// dependent load is left for the end.  f(r, sum) runs on every lane whose row
// exists.  STREAM: the entries are loaded with the evict-first hint, so that
// a matrix larger than L2 does not push the vectors (x and the solver's
// vectors) out of it; FP32 slices (the refined solve's inner product) are
// also requested into L2 with one bulk prefetch of their entries and one of
// their column indices when the warp starts the slice, so that the later
// steps' loads find them there instead of waiting on DRAM one step at a time
// (the registers hold only two pairs' loads per step).  Measured on the Q1
// 96^3 matrix: 42.4 -> 38.3 us per FP32 inner SpMV phase; the same prefetch
// slows the FP64 row product (53.8 -> 62.6 us; offsets alone 55.9 us).
// NC: how x is gathered (GATHER_NC where x is not written during the kernel,
// GATHER_CA where it was written during the kernel: ld_x).
constexpr int16_t SELL_PAD16 = -32768;

// The two column indices of a pair (entries 2m, 2m + 1 of a lane's row): from
// the 32-bit columns, or decoded from the two 16-bit offsets; padding -1.
template <bool STREAM>
__device__ __forceinline__ int2 sell_pair_cols(const int2 *__restrict__ c2,
                                               const int *__restrict__ o2, int pi, int r) {
  if (o2) {
    const int o = ld_entry<STREAM>(o2 + pi);
    const int lo = (int)(int16_t)o, hi = o >> 16;
    return make_int2(lo == SELL_PAD16 ? -1 : r + lo, hi == SELL_PAD16 ? -1 : r + hi);
  }
  return ld_entry<STREAM>(c2 + pi);
}

// Slices with column patterns (S.pat set: every slice has one).
template <typename T, bool STREAM, int NC, class F>
__device__ __forceinline__ void sell_rows_pat(const SellView &S, const T *__restrict__ sval,
                                              const T *x, int s0, int s1, F &f) {
  typedef typename Pair<T>::type P;
  const P *__restrict__ v2 = reinterpret_cast<const P *>(sval);
  const int lane = threadIdx.x & 31;
  for (int sl = s0 + (int)(threadIdx.x >> 5); sl < s1; sl += (int)(blockDim.x >> 5)) {
    const int b0 = __ldg(S.ptr + sl), b1 = __ldg(S.ptr + sl + 1);
    const int r = __ldg(S.row0 + sl) + lane, re = __ldg(S.row0 + sl + 1);
    const int2 *__restrict__ pat2 = reinterpret_cast<const int2 *>(S.pool + __ldg(S.pat + sl));
    uint32_t mk = __ldg(S.mask + 32 * (int64_t)sl + lane);
    if constexpr (STREAM && sizeof(T) == 4) {  // the slice's whole run in flight at once
      if (lane == 0) prefetch_rows(sval, b0, b1);
    }
    int pi = (b0 >> 1) + lane;
    const int pend = pi + 32 * ((b1 - b0) >> 6);
    T acc = T(0);
    for (; pi + 32 < pend; pi += 64, pat2 += 2, mk >>= 4) {
      const int2 oa = __ldg(pat2), ob = __ldg(pat2 + 1);
      const P va = ld_entry<STREAM>(v2 + pi), vb = ld_entry<STREAM>(v2 + pi + 32);
      if (mk & 1u) acc = fma_rn(va.x, ld_x<NC>(x + r + oa.x), acc);
      if (mk & 2u) acc = fma_rn(va.y, ld_x<NC>(x + r + oa.y), acc);
      if (mk & 4u) acc = fma_rn(vb.x, ld_x<NC>(x + r + ob.x), acc);
      if (mk & 8u) acc = fma_rn(vb.y, ld_x<NC>(x + r + ob.y), acc);
    }
    if (pi < pend) {
      const int2 oa = __ldg(pat2);
      const P va = ld_entry<STREAM>(v2 + pi);
      if (mk & 1u) acc = fma_rn(va.x, ld_x<NC>(x + r + oa.x), acc);
      if (mk & 2u) acc = fma_rn(va.y, ld_x<NC>(x + r + oa.y), acc);
      mk >>= 2;
      ++pat2;
    }
    if ((((b1 - b0) >> 5) & 1) && (mk & 1u)) {  // the odd last entry
      const int o = __ldg(reinterpret_cast<const int *>(pat2));
      acc = fma_rn(ld_entry<STREAM>(sval + (b1 - 32 + lane)), ld_x<NC>(x + r + o), acc);
    }
    if (r < re) f(r, acc);
  }
}

template <typename T, bool STREAM, int NC, class F>
__device__ __forceinline__ void sell_rows(const SellView &S, const T *__restrict__ sval,
                                          const T *x, int s0, int s1, F &f) {
  if (S.pat) {
    sell_rows_pat<T, STREAM, NC>(S, sval, x, s0, s1, f);
    return;
  }
  typedef typename Pair<T>::type P;
  const int2 *__restrict__ c2 = reinterpret_cast<const int2 *>(S.col);
  const int *__restrict__ o2 = reinterpret_cast<const int *>(S.off);  // two offsets per int
  const P *__restrict__ v2 = reinterpret_cast<const P *>(sval);
  const int lane = threadIdx.x & 31;
  for (int sl = s0 + (int)(threadIdx.x >> 5); sl < s1; sl += (int)(blockDim.x >> 5)) {
    const int b0 = __ldg(S.ptr + sl), b1 = __ldg(S.ptr + sl + 1);
    const int r = __ldg(S.row0 + sl) + lane, re = __ldg(S.row0 + sl + 1);
    if constexpr (STREAM && sizeof(T) == 4) {  // the slice's whole run in flight at once
      if (lane == 0) prefetch_rows(sval, b0, b1);
      else if (lane == 1) {
        if (S.off) prefetch_rows(S.off, b0, b1);
        else prefetch_rows(S.col, b0, b1);
      }
    }
    // pair index of this lane's first pair, and one past its last full pair
    int pi = (b0 >> 1) + lane;
    const int pend = pi + 32 * ((b1 - b0) >> 6);
    T acc = T(0);
    for (; pi + 32 < pend; pi += 64) {
      const int2 ca = sell_pair_cols<STREAM>(c2, o2, pi, r);
      const int2 cb = sell_pair_cols<STREAM>(c2, o2, pi + 32, r);
      const P va = ld_entry<STREAM>(v2 + pi), vb = ld_entry<STREAM>(v2 + pi + 32);
      if (ca.x >= 0) acc = fma_rn(va.x, ld_x<NC>(x + ca.x), acc);
      if (ca.y >= 0) acc = fma_rn(va.y, ld_x<NC>(x + ca.y), acc);
      if (cb.x >= 0) acc = fma_rn(vb.x, ld_x<NC>(x + cb.x), acc);
      if (cb.y >= 0) acc = fma_rn(vb.y, ld_x<NC>(x + cb.y), acc);
    }
    if (pi < pend) {
      const int2 ca = sell_pair_cols<STREAM>(c2, o2, pi, r);
      const P va = ld_entry<STREAM>(v2 + pi);
      if (ca.x >= 0) acc = fma_rn(va.x, ld_x<NC>(x + ca.x), acc);
      if (ca.y >= 0) acc = fma_rn(va.y, ld_x<NC>(x + ca.y), acc);
    }
    if (((b1 - b0) >> 5) & 1) {  // the odd last entry, stored after the pairs
      const int q = b1 - 32 + lane;
      int c;
      if (S.off) {
        const int o = ld_entry<STREAM>(S.off + q);
        c = o == SELL_PAD16 ? -1 : r + o;
      } else {
        c = ld_entry<STREAM>(S.col + q);
      }
      if (c >= 0) acc = fma_rn(ld_entry<STREAM>(sval + q), ld_x<NC>(x + c), acc);
    }
    if (r < re) f(r, acc);
  }
}

// The row products of block b (rows [r0, r1) of table ta) with the plan's
// kernel: L == 0 sliced ELL, else CSR-vector with L lanes per row.// The row products of block b (rows [r0, r1) of table ta) with the plan's
// kernel: L == 0 sliced ELL, else CSR-vector with L lanes per row.
template <typename T, int L, class F>
__device__ __forceinline__ void row_products(const PcgArgs &a, int b, int r0, int r1,
                                             const T *csr_val, const T *sell_val, const T *x,
                                             F &f) {
  if constexpr (L == 0) {
    const int s0 = __ldg(a.ta.slice0 + b), s1 = blk_slice_end(a.ta, b);
    if (a.stream_matrix)
      sell_rows<T, true, GATHER_NC>(a.sv, sell_val, x, s0, s1, f);
    else
      sell_rows<T, false, GATHER_NC>(a.sv, sell_val, x, s0, s1, f);
  } else
    csr_rows<T, L>(a.row_ptr, a.col, csr_val, x, r0, r1, f);
}

// The convergence threshold thr = rtol ||b_s|| and two bounds of thr^2
// (FP64 roundings included: thr2lo <= thr^2 (1 - 2^-51) and thr2hi >=
// thr^2 (1 + 2^-49) in real arithmetic), so that ||r|| <= thr, i.e.
// RN(sqrt(rr)) <= thr, is decided from rr alone except within about 2^-49
// of thr^2: rr <= thr2lo gives sqrt(rr) <= thr exactly, hence its rounding
// too (thr is a double), and rr > thr2hi gives sqrt(rr) > thr (1 + 2^-51),
// which rounds above thr (half an ulp of thr is at most thr 2^-53).  Where
// thr^2 leaves the normal range the square root decides.
__device__ __forceinline__ void set_thr(SysState &S, double thr) {
  S.thr = thr;
  S.thr2lo = thr * thr * (1.0 - 0x1p-50);
  S.thr2hi = thr * thr * (1.0 + 0x1p-48);
}
// ||r|| <= thr from rr = ||r||^2 >= 0 (the comparisons on the bits, valid
// for non-negative doubles; NaN compares above every bound and fails).
__device__ __forceinline__ bool meets_thr(double rr, const SysState &S) {
  const long long b = __double_as_longlong(rr);
  const long long lo = __double_as_longlong(S.thr2lo), hi = __double_as_longlong(S.thr2hi);
  constexpr long long NORMAL_MIN = 0x0010000000000000LL;  // bits of 2^-1022
  if (b <= lo && lo >= NORMAL_MIN) return true;
  if (b > hi && hi >= NORMAL_MIN) return false;
  return sqrt(rr) <= S.thr;
}

// A system's state as a kernel reads it on meeting the system (want): it was
// written by earlier kernels only -- a fin writes it after every CTA of its
// launch that touches the system has read it -- and L1 holds nothing across
// launches, so the warps of a CTA may read it through L1: about one L2
// request per CTA instead of one per warp.  (With L2 loads the whole grid's
// warps queued on the same few lines at one L2 slice: measured on GB300, a
// 607-CTA launch's CTAs began their work over 8 us instead of 2.6 us, and
// CG on the Q1 96^3 system took 77.3 instead of 75.3 us per iteration.)
template <typename T>
__device__ __forceinline__ T ld_state(const T *p) {
  return __ldca(p);
}

// Per-system scalars a phase needs, read once per system run.
struct SysView {
  double alpha, beta, scale;
  int mode, first, zero;
};
__device__ __forceinline__ SysView view_sys(const PcgArgs &a, int s) {
  const SysState *S = a.st + s;
  return SysView{ld_state(&S->alpha), ld_state(&S->beta), ld_state(&S->scale),
                 ld_state(&S->mode),  ld_state(&S->first), ld_state(&S->zero_x)};
}
__device__ __forceinline__ bool sys_active(const PcgArgs &a, int s) {
  return ld_state(&a.st[s].active) != 0;
}

// ------------------------------------------------------------------ setup
// r = b - A x0 (x0 = 0 unless nonzero_guess), z = D^-1 r, p = z (FP64 mode),
// partials r.z, r.r, b.b and the count of missing diagonals; fin initialises
// each system's state and its status.  Runs on table ta.
template <bool REFINED, int L>
__device__ __forceinline__ void phase_setup(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  const bool guess = C.nonzero_guess != 0;
  auto want = [&](int) -> int { return 1; };
  auto row = [&](int r, double t, double(&acc)[4]) {
    const double bv = b[r];
    const double rv = bv - t;
    const double dv = a.dinv[r];
    if (REFINED) {
      a.r[r] = rv;
      acc[0] = fma(rv, rv, acc[0]);
    } else {
      const double z = dv * rv;
      a.r[r] = rv;
      a.p[r] = z;
      acc[0] = fma(rv, z, acc[0]);
      acc[1] = fma(rv, rv, acc[1]);
    }
    acc[2] = fma(bv, bv, acc[2]);
    acc[3] += (dv == 0.0) ? 1.0 : 0.0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[4]) {
    if (guess) {
      auto f = [&](int r, double t) { row(r, t, acc); };
      row_products<double, L>(a, blk, r0, r1, a.val, a.sval, x, f);
    } else {
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        x[r] = 0.0;
        row(r, 0.0, acc);
      }
    }
  };
  auto fin = [&](int s, double(&tot)[4]) {
    SysState &S = a.st[s];
    const double bb = tot[2], nbad = tot[3];
    const double rr = REFINED ? tot[0] : tot[1];
    const double rho = REFINED ? 0.0 : tot[0];
    memset(&S, 0, sizeof(SysState));
    S.bb = bb;
    set_thr(S, C.rtol * sqrt(S.bb));
    S.rho = rho;
    S.rr = rr;
    S.rnorm0 = S.rnorm = sqrt(rr);
    int status = -1;
    if (nbad > 0.0) status = GBS_ERR_NOT_SPD;
    else if (!isfinite(bb)) status = GBS_ERR_NAN;
    else if (bb == 0.0) {
      status = GBS_OK;
      S.zero_x = 1;
      S.rnorm0 = S.rnorm = 0.0;
    } else if (!isfinite(rr) || !isfinite(rho)) status = GBS_ERR_NAN;
    else if (sqrt(rr) <= C.rtol * sqrt(bb)) status = GBS_OK;
    else if (REFINED ? (C.max_outer <= 0) : (C.maxit <= 0)) status = GBS_ERR_MAXIT;
    if (status >= 0) {
      S.status = status;
      S.active = 0;
    } else {
      S.status = GBS_OK;
      S.active = 1;
      if (REFINED) {
        S.prev_rn = S.rnorm;
        S.scale = S.rnorm;
        S.mode = M_START;
      }
      atomicAdd(&a.ctl->n_active, 1);
    }
  };
  walk<4>(a, a.ta, 0, red, want, work, fin);
}

// ------------------------------------------------------------------ phase A
// FP64: q = A p, p.q -> alpha.  Refined: the FP32 inner product q32 = A32 p32
// and p32.q32 (M_INNER), or the FP64 outer residual r = b - A x and ||r||
// with the refinement tests (M_XUPD).
template <bool REFINED, int L>
__device__ __forceinline__ void phase_A(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  auto fin = [&](int s, double(&tot)[1]) {
    SysState &S = a.st[s];
    if (!REFINED) {  // (tests on the bits: see finite64)
      const double sigma = tot[0];
      S.iterations += 1;
      if (nan64(sigma)) deactivate(a, S, GBS_ERR_NAN);
      else if (!positive64(sigma)) deactivate(a, S, GBS_ERR_BREAKDOWN);
      else S.alpha = S.rho / sigma;
    } else if (S.mode == M_INNER) {
      const float sigma = (float)tot[0];
      S.first = 0;
      if (!(sigma > 0.0f)) {
        if (S.inner_it == 0) deactivate(a, S, GBS_ERR_BREAKDOWN);
        else {
          S.mode = M_XUPD;
          S.outer += 1;
        }
      } else {
        S.alpha = (double)((float)S.rho / sigma);
        S.inner_it += 1;
        S.iterations += 1;
      }
    } else {  // outer residual
      const double rn = sqrt(tot[0]);
      S.rnorm = rn;
      if (!isfinite(rn)) deactivate(a, S, GBS_ERR_NAN);
      else if (rn <= S.thr) deactivate(a, S, GBS_OK);
      else if (S.outer >= C.max_outer) deactivate(a, S, GBS_ERR_MAXIT);
      else {
        S.stall = (rn > 0.5 * S.prev_rn) ? S.stall + 1 : 0;
        if (S.stall >= 2) deactivate(a, S, GBS_ERR_STAGNATION);
        else {
          S.prev_rn = rn;
          S.scale = rn;
          S.mode = M_START;
        }
      }
    }
  };
  int mode = M_INNER;
  auto want = [&](int s) -> int {
    mode = ld_state(&a.st[s].mode);  // issued with the active flag: one round trip
    if (!sys_active(a, s)) return 0;
    if (!REFINED) return 1;
    return mode == M_INNER ? 2 : (mode == M_XUPD ? 1 : 0);
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[1]) {
    if (!REFINED) {
      double pq = acc[0];
      auto f = [&](int r, double qv) {
        a.q[r] = qv;
        pq = fma(__ldg(a.p + r), qv, pq);
      };
      row_products<double, L>(a, blk, r0, r1, a.val, a.sval, a.p, f);
      acc[0] = pq;
    } else if (mode == M_INNER) {
      float pq = 0.0f;
      auto f = [&](int r, float qv) {
        a.q32[r] = qv;
        pq = fmaf(__ldg(a.p32 + r), qv, pq);
      };
      row_products<float, L>(a, blk, r0, r1, a.val32, a.sval32, a.p32, f);
      acc[0] = (double)((float)acc[0] + pq);
    } else {  // FP64 outer residual
      const double *b = C.b;
      double rr = acc[0];
      auto f = [&](int r, double t) {
        const double rv = b[r] - t;
        a.r[r] = rv;
        rr = fma(rv, rv, rr);
      };
      row_products<double, L>(a, blk, r0, r1, a.val, a.sval, C.x, f);
      acc[0] = rr;
    }
  };
  walk<1>(a, a.ta, 0, red, want, work, fin);
}

// ------------------------------------------------------------------ phase B
template <bool REFINED>
__device__ __forceinline__ void phase_B(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  double *x = C.x;
  auto fin = [&](int s, double(&tot)[2]) {
    SysState &S = a.st[s];
    if (!REFINED) {
      // tests on the bits, ||r|| <= thr from ||r||^2, and the square root
      // only when the system stops (the closing kernel takes it otherwise)
      const double rho_new = tot[0], rr = tot[1];
      S.rr = rr;
      int st = -1;
      if (!finite64(rr) || !finite64(rho_new)) st = GBS_ERR_NAN;
      else if (meets_thr(rr, S)) st = GBS_OK;
      else if (S.iterations >= C.maxit) st = GBS_ERR_MAXIT;
      if (st >= 0) {
        S.rnorm = sqrt(rr);
        S.rn_stale = 0;
        deactivate(a, S, st);
      } else {
        S.rn_stale = 1;
        S.beta = rho_new / S.rho;
        S.rho = rho_new;
      }
    } else if (S.mode == M_START) {
      const float rho = (float)tot[0], rr = (float)tot[1];
      const float r0 = sqrtf(rr);
      // inner target: inner_rtol, or the smaller reduction that already
      // brings the outer residual to half of rtol ||b||
      const double tgt = fmax(C.inner_rtol, 0.5 * S.thr / S.scale);
      S.rho = rho;
      S.rr = rr;
      S.r0in = tgt * (double)r0;  // the inner stopping threshold
      S.inner_it = 0;
      if (!((double)r0 > C.inner_rtol * (double)r0) || C.inner_maxit <= 0)
        deactivate(a, S, GBS_ERR_BREAKDOWN);
      else {
        S.mode = M_INNER;
        S.first = 1;
      }
    } else {  // M_INNER
      const float rho_new = (float)tot[0], rr = (float)tot[1];
      const float beta = rho_new / (float)S.rho;
      S.rho = rho_new;
      S.rr = rr;
      if (!((double)sqrtf(rr) > S.r0in) || S.inner_it >= C.inner_maxit) {
        S.mode = M_XUPD;
        S.outer += 1;
      } else {
        S.beta = beta;
      }
    }
  };
  SysView v{};
  auto want = [&](int s) -> int {
    v = view_sys(a, s);  // issued with the active flag: one round trip
    if (!sys_active(a, s)) return 0;
    if (!REFINED) return 1;
    return (v.mode == M_INNER || v.mode == M_START) ? 2 : 0;
  };
  auto work = [&](int, int, int r0, int r1, double(&acc)[2]) {
    if (!REFINED) {
      const double al = v.alpha;
      double a0 = acc[0], a1 = acc[1];
      auto load = [&](int r) {
        return Vals<double, 5>{{a.p[r], a.q[r], x[r], a.r[r], a.dinv[r]}};
      };
      auto apply = [&](int r, const Vals<double, 5> &u) {
        const double rv = fma(-al, u.v[1], u.v[3]);
        const double z = u.v[4] * rv;
        x[r] = fma(al, u.v[0], u.v[2]);
        a.r[r] = rv;
        a.q[r] = z;
        a0 = fma(rv, z, a0);
        a1 = fma(rv, rv, a1);
      };
      rows2(r0, r1, load, apply);
      acc[0] = a0;
      acc[1] = a1;
    } else if (v.mode == M_INNER) {
      const float al = (float)v.alpha;
      float a0 = (float)acc[0], a1 = (float)acc[1];
      auto load = [&](int r) {
        return Vals<float, 5>{{a.p32[r], a.q32[r], a.d32[r], a.r32[r], a.dinv32[r]}};
      };
      auto apply = [&](int r, const Vals<float, 5> &u) {
        const float rv = fmaf(-al, u.v[1], u.v[3]);
        const float z = u.v[4] * rv;
        a.d32[r] = fmaf(al, u.v[0], u.v[2]);
        a.r32[r] = rv;
        a.q32[r] = z;
        a0 = fmaf(rv, z, a0);
        a1 = fmaf(rv, rv, a1);
      };
      rows2(r0, r1, load, apply);
      acc[0] = (double)a0;
      acc[1] = (double)a1;
    } else {  // M_START: inner restart on the scaled FP64 residual
      float a0 = (float)acc[0], a1 = (float)acc[1];
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const float rv = __double2float_rn(a.r[r] / v.scale);
        const float z = a.dinv32[r] * rv;
        a.r32[r] = rv;
        a.d32[r] = 0.0f;
        a.q32[r] = z;
        a0 = fmaf(rv, z, a0);
        a1 = fmaf(rv, rv, a1);
      }
      acc[0] = (double)a0;
      acc[1] = (double)a1;
    }
  };
  walk<2>(a, a.te, a.part_e, red, want, work, fin);
}

// ------------------------------------------------------------------ phase C
// FP64: p = z + beta p.  Refined: p32 = z32 (+ beta p32) (M_INNER) or the
// refinement step x += s d (M_XUPD).
template <bool REFINED>
__device__ __forceinline__ void phase_C(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  double *x = C.x;
  auto fin = [&](int, double(&)[1]) {};
  SysView v{};
  auto want = [&](int s) -> int {
    v = view_sys(a, s);  // issued with the active flag: one round trip
    if (!sys_active(a, s)) return 0;
    if (!REFINED) return 1;
    return (v.mode == M_INNER || v.mode == M_XUPD) ? 1 : 0;
  };
  auto work = [&](int, int, int r0, int r1, double(&)[1]) {
    if (!REFINED) {
      const double be = v.beta;
      auto load = [&](int r) { return Vals<double, 2>{{a.p[r], a.q[r]}}; };
      auto apply = [&](int r, const Vals<double, 2> &u) { a.p[r] = fma(be, u.v[0], u.v[1]); };
      rows2(r0, r1, load, apply);
    } else if (v.mode == M_INNER) {
      const float be = v.first ? 0.0f : (float)v.beta;  // first step: p = z
      auto load = [&](int r) { return Vals<float, 2>{{a.p32[r], a.q32[r]}}; };
      auto apply = [&](int r, const Vals<float, 2> &u) {
        a.p32[r] = v.first ? u.v[1] : fmaf(be, u.v[0], u.v[1]);
      };
      rows2(r0, r1, load, apply);
    } else {  // M_XUPD: x += s d
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x)
        x[r] = fma(v.scale, (double)a.d32[r], x[r]);
    }
  };
  walk<0>(a, a.te, a.part_e, red, want, work, fin);
}

// The last CTA of phase C: count the trip and set the loop condition (not
// CTA 0, which already stamps the phase timer).  Every phase that can retire
// a system (setup, A, B) has completed, so n_active is final for this trip.
// The trip cap and the wall-clock limit end the loop with the remaining
// systems still active (reported as GBS_ERR_MAXIT / TIMEOUT).  A trip that
// did not run (host-stepped loop) passes the stop on.
__device__ __forceinline__ void loop_control(const PcgArgs &a, bool live) {
  if (blockIdx.x != gridDim.x - 1 || threadIdx.x != 0) return;
  const CallArgs &C = *a.call;
  DevCtl *c = a.ctl;
  int go = 0;
  if (live) {
    const int64_t trips = c->trips + 1;
    c->trips = trips;
    go = (ldcg(&c->n_active) > 0 && trips < C.max_trips) ? 1 : 0;
    if (go && C.timeout_ns > 0 && (int64_t)global_ns() - c->t_start > C.timeout_ns) {
      c->err = GBS_ERR_TIMEOUT;
      go = 0;
    }
  }
  if (a.stepped) c->stop[(a.trip + 1) & 1] = go ? 0 : 1;
  else cudaGraphSetConditional(a.cond, go ? 1u : 0u);
}

// ------------------------------------------------------------------ closing residual
// ||b - A x||^2 per system (x = 0 exactly where b = 0).  Runs on table ta.
template <int L>
__device__ __forceinline__ void phase_final(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  int zero = 0;
  auto want = [&](int s) -> int {
    zero = ld_state(&a.st[s].zero_x);
    return 1;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[1]) {
    if (zero) {
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) x[r] = 0.0;
      return;
    }
    double tt = acc[0];
    auto f = [&](int r, double t) {
      const double d = b[r] - t;
      tt = fma(d, d, tt);
    };
    row_products<double, L>(a, blk, r0, r1, a.val, a.sval, x, f);
    acc[0] = tt;
  };
  auto fin = [&](int s, double(&tot)[1]) {
    SysState &S = a.st[s];
    S.tt = tot[0];
    if (S.rn_stale) {  // a loop stopped with the system running (trip cap, time limit)
      S.rnorm = sqrt(S.rr);
      S.rn_stale = 0;
    }
  };
  walk<1>(a, a.ta, 0, red, want, work, fin);
}

}  // namespace gbs
