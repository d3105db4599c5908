// COO -> CSR assembly on the device (Sec. 5: MatSetPreallocationCOO /
// MatSetValuesCOO), the Jacobi diagonal (Sec. 7), the FP32 copy used by the
// refined solve (Sec. 2, A7) and the adjoint scatter over the pattern.
//
// Symbolic stage, all on the GPU:
//   1. keep flags (negative index -> ignored; out of range -> error) and an
//      exclusive scan, compaction into 64-bit keys i*ncols + j with the
//      original COO index as payload;
//   2. stable LSD radix sort of the keys (8-bit digits, as many passes as the
//      largest key needs): per-tile digit histograms, one scan of the
//      digit-major count table, then a stable scatter that ranks equal digits
//      with warp match/ballot in input order;
//   3. segment heads of the sorted keys and a scan -> nnz, jmap (segment
//      offsets), the unique keys, then col, the diagonal positions and
//      row_ptr (lower bound of r*ncols in the unique keys).
// The sorted payload is perm (sorted position -> original COO index): equal
// keys keep increasing COO index, which is what makes the numeric stage's
// in-order sum well defined.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

// ------------------------------------------------------------------ scan

constexpr int SCAN_T = 256, SCAN_IPT = 16, SCAN_TILE = SCAN_T * SCAN_IPT;

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *warp_tot,
                                                        uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t y = __shfl_up_sync(FULL_MASK, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < nw; ++w) {
      uint32_t t = warp_tot[w];
      warp_tot[w] = run;
      run += t;
    }
    *total = run;
  }
  __syncthreads();
  const uint32_t r = warp_tot[warp] + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t *in, int64_t n,
                                                        uint32_t *tile_sums) {
  __shared__ uint32_t red[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_T) {
    const int64_t idx = base + k;
    if (idx < n) s += in[idx];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL_MASK, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < SCAN_T / 32; ++w) t += red[w];
    tile_sums[blockIdx.x] = t;
  }
}

// One CTA: exclusive scan of tile_sums in place; grand total to *total.
__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t *tile_sums, int64_t ntiles,
                                                     uint32_t *total) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t chunk_tot;
  uint32_t carry = 0;
  for (int64_t c0 = 0; c0 < ntiles; c0 += blockDim.x) {
    const int64_t idx = c0 + threadIdx.x;
    const uint32_t v = idx < ntiles ? tile_sums[idx] : 0u;
    const uint32_t ex = block_excl_scan_u32(v, warp_tot, &chunk_tot);
    if (idx < ntiles) tile_sums[idx] = carry + ex;
    carry += chunk_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__device__ __forceinline__ int pad_idx(int k) { return k + (k >> 5); }

__global__ void __launch_bounds__(SCAN_T) k_scan_down(const uint32_t *in, int64_t n,
                                                      const uint32_t *tile_offs,
                                                      uint32_t *out) {
  __shared__ uint32_t tile[SCAN_TILE + SCAN_TILE / 32];
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_T) {
    const int64_t idx = base + k;
    tile[pad_idx(k)] = idx < n ? in[idx] : 0u;
  }
  __syncthreads();
  uint32_t loc[SCAN_IPT];
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_IPT; ++q) {
    loc[q] = s;
    s += tile[pad_idx(threadIdx.x * SCAN_IPT + q)];
  }
  const uint32_t ex = block_excl_scan_u32(s, warp_tot, &tot) + tile_offs[blockIdx.x];
#pragma unroll
  for (int q = 0; q < SCAN_IPT; ++q) tile[pad_idx(threadIdx.x * SCAN_IPT + q)] = ex + loc[q];
  __syncthreads();
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_T) {
    const int64_t idx = base + k;
    if (idx < n) out[idx] = tile[pad_idx(k)];
  }
}

// Exclusive scan of n uint32 (in may equal out), reduce-then-scan; the tile
// sums are scanned by one CTA when they fit one tile, else recursively.
// tmp: scan_tmp_words(n) words.  Grand total written to *total (device) when
// non-null.
static int exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                          uint32_t *total, cudaStream_t s) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles == 0) {
    if (total) GBS_TRY_CUDA(cudaMemsetAsync(total, 0, sizeof(uint32_t), s));
    return GBS_OK;
  }
  k_scan_reduce<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, n, tmp);
  GBS_LAUNCHED(1);
  if (ntiles <= SCAN_TILE) {
    k_scan_tiles<<<1, 1024, 0, s>>>(tmp, ntiles, total);
    GBS_LAUNCHED(1);
  } else {
    GBS_TRY(exclusive_scan(tmp, tmp, ntiles, tmp + ntiles + 1, total, s));
  }
  k_scan_down<<<(unsigned)ntiles, SCAN_T, 0, s>>>(in, n, tmp, out);
  GBS_LAUNCHED(1);
  return GBS_OK;
}

static int64_t scan_tmp_words(int64_t n) {
  int64_t w = 1, t = (n + SCAN_TILE - 1) / SCAN_TILE;
  for (;;) {
    w += t + 1;
    if (t <= SCAN_TILE) break;
    t = (t + SCAN_TILE - 1) / SCAN_TILE;
  }
  return w;
}

// ------------------------------------------------------------------ keep + compact

// Batched handles pass per-system COO offsets (coo_off, nsys+1) and row offsets
// (row_off, nsys+1): local indices are shifted to the block-diagonal numbering.
struct KeepArgs {
  const int32_t *i, *j;
  int64_t ncoo, nrows, ncols;
  const int64_t *coo_off, *row_off;  // null for a single system
  int32_t nsys;
};

__device__ __forceinline__ bool keep_entry(const KeepArgs &a, int64_t k, int64_t &gi,
                                           int64_t &gj, bool &bad) {
  const int32_t li = a.i[k], lj = a.j[k];
  bad = false;
  if (li < 0 || lj < 0) return false;
  if (a.coo_off) {
    int lo = 0, hi = a.nsys;  // find s with coo_off[s] <= k < coo_off[s+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(a.coo_off + mid) <= k) lo = mid; else hi = mid;
    }
    const int64_t r0 = __ldg(a.row_off + lo), n = __ldg(a.row_off + lo + 1) - r0;
    if (li >= n || lj >= n) {
      bad = true;
      return false;
    }
    gi = r0 + li;
    gj = r0 + lj;
  } else {
    if (li >= a.nrows || lj >= a.ncols) {
      bad = true;
      return false;
    }
    gi = li;
    gj = lj;
  }
  return true;
}

__global__ void k_keep_flags(KeepArgs a, uint32_t *flags, int32_t *err) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.ncoo;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t gi, gj;
    bool bad;
    const bool keep = keep_entry(a, k, gi, gj, bad);
    if (bad) atomicExch(err, GBS_ERR_INDEX);
    flags[k] = keep ? 1u : 0u;
  }
}

__global__ void k_compact(KeepArgs a, const uint32_t *pos, uint64_t *keys, uint32_t *vals) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.ncoo;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t gi, gj;
    bool bad;
    if (keep_entry(a, k, gi, gj, bad)) {
      const uint32_t d = pos[k];
      keys[d] = (uint64_t)gi * (uint64_t)a.ncols + (uint64_t)gj;
      vals[d] = (uint32_t)k;
    }
  }
}

// ------------------------------------------------------------------ radix sort

constexpr int RS_T = 256, RS_WARPS = RS_T / 32, RS_SLOTS = 16, RS_TILE = RS_T * RS_SLOTS;

__global__ void __launch_bounds__(RS_T) k_radix_hist(const uint64_t *keys, int64_t n,
                                                     int shift, uint32_t *counts,
                                                     int64_t ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_T) {
    const int64_t idx = base + k;
    const uint32_t d = idx < n ? (uint32_t)((keys[idx] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(FULL_MASK, d);
    if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns the contiguous items
// [base + w*SLOTS*32, base + (w+1)*SLOTS*32); it walks them slot by slot, lane
// order within a slot, which is the input order, so ranks of equal digits
// follow input order.  The tile is first reordered by digit in shared memory
// (stable), then written out by consecutive threads to consecutive addresses
// of each digit's run, so the stores coalesce instead of scattering single
// items over 256 runs.  vals_in == null means payload = item index.
struct RadixShared {
  uint64_t key[RS_TILE];
  uint32_t val[RS_TILE];
  uint32_t whist[RS_WARPS][256];  // per-warp digit counts, then per-warp offsets in the tile
  uint32_t toff[256];             // the tile's global offset of each digit
  uint32_t dbase[256];            // first position of each digit in the reordered tile
};

__global__ void __launch_bounds__(RS_T) k_radix_scatter(const uint64_t *keys_in,
                                                        const uint32_t *vals_in, int64_t n,
                                                        int shift, const uint32_t *offsets,
                                                        int64_t ntiles, uint64_t *keys_out,
                                                        uint32_t *vals_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  RadixShared &S = *reinterpret_cast<RadixShared *>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < RS_WARPS; ++w) S.whist[w][threadIdx.x] = 0;
  S.toff[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t base = tile0 + (int64_t)warp * RS_SLOTS * 32;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t key[RS_SLOTS];
  uint32_t val[RS_SLOTS], rank[RS_SLOTS];
#pragma unroll
  for (int sl = 0; sl < RS_SLOTS; ++sl) {
    const int64_t idx = base + sl * 32 + lane;
    const bool ok = idx < n;
    key[sl] = ok ? keys_in[idx] : 0ull;
    val[sl] = ok ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
  }
#pragma unroll
  for (int sl = 0; sl < RS_SLOTS; ++sl) {
    const int64_t idx = base + sl * 32 + lane;
    const uint32_t d = idx < n ? (uint32_t)((key[sl] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(FULL_MASK, d);
    const uint32_t before = d < 256u ? S.whist[warp][d] : 0u;
    rank[sl] = before + (uint32_t)__popc(peers & lt_mask);
    __syncwarp();
    if (d < 256u && lane == __ffs(peers) - 1) S.whist[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: exclusive prefix over warps; the digit's total
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = S.whist[w][d];
      S.whist[w][d] = run;
      run += c;
    }
    S.dbase[d] = run;
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the 256 digit totals (8 per lane)
    uint32_t t[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      t[k] = S.dbase[lane * 8 + k];
      sum += t[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL_MASK, incl, off);
      if (lane >= off) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      S.dbase[lane * 8 + k] = run;
      run += t[k];
    }
  }
  __syncthreads();
#pragma unroll
  for (int sl = 0; sl < RS_SLOTS; ++sl) {  // reorder the tile by digit (stable)
    const int64_t idx = base + sl * 32 + lane;
    if (idx < n) {
      const uint32_t d = (uint32_t)((key[sl] >> shift) & 255u);
      const uint32_t lp = S.dbase[d] + S.whist[warp][d] + rank[sl];
      S.key[lp] = key[sl];
      S.val[lp] = val[sl];
    }
  }
  __syncthreads();
  const int cnt = (int)(n - tile0 < RS_TILE ? n - tile0 : RS_TILE);
  for (int i = threadIdx.x; i < cnt; i += RS_T) {  // runs of a digit go to consecutive addresses
    const uint64_t k = S.key[i];
    const uint32_t d = (uint32_t)((k >> shift) & 255u);
    const uint32_t dst = S.toff[d] + (uint32_t)i - S.dbase[d];
    keys_out[dst] = k;
    vals_out[dst] = S.val[i];
  }
}

// ------------------------------------------------------------------ segments

__global__ void k_seg_flags(const uint64_t *keys, int64_t n, uint32_t *flags) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    flags[t] = (t == 0 || keys[t] != keys[t - 1]) ? 1u : 0u;
}

__global__ void k_seg_write(const uint64_t *keys, int64_t n, const uint32_t *flags,
                            const uint32_t *seg, uint64_t *ukey, int32_t *jmap) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (flags[t]) {
      const uint32_t s = seg[t];
      ukey[s] = keys[t];
      jmap[s] = (int32_t)t;
    }
  }
}

// Columns, diagonal positions and the largest |col - row| (capped at 2^30,
// into *span): the sliced copy stores 16-bit column offsets when it is
// below 2^15.
__global__ void k_csr_cols(const uint64_t *ukey, int64_t nnz, int64_t ncols, int32_t *col,
                           int32_t *diag_pos, int32_t *span) {
  int32_t m = 0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nnz;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ukey[s];
    const int64_t r = (int64_t)(k / (uint64_t)ncols), c = (int64_t)(k % (uint64_t)ncols);
    col[s] = (int32_t)c;
    if (r == c) diag_pos[r] = (int32_t)s;
    const int64_t d = c - r, ad = d < 0 ? -d : d;
    m = max(m, (int32_t)(ad > (1 << 30) ? (1 << 30) : ad));
  }
  m = (int32_t)__reduce_max_sync(FULL_MASK, (unsigned)m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(span, m);
}

// row_ptr[r] = first unique key >= r * ncols, for r in [0, nrows].
__global__ void k_row_ptr(const uint64_t *ukey, int64_t nnz, int64_t ncols, int64_t nrows,
                          int32_t *row_ptr) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t target = (uint64_t)r * (uint64_t)ncols;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ukey[mid] < target) lo = mid + 1; else hi = mid;
    }
    row_ptr[r] = (int32_t)lo;
  }
}

__global__ void k_max_row(const int32_t *row_ptr, int64_t nrows, int32_t *out) {
  int32_t m = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x)
    m = max(m, row_ptr[r + 1] - row_ptr[r]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(FULL_MASK, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

static unsigned grid_for(int64_t n, int tpb) {
  int64_t g = (n + tpb - 1) / tpb;
  if (g < 1) g = 1;
  if (g > 1048576) g = 1048576;
  return (unsigned)g;
}

// Error exits of the symbolic stages: set status and jump to cleanup.
#define SYM_CUDA(call)                                                            \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      status = (e_ == cudaErrorMemoryAllocation) ? GBS_ERR_ALLOC : GBS_ERR_CUDA;  \
      goto cleanup;                                                               \
    }                                                                             \
  } while (0)
#define SYM_TRY(call)                                                             \
  do {                                                                            \
    status = (call);                                                              \
    if (status != GBS_OK) goto cleanup;                                           \
  } while (0)

// ------------------------------------------------------------------ row-bucketed symbolic stage
//
// The symbolic stage for patterns whose rows hold at most ROW_SORT_CTA COO
// entries (finite-element, stencil and graph matrices): no global sort.
//   1. per-row counts of the kept entries (warp-aggregated atomics: one
//      atomic per distinct row in a warp);
//   2. their exclusive scan -> each row's range of the kept entries;
//   3. every kept entry placed in its row's range as the 64-bit key
//      (j << 32) | k (the order inside a row depends on atomic timing);
//   4. each row sorted by that key (a warp's register bitonic sort up to
//      ROW_SORT_WARP entries, a CTA's shared-memory one up to ROW_SORT_CTA):
//      the keys are distinct, so the result is the same on every run, and it
//      is the order of the radix path -- rows ascending, columns ascending,
//      equal (i, j) by increasing COO index; the low halves are perm, and
//      each row's distinct columns are counted;
//   5. the scan of those counts is row_ptr (and nnz), and one pass writes
//      col, jmap and the diagonal positions.
// Traffic: about 56 bytes per kept entry, against about 140 for the 5-pass
// radix sort of 40-bit keys.  A longer row sends the pattern to the radix
// path.
constexpr int ROW_SORT_WARP = 64, ROW_SORT_CTA = 4096, ROW_SORT_TPB = 512;

// The lanes in `active` that share `key` add their count to cnt[key] with one
// atomic; returns the old value, and in rank each lane's position among them.
__device__ __forceinline__ uint32_t warp_agg_add(uint32_t *cnt, uint32_t key, unsigned active,
                                                 uint32_t &rank) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(active, key);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(cnt + key, (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
  return base;
}

// mode 0: count the kept entries per row (and flag out-of-range indices);
// mode 1: place each at rstart[row] + its slot as (j << 32) | k.
template <int MODE>
__global__ void k_row_bucket(KeepArgs a, uint32_t *cnt, const uint32_t *__restrict__ rstart,
                             uint64_t *keys, int32_t *err) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < a.ncoo;
       base += nw * 32) {
    const int64_t k = base + lane;
    int64_t gi = 0, gj = 0;
    bool bad = false;
    const bool keep = k < a.ncoo && keep_entry(a, k, gi, gj, bad);
    if (MODE == 0 && bad) atomicExch(err, GBS_ERR_INDEX);
    const unsigned active = __ballot_sync(FULL_MASK, keep);
    if (keep) {
      uint32_t rank;
      const uint32_t b = warp_agg_add(cnt, (uint32_t)gi, active, rank);
      if (MODE == 1)
        keys[rstart[gi] + b + rank] = ((uint64_t)(uint32_t)gj << 32) | (uint32_t)k;
    }
  }
}

// Ascending bitonic sort of 64 keys held two per lane (element 2 lane + h).
__device__ __forceinline__ void warp_sort64(uint64_t &a0, uint64_t &a1) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
    const bool asc = ((2 * lane) & k) == 0;
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 1) {
        const uint64_t lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
        a0 = asc ? lo : hi;
        a1 = asc ? hi : lo;
      } else {
        const int lj = j >> 1;
        const uint64_t b0 = __shfl_xor_sync(FULL_MASK, a0, lj);
        const uint64_t b1 = __shfl_xor_sync(FULL_MASK, a1, lj);
        const bool keep_min = ((lane & lj) == 0) == asc;
        a0 = keep_min ? (a0 < b0 ? a0 : b0) : (a0 < b0 ? b0 : a0);
        a1 = keep_min ? (a1 < b1 ? a1 : b1) : (a1 < b1 ? b1 : a1);
      }
    }
  }
}

// Rows of at most ROW_SORT_WARP entries, one warp each: sort, write back the
// keys and perm (their low halves), count the distinct columns into ucnt.
// Longer rows go to long_rows (count in *nlong) for k_row_sort_cta.
__global__ void k_row_sort_warp(int64_t nrows, const uint32_t *__restrict__ rstart,
                                uint64_t *__restrict__ keys, int32_t *__restrict__ perm,
                                uint32_t *__restrict__ ucnt, int32_t *__restrict__ long_rows,
                                uint32_t *nlong) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
    const uint32_t s0 = rstart[r];
    const int len = (int)(rstart[r + 1] - s0);
    if (len > ROW_SORT_WARP) {
      if (lane == 0) long_rows[atomicAdd(nlong, 1u)] = (int32_t)r;
      continue;
    }
    const int q0 = 2 * lane, q1 = 2 * lane + 1;
    uint64_t a0 = q0 < len ? keys[s0 + q0] : ~0ull, a1 = q1 < len ? keys[s0 + q1] : ~0ull;
    warp_sort64(a0, a1);
    const uint32_t j0 = (uint32_t)(a0 >> 32), j1 = (uint32_t)(a1 >> 32);
    const uint32_t jprev = __shfl_up_sync(FULL_MASK, j1, 1);
    const bool h0 = q0 < len && (lane == 0 || j0 != jprev), h1 = q1 < len && j1 != j0;
    if (q0 < len) {
      keys[s0 + q0] = a0;
      perm[s0 + q0] = (int32_t)(uint32_t)a0;
    }
    if (q1 < len) {
      keys[s0 + q1] = a1;
      perm[s0 + q1] = (int32_t)(uint32_t)a1;
    }
    const int u = __popc(__ballot_sync(FULL_MASK, h0)) + __popc(__ballot_sync(FULL_MASK, h1));
    if (lane == 0) ucnt[r] = (uint32_t)u;
  }
}

// The long rows (ROW_SORT_WARP < len <= ROW_SORT_CTA), one CTA each: a
// bitonic sort in shared memory, then as k_row_sort_warp.
__global__ void __launch_bounds__(ROW_SORT_TPB)
    k_row_sort_cta(const uint32_t *__restrict__ rstart, uint64_t *__restrict__ keys,
                   int32_t *__restrict__ perm, uint32_t *__restrict__ ucnt,
                   const int32_t *__restrict__ long_rows, const uint32_t *nlong) {
  __shared__ uint64_t sk[ROW_SORT_CTA];
  __shared__ int cnt_w[ROW_SORT_TPB / 32];
  const uint32_t nl = *nlong;
  for (uint32_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const int32_t r = long_rows[li];
    const uint32_t s0 = rstart[r];
    const int len = (int)(rstart[r + 1] - s0);
    int m = 1;
    while (m < len) m <<= 1;
    for (int q = threadIdx.x; q < m; q += blockDim.x) sk[q] = q < len ? keys[s0 + q] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
          const int pq = q ^ j;
          if (pq > q) {
            const uint64_t x = sk[q], y = sk[pq];
            const bool asc = (q & k) == 0;
            if ((x > y) == asc) {
              sk[q] = y;
              sk[pq] = x;
            }
          }
        }
        __syncthreads();
      }
    int u = 0;
    for (int q = threadIdx.x; q < len; q += blockDim.x) {
      const uint64_t x = sk[q];
      keys[s0 + q] = x;
      perm[s0 + q] = (int32_t)(uint32_t)x;
      u += (q == 0 || (x >> 32) != (sk[q - 1] >> 32)) ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) u += __shfl_xor_sync(FULL_MASK, u, off);
    if ((threadIdx.x & 31) == 0) cnt_w[threadIdx.x >> 5] = u;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += cnt_w[w];
      ucnt[r] = (uint32_t)t;
    }
    __syncthreads();
  }
}

// col, jmap and diag_pos from the sorted rows, one warp per row; the
// largest |col - row| into *span.
__global__ void k_row_emit(int64_t nrows, const uint32_t *__restrict__ rstart,
                           const uint64_t *__restrict__ keys, const int32_t *__restrict__ row_ptr,
                           int32_t *__restrict__ jmap, int32_t *__restrict__ col,
                           int32_t *__restrict__ diag_pos, int32_t *span) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t m = 0;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
    const uint32_t s0 = rstart[r];
    const int len = (int)(rstart[r + 1] - s0);
    int run = row_ptr[r];
    uint32_t prev = 0;  // the column of the chunk's previous entry (lane 31 of the last chunk)
    for (int c = 0; c < len; c += 32) {
      const int q = c + lane;
      const bool valid = q < len;
      const uint32_t jq = valid ? (uint32_t)(keys[s0 + q] >> 32) : 0u;
      const uint32_t jl = __shfl_up_sync(FULL_MASK, jq, 1);
      const uint32_t before = lane == 0 ? prev : jl;
      const bool head = valid && (q == 0 || jq != before);
      const unsigned hb = __ballot_sync(FULL_MASK, head);
      if (head) {
        const int u = run + __popc(hb & ((1u << lane) - 1u));
        jmap[u] = (int32_t)(s0 + q);
        col[u] = (int32_t)jq;
        if ((int64_t)jq == r) diag_pos[r] = u;
        const int64_t d = (int64_t)jq - r, ad = d < 0 ? -d : d;
        m = max(m, (int32_t)(ad > (1 << 30) ? (1 << 30) : ad));
      }
      run += __popc(hb);
      prev = __shfl_sync(FULL_MASK, jq, 31);
    }
  }
  m = (int32_t)__reduce_max_sync(FULL_MASK, (unsigned)m);
  if (lane == 0 && m > 0) atomicMax(span, m);
}

// Symbolic stage.  coo_off_h (host, nsys+1) is non-null for batched handles;
// A->row_off_h, nrows, ncols, ncoo, nsys are set by the caller.  The
// row-bucketed path runs unless a row holds more than ROW_SORT_CTA entries.
static int symbolic_radix(gbs_mat A, const int32_t *i, const int32_t *j,
                          const int64_t *coo_off_h, cudaStream_t s);
static int symbolic_rows(gbs_mat A, const int32_t *i, const int32_t *j,
                         const int64_t *coo_off_h, cudaStream_t s, bool *done);

int symbolic(gbs_mat A, const int32_t *i, const int32_t *j, const int64_t *coo_off_h,
             cudaStream_t s) {
  bool done = false;
  const int st = symbolic_rows(A, i, j, coo_off_h, s, &done);
  if (st != GBS_OK || done) return st;
  return symbolic_radix(A, i, j, coo_off_h, s);
}

static int symbolic_rows(gbs_mat A, const int32_t *i, const int32_t *j,
                         const int64_t *coo_off_h, cudaStream_t s, bool *done) {
  *done = false;
  const int64_t ncoo = A->ncoo, n = A->nrows;
  KeepArgs ka{i, j, ncoo, A->nrows, A->ncols, nullptr, nullptr, A->nsys};
  int64_t *d_off = nullptr;
  uint32_t *cnt = nullptr, *rstart = nullptr, *scan_tmp = nullptr, *ucnt = nullptr;
  uint64_t *keys = nullptr;
  int32_t *perm = nullptr, *long_rows = nullptr;
  int status = GBS_OK;
  struct Ctl {
    uint32_t nkept, nnz;
    int32_t err, maxcnt, maxrow, span;
    uint32_t nlong, pad;
  } hc{};
  Ctl *dctl = nullptr;
  const int64_t n1 = std::max<int64_t>(n, 1);
  const int64_t nwarp_rows = std::max<int64_t>(n, 1) * 32;

  {
    SYM_TRY(dev_alloc(&dctl, 1, s));
    SYM_CUDA(cudaMemsetAsync(dctl, 0, sizeof(Ctl), s));
    if (coo_off_h) {
      SYM_TRY(dev_alloc(&d_off, 2 * (A->nsys + 1), s));
      SYM_CUDA(cudaMemcpyAsync(d_off, coo_off_h, sizeof(int64_t) * (A->nsys + 1),
                               cudaMemcpyHostToDevice, s));
      SYM_CUDA(cudaMemcpyAsync(d_off + A->nsys + 1, A->row_off_h.data(),
                               sizeof(int64_t) * (A->nsys + 1), cudaMemcpyHostToDevice, s));
      ka.coo_off = d_off;
      ka.row_off = d_off + A->nsys + 1;
    }
    // 1-2. counts per row, their scan (total: nkept), the largest count
    SYM_TRY(dev_alloc(&cnt, n1 + 1, s));
    SYM_TRY(dev_alloc(&rstart, n1 + 1, s));
    SYM_TRY(dev_alloc(&scan_tmp, scan_tmp_words(n1 + 1), s));
    SYM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (n1 + 1), s));
    if (ncoo > 0) {
      k_row_bucket<0><<<grid_for(ncoo, 256), 256, 0, s>>>(ka, cnt, nullptr, nullptr, &dctl->err);
      GBS_LAUNCHED(1);
    }
    SYM_TRY(exclusive_scan(cnt, rstart, n + 1, scan_tmp, &dctl->nkept, s));
    if (n > 0) {
      k_max_row<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const int32_t *>(rstart), n,
                                                 &dctl->maxcnt);
      GBS_LAUNCHED(1);
    }
    SYM_CUDA(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    if (hc.err != 0) {
      set_error("mat_create_coo: a kept COO index is out of range");
      status = GBS_ERR_INDEX;
      goto cleanup;
    }
    if (hc.maxcnt > ROW_SORT_CTA) goto cleanup;  // the radix path takes it
    const int64_t nkept = hc.nkept;
    const int64_t nk = std::max<int64_t>(nkept, 1);
    // 3. placement
    SYM_TRY(dev_alloc(&keys, nk, s));
    SYM_TRY(dev_alloc(&perm, nk, s));
    SYM_TRY(dev_alloc(&ucnt, n1 + 1, s));
    SYM_TRY(dev_alloc(&long_rows, n1, s));
    SYM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (n1 + 1), s));
    SYM_CUDA(cudaMemsetAsync(ucnt, 0, sizeof(uint32_t) * (n1 + 1), s));
    if (ncoo > 0) {
      k_row_bucket<1><<<grid_for(ncoo, 256), 256, 0, s>>>(ka, cnt, rstart, keys, nullptr);
      GBS_LAUNCHED(1);
    }
    // 4. per-row sorts, distinct columns
    if (n > 0) {
      k_row_sort_warp<<<grid_for(nwarp_rows, 256), 256, 0, s>>>(n, rstart, keys, perm, ucnt,
                                                                 long_rows, &dctl->nlong);
      k_row_sort_cta<<<1024, ROW_SORT_TPB, 0, s>>>(rstart, keys, perm, ucnt, long_rows,
                                                   &dctl->nlong);
      GBS_LAUNCHED(2);
    }
    // 5. row_ptr, nnz; then col, jmap, diagonal positions
    SYM_TRY(dev_alloc(&A->row_ptr, n + 1, s));
    SYM_TRY(exclusive_scan(ucnt, reinterpret_cast<uint32_t *>(A->row_ptr), n + 1, scan_tmp,
                           &dctl->nnz, s));
    SYM_CUDA(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    const int64_t nnz = hc.nnz;
    A->nkept = nkept;
    A->nnz = nnz;
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    SYM_TRY(dev_alloc(&A->jmap, nnz + 1, s));
    SYM_TRY(dev_alloc(&A->col, nz1, s));
    SYM_TRY(dev_alloc(&A->val, nz1, s));
    SYM_TRY(dev_alloc(&A->diag_pos, n1, s));
    SYM_TRY(dev_alloc(&A->dinv, n1, s));
    SYM_CUDA(cudaMemsetAsync(A->val, 0, sizeof(double) * nz1, s));
    SYM_CUDA(cudaMemsetAsync(A->diag_pos, 0xff, sizeof(int32_t) * n1, s));
    SYM_CUDA(cudaMemsetAsync(A->dinv, 0, sizeof(double) * n1, s));
    {
      const int32_t nk32 = (int32_t)nkept;
      SYM_CUDA(cudaMemcpyAsync(A->jmap + nnz, &nk32, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    if (n > 0) {
      k_row_emit<<<grid_for(nwarp_rows, 256), 256, 0, s>>>(n, rstart, keys, A->row_ptr, A->jmap,
                                                            A->col, A->diag_pos, &dctl->span);
      k_max_row<<<grid_for(n, 256), 256, 0, s>>>(A->row_ptr, n, &dctl->maxrow);
      GBS_LAUNCHED(2);
    }
    SYM_CUDA(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    A->max_row_nnz = hc.maxrow;
    A->col_span = hc.span;
    A->perm = perm;
    perm = nullptr;
    *done = true;
  }

cleanup:
  for (void *p : {(void *)dctl, (void *)d_off, (void *)cnt, (void *)rstart, (void *)scan_tmp,
                  (void *)ucnt, (void *)keys, (void *)perm, (void *)long_rows})
    dev_free(p, s);
  cudaStreamSynchronize(s);
  return status;
}

// The radix path: keep flags and compaction, a stable LSD radix sort of the
// 64-bit keys i * ncols + j, segment heads.
static int symbolic_radix(gbs_mat A, const int32_t *i, const int32_t *j,
                          const int64_t *coo_off_h, cudaStream_t s) {
  const int64_t ncoo = A->ncoo;
  KeepArgs ka{i, j, ncoo, A->nrows, A->ncols, nullptr, nullptr, A->nsys};
  int64_t *d_off = nullptr;
  uint32_t *flags = nullptr, *scan_tmp = nullptr, *dsc = nullptr;
  uint64_t *kA = nullptr, *kB = nullptr, *ukey = nullptr;
  uint32_t *vA = nullptr, *vB = nullptr, *counts = nullptr;
  int status = GBS_OK;
  // host mirrors read back after each synchronisation
  struct Ctl {
    uint32_t nkept, nnz;
    int32_t err, maxrow, span, pad;
  } hc{};
  Ctl *dctl = nullptr;


  {
    SYM_TRY(dev_alloc(&dctl, 1, s));
    SYM_CUDA(cudaMemsetAsync(dctl, 0, sizeof(Ctl), s));
    if (coo_off_h) {
      SYM_TRY(dev_alloc(&d_off, 2 * (A->nsys + 1), s));
      SYM_CUDA(cudaMemcpyAsync(d_off, coo_off_h, sizeof(int64_t) * (A->nsys + 1),
                               cudaMemcpyHostToDevice, s));
      SYM_CUDA(cudaMemcpyAsync(d_off + A->nsys + 1, A->row_off_h.data(),
                               sizeof(int64_t) * (A->nsys + 1), cudaMemcpyHostToDevice, s));
      ka.coo_off = d_off;
      ka.row_off = d_off + A->nsys + 1;
    }
    const int64_t nflag = std::max<int64_t>(ncoo, 1);
    SYM_TRY(dev_alloc(&flags, nflag, s));
    SYM_TRY(dev_alloc(&dsc, nflag, s));
    SYM_TRY(dev_alloc(&scan_tmp, scan_tmp_words(nflag), s));

    // 1. keep flags, positions, nkept
    if (ncoo > 0) {
      k_keep_flags<<<grid_for(ncoo, 256), 256, 0, s>>>(ka, flags, &dctl->err);
      GBS_LAUNCHED(1);
    }
    SYM_TRY(exclusive_scan(flags, dsc, ncoo, scan_tmp, &dctl->nkept, s));
    SYM_CUDA(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    if (hc.err != 0) {
      set_error("mat_create_coo: a kept COO index is out of range");
      status = GBS_ERR_INDEX;
      goto cleanup;
    }
    const int64_t nkept = hc.nkept;
    A->nkept = nkept;
    const int64_t nk = std::max<int64_t>(nkept, 1);
    SYM_TRY(dev_alloc(&kA, nk, s));
    SYM_TRY(dev_alloc(&kB, nk, s));
    SYM_TRY(dev_alloc(&vA, nk, s));
    SYM_TRY(dev_alloc(&vB, nk, s));  // becomes perm
    if (ncoo > 0) {
      k_compact<<<grid_for(ncoo, 256), 256, 0, s>>>(ka, dsc, kA, vA);
      GBS_LAUNCHED(1);
    }

    // 2. stable LSD radix sort (the scatter stages a tile in ~58 KB of shared memory)
    {
      static bool smem_opt_in = false;
      if (!smem_opt_in) {
        SYM_CUDA(cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(RadixShared)));
        smem_opt_in = true;
      }
    }
    const uint64_t maxkey = (uint64_t)A->nrows * (uint64_t)A->ncols;
    int bits = 0;
    while (bits < 64 && (maxkey > 1) && ((maxkey - 1) >> bits) != 0) ++bits;
    const int passes = (bits + 7) / 8;
    const int64_t ntiles = (nkept + RS_TILE - 1) / RS_TILE;
    if (ntiles > 0 && passes > 0) {
      const int64_t ncount = 256 * ntiles;
      SYM_TRY(dev_alloc(&counts, ncount, s));
      uint32_t *ctmp = nullptr;
      SYM_TRY(dev_alloc(&ctmp, scan_tmp_words(ncount), s));
      uint64_t *kin = kA, *kout = kB;
      uint32_t *vin = vA, *vout = vB;
      for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_radix_hist<<<(unsigned)ntiles, RS_T, 0, s>>>(kin, nkept, shift, counts, ntiles);
        GBS_LAUNCHED(1);
        status = exclusive_scan(counts, counts, ncount, ctmp, nullptr, s);
        if (status != GBS_OK) {
          dev_free(ctmp, s);
          goto cleanup;
        }
        k_radix_scatter<<<(unsigned)ntiles, RS_T, sizeof(RadixShared), s>>>(
            kin, vin, nkept, shift, counts, ntiles, kout, vout);
        GBS_LAUNCHED(1);
        std::swap(kin, kout);
        std::swap(vin, vout);
      }
      dev_free(ctmp, s);
      // sorted data is in kin / vin; make kA / vB hold it
      if (kin != kA) std::swap(kA, kB);
      if (vin != vB) {
        // vin == vA: copy into vB (the buffer that becomes perm)
        SYM_CUDA(cudaMemcpyAsync(vB, vA, sizeof(uint32_t) * nkept, cudaMemcpyDeviceToDevice, s));
      }
    } else if (nkept > 0) {
      SYM_CUDA(cudaMemcpyAsync(vB, vA, sizeof(uint32_t) * nkept, cudaMemcpyDeviceToDevice, s));
    }

    // 3. segments
    if (nkept > 0) {
      k_seg_flags<<<grid_for(nkept, 256), 256, 0, s>>>(kA, nkept, flags);
      GBS_LAUNCHED(1);
    }
    SYM_TRY(exclusive_scan(flags, dsc, nkept, scan_tmp, &dctl->nnz, s));
    SYM_CUDA(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    const int64_t nnz = hc.nnz;
    A->nnz = nnz;
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    SYM_TRY(dev_alloc(&A->jmap, nnz + 1, s));
    SYM_TRY(dev_alloc(&A->col, nz1, s));
    SYM_TRY(dev_alloc(&A->val, nz1, s));
    SYM_TRY(dev_alloc(&A->row_ptr, A->nrows + 1, s));
    SYM_TRY(dev_alloc(&A->diag_pos, std::max<int64_t>(A->nrows, 1), s));
    SYM_TRY(dev_alloc(&A->dinv, std::max<int64_t>(A->nrows, 1), s));
    SYM_CUDA(cudaMemsetAsync(A->val, 0, sizeof(double) * nz1, s));
    SYM_CUDA(cudaMemsetAsync(A->diag_pos, 0xff, sizeof(int32_t) * std::max<int64_t>(A->nrows, 1), s));
    SYM_CUDA(cudaMemsetAsync(A->dinv, 0, sizeof(double) * std::max<int64_t>(A->nrows, 1), s));
    SYM_TRY(dev_alloc(&ukey, nz1, s));
    A->perm = (int32_t *)vB;
    vB = nullptr;
    {
      const int32_t nk32 = (int32_t)nkept;
      SYM_CUDA(cudaMemcpyAsync(A->jmap + nnz, &nk32, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    if (nkept > 0) {
      k_seg_write<<<grid_for(nkept, 256), 256, 0, s>>>(kA, nkept, flags, dsc, ukey, A->jmap);
      GBS_LAUNCHED(1);
    }
    if (nnz > 0) {
      k_csr_cols<<<grid_for(nnz, 256), 256, 0, s>>>(ukey, nnz, A->ncols, A->col, A->diag_pos,
                                                    &dctl->span);
      GBS_LAUNCHED(1);
    }
    k_row_ptr<<<grid_for(A->nrows + 1, 256), 256, 0, s>>>(ukey, nnz, A->ncols, A->nrows,
                                                          A->row_ptr);
    k_max_row<<<grid_for(A->nrows, 256), 256, 0, s>>>(A->row_ptr, A->nrows, &dctl->maxrow);
    GBS_LAUNCHED(2);
    SYM_CUDA(cudaMemcpyAsync(&hc, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    A->max_row_nnz = hc.maxrow;
    A->col_span = hc.span;
  }

cleanup:
  for (void *p : {(void *)dctl, (void *)d_off, (void *)flags, (void *)dsc, (void *)scan_tmp,
                  (void *)kA, (void *)kB, (void *)vA, (void *)counts, (void *)ukey, (void *)vB})
    dev_free(p, s);
  cudaStreamSynchronize(s);
  return status;
}

// ------------------------------------------------------------------ numeric

// One thread per nonzero: a_p = v[perm[jmap[p]]] + v[perm[jmap[p]+1]] + ...
// in increasing COO index order (Sec. 5: each thread accumulates into a single
// nonzero, no atomics).  A segment's sum is a chain of dependent FP64 adds,
// and a warp issues each add step for all its lanes: with consecutive
// nonzeros on consecutive lanes every warp runs as many steps as its longest
// segment (on the Q1 matrix segments hold 1, 2, 4 or 8 terms and nearly every
// warp an 8), and FP64 instructions, scarce on this part, bound the kernel.
// So a CTA takes a tile of NUM_TILE consecutive nonzeros, orders them by
// segment length in shared memory (a counting sort over a few length
// classes), and its warps sum them in that order -- lanes of a warp then
// hold segments of about one length and issue only the adds those need --
// into a shared buffer that the CTA writes back in nonzero order (coalesced).
// Each thread takes two nonzeros and loads each segment's COO indices
// NUM_BATCH at a time before their values, so its two chains of dependent
// loads (COO indices -> values) are in flight together.  The lane a nonzero
// lands on depends on shared-memory atomics; its sum does not.
constexpr int NUM_BATCH = 4;
constexpr int NUM_TPB = 256, NUM_TILE = 2 * NUM_TPB, NUM_CLASSES = 5;

__device__ __forceinline__ int length_class(int32_t len) {
  return len <= 1 ? 0 : (len == 2 ? 1 : (len <= 4 ? 2 : (len <= 8 ? 3 : 4)));
}

__global__ void __launch_bounds__(NUM_TPB)
    k_coo_numeric(int64_t nnz, const int32_t *__restrict__ jmap,
                  const int32_t *__restrict__ perm, const double *__restrict__ v, int mode,
                  double *__restrict__ val) {
  __shared__ int32_t s_j0[NUM_TILE], s_j1[NUM_TILE];
  __shared__ int16_t s_order[NUM_TILE];
  __shared__ double s_sum[NUM_TILE];
  __shared__ int32_t s_cnt[NUM_CLASSES], s_base[NUM_CLASSES];
  const int tid = (int)threadIdx.x;
  for (int64_t t0 = (int64_t)blockIdx.x * NUM_TILE; t0 < nnz;
       t0 += (int64_t)gridDim.x * NUM_TILE) {
    const int nt = nnz - t0 < NUM_TILE ? (int)(nnz - t0) : NUM_TILE;
    if (tid < NUM_CLASSES) s_cnt[tid] = 0;
    __syncthreads();
    // 1. segment bounds and length classes; ranks within a class
    int cls[2], rank[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = tid + h * NUM_TPB;
      cls[h] = -1;
      if (i < nt) {
        const int32_t j0 = __ldg(jmap + t0 + i), j1 = __ldg(jmap + t0 + i + 1);
        s_j0[i] = j0;
        s_j1[i] = j1;
        cls[h] = length_class(j1 - j0);
        rank[h] = atomicAdd(&s_cnt[cls[h]], 1);
      }
    }
    __syncthreads();
    if (tid == 0) {
      int b = 0;
      for (int c = 0; c < NUM_CLASSES; ++c) {
        s_base[c] = b;
        b += s_cnt[c];
      }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (cls[h] >= 0) s_order[s_base[cls[h]] + rank[h]] = (int16_t)(tid + h * NUM_TPB);
    __syncthreads();
    // 2. the sums, in class order: positions tid and tid + NUM_TPB
    const bool has_a = tid < nt, has_b = tid + NUM_TPB < nt;
    const int ia = has_a ? s_order[tid] : 0, ib = has_b ? s_order[tid + NUM_TPB] : 0;
    int32_t ta = has_a ? s_j0[ia] : 0, tb = has_b ? s_j0[ib] : 0;
    const int32_t ea = has_a ? s_j1[ia] : 0, eb = has_b ? s_j1[ib] : 0;
    double sa = 0.0, sb = 0.0;
    for (bool first = true; ta < ea || tb < eb; first = false) {
      int32_t ka[NUM_BATCH], kb[NUM_BATCH];
      double xa[NUM_BATCH], xb[NUM_BATCH];
#pragma unroll
      for (int u = 0; u < NUM_BATCH; ++u) {
        ka[u] = ta + u < ea ? __ldg(perm + ta + u) : 0;
        kb[u] = tb + u < eb ? __ldg(perm + tb + u) : 0;
      }
#pragma unroll
      for (int u = 0; u < NUM_BATCH; ++u) {
        xa[u] = ta + u < ea ? __ldg(v + ka[u]) : 0.0;
        xb[u] = tb + u < eb ? __ldg(v + kb[u]) : 0.0;
      }
      if (first) {  // a segment's first term starts its sum
        sa = xa[0];
        sb = xb[0];
      }
#pragma unroll
      for (int u = 0; u < NUM_BATCH; ++u) {  // in increasing COO index: plain adds
        if ((!first || u > 0) && ta + u < ea) sa = __dadd_rn(sa, xa[u]);
        if ((!first || u > 0) && tb + u < eb) sb = __dadd_rn(sb, xb[u]);
      }
      ta += NUM_BATCH;
      tb += NUM_BATCH;
    }
    if (has_a) s_sum[ia] = sa;
    if (has_b) s_sum[ib] = sb;
    __syncthreads();
    // 3. back in nonzero order
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = tid + h * NUM_TPB;
      if (i < nt) {
        const double x = s_sum[i];
        val[t0 + i] = (mode == GBS_ADD) ? __dadd_rn(val[t0 + i], x) : x;
      }
    }
    __syncthreads();  // the shared arrays are reused by the next tile
  }
}

// Jacobi: dinv_r = 1 / a_rr; a missing or non-positive diagonal stores 0,
// which the solves report as GBS_ERR_NOT_SPD for the system holding that row.
__global__ void k_jacobi(int64_t nrows, const int32_t *__restrict__ diag_pos,
                         const double *__restrict__ val, double *__restrict__ dinv) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = diag_pos[r];
    const double d = q >= 0 ? val[q] : 0.0;
    dinv[r] = (d > 0.0) ? 1.0 / d : 0.0;
  }
}

int launch_set_values(gbs_mat A, const double *v, int mode, cudaStream_t s) {
  if (A->nnz > 0) {
    k_coo_numeric<<<grid_for((A->nnz + NUM_TILE - 1) / NUM_TILE, 1), NUM_TPB, 0, s>>>(
        A->nnz, A->jmap, A->perm, v, mode, A->val);
    GBS_LAUNCHED(1);
  }
  if (A->nrows > 0) {
    k_jacobi<<<grid_for(A->nrows, 256), 256, 0, s>>>(A->nrows, A->diag_pos, A->val, A->dinv);
    GBS_LAUNCHED(1);
  }
  GBS_TRY(sell_values(A, s));
  A->values_set = true;
  A->val32_valid = false;
  A->values_version += 1;
  return GBS_OK;
}

// FP32 copies for the refined solve: val32 = RN(val), dinv32 = RN(dinv).
__global__ void k_to_fp32(int64_t nnz, const double *__restrict__ val, float *__restrict__ val32,
                          int64_t nrows, const double *__restrict__ dinv,
                          float *__restrict__ dinv32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
    val32[p] = __double2float_rn(val[p]);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride)
    dinv32[r] = __double2float_rn(dinv[r]);
}

int launch_to_fp32(gbs_mat A, cudaStream_t s) {
  if (!A->val32) {
    GBS_TRY(dev_alloc(&A->val32, std::max<int64_t>(A->nnz, 1), s));
    GBS_TRY(dev_alloc(&A->dinv32, std::max<int64_t>(A->nrows, 1), s));
  }
  k_to_fp32<<<grid_for(std::max(A->nnz, A->nrows), 256), 256, 0, s>>>(
      A->nnz, A->val, A->val32, A->nrows, A->dinv, A->dinv32);
  GBS_LAUNCHED(1);
  GBS_TRY(sell_values32(A, s));
  A->val32_valid = true;
  return GBS_OK;
}

// ------------------------------------------------------------------ vectors

// y[r] = a_{p(r)} (INSERT) or y[r] + a_{p(r)} (ADD) for every index r that
// has an entry (its row of the n x 1 pattern is non-empty); other y[r] keep.
__global__ void k_vec_scatter(int64_t n, const int32_t *__restrict__ row_ptr,
                              const double *__restrict__ val, int mode, double *__restrict__ y) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = row_ptr[r];
    if (row_ptr[r + 1] > p) y[r] = (mode == GBS_ADD) ? y[r] + val[p] : val[p];
  }
}

// Vector numeric stage: the in-order sums of the n x 1 pattern (the matrix
// numeric kernel, INSERT into val), then the scatter into y.
int launch_vec_set_values(gbs_mat A, const double *v, int mode, double *y, cudaStream_t s) {
  if (A->nnz > 0) {
    k_coo_numeric<<<grid_for((A->nnz + NUM_TILE - 1) / NUM_TILE, 1), NUM_TPB, 0, s>>>(
        A->nnz, A->jmap, A->perm, v, GBS_INSERT, A->val);
    GBS_LAUNCHED(1);
  }
  if (A->nrows > 0) {
    k_vec_scatter<<<grid_for(A->nrows, 256), 256, 0, s>>>(A->nrows, A->row_ptr, A->val, mode, y);
    GBS_LAUNCHED(1);
  }
  return GBS_OK;
}

// ------------------------------------------------------------------ adjoint scatter

// dLda[p] = -lambda[row p] * x[col p]; dLdv[perm[t]] = dLda[p] for t in the
// segment of p.  One thread per nonzero, so the reads of col, jmap and perm
// and the writes of dLda are coalesced.  A warp takes 32 consecutive
// nonzeros: lane 0 finds the row of the first by binary search over row_ptr
// (the last r with row_ptr[r] <= p0, which skips empty rows), and each lane
// walks forward from there to its own row -- at most the number of rows the
// warp's nonzeros span.  Ignored COO entries are zeroed by the caller's
// memset.
__global__ void k_adjoint_scatter(int64_t nnz, int64_t nrows, const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col,
                                  const int32_t *__restrict__ jmap,
                                  const int32_t *__restrict__ perm,
                                  const double *__restrict__ lambda,
                                  const double *__restrict__ x, double *__restrict__ dLda,
                                  double *__restrict__ dLdv) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c * 32 < nnz; c += nw) {
    const int64_t p0 = c * 32, p = p0 + lane;
    int64_t r0 = 0;
    if (lane == 0) {
      int64_t lo = 0, hi = nrows;  // row_ptr[0] = 0 <= p0 < nnz = row_ptr[nrows]
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (row_ptr[mid] <= p0) lo = mid;
        else hi = mid - 1;
      }
      r0 = lo;
    }
    r0 = __shfl_sync(FULL_MASK, r0, 0);
    if (p < nnz) {
      int64_t r = r0;
      while (row_ptr[r + 1] <= p) ++r;
      const double g = -(lambda[r] * x[col[p]]);
      if (dLda) dLda[p] = g;
      if (dLdv)
        for (int32_t t = jmap[p]; t < jmap[p + 1]; ++t) dLdv[perm[t]] = g;
    }
  }
}

int launch_adjoint_scatter(gbs_mat A, const double *lambda, const double *x, double *dLda,
                           double *dLdv, cudaStream_t s) {
  if (dLdv && A->ncoo > 0 && A->nkept < A->ncoo)
    GBS_TRY_CUDA(cudaMemsetAsync(dLdv, 0, sizeof(double) * A->ncoo, s));
  if ((dLda || dLdv) && A->nnz > 0) {
    k_adjoint_scatter<<<grid_for((A->nnz + 31) / 32 * 32, 256), 256, 0, s>>>(
        A->nnz, A->nrows, A->row_ptr, A->col, A->jmap, A->perm, lambda, x, dLda, dLdv);
    GBS_LAUNCHED(1);
  }
  return GBS_OK;
}

}  // namespace gbs
