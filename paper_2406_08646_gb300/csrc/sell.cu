// Sliced-ELL copy of the assembled CSR matrix for the row products of the
// solves and of MatMult (Sec. 6.1).  The CSR arrays stay the assembled matrix
// (Sec. 5); this copy only changes how a warp reads it.
//
// Rows are cut into slices of 32 consecutive rows (aligned to each system's
// first row, so no slice straddles two systems).  Slice s has width w_s (its
// longest row) and holds 32 x w_s entries from b = sell_ptr[s] on, padding
// with column -1 and value 0.  Entries 2m and 2m + 1 of the slice's row i sit
// side by side at b + 64 m + 2 i (+1) for m < w_s / 2; an odd last entry sits
// at b + 64 (w_s / 2) + i.  A warp reads one slice with lane i on row i: each
// load instruction fetches a contiguous 256-byte (columns, FP32 values) or
// 512-byte (FP64 values) run holding two entries per lane, the x gathers of a
// stencil-like pattern are contiguous too, each row is summed in CSR order
// with one FMA per stored nonzero, and no cross-lane adds are needed.  b is a
// multiple of 32 entries, so the paired loads are aligned.
//
// Column patterns.  When the rows of every slice draw their offsets col -
// row from a common set of at most 32 (a stencil matrix's slices), each slice
// stores that set once (its pattern, ascending) and one 32-bit mask per row
// (bit k: the row holds pattern entry k); entry k of row i is then the value
// at the pattern's k-th offset, 0 where the row lacks it, and the slice's
// width is the pattern's size U.  The row products then read no column
// index: the columns follow from the row, the pattern (one broadcast load a
// pair) and the mask, which also skips the absent entries, so each row still
// takes one FMA per nonzero in CSR order (the same sums, bit for bit, as with
// column indices).  The copy takes patterns when every slice has U <= 32 and
// the U add up to at most 1.25 times the slices' longest rows (which bounds
// the zeros they add; slices across a layer seam of a stencil have U above
// their longest row); else it keeps column indices.  8 bytes per FP64 entry
// plus 4 per row instead of 10 or 12.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

static unsigned grid_of(int64_t n, int tpb) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + tpb - 1) / tpb, 1 << 20));
}

// The union of the offsets col - row of a slice's rows (lane i holds row r,
// its entries [j, je)), smallest first, by repeated warp minima over the
// rows' next offsets (a row's offsets ascend).  Returns its size, or 33 once
// it passes 32.  With pool set, lane 0 writes the offsets there and *mk gets
// each lane's mask.
__device__ int slice_union(const int32_t *__restrict__ col, int32_t r, int32_t j, int32_t je,
                           int lane, int32_t *__restrict__ pool, uint32_t *mk) {
  uint32_t m = 0;
  int n = 0;
  for (;;) {
    const int32_t c = j < je ? col[j] - r : INT32_MAX;
    const int32_t lo = __reduce_min_sync(0xffffffffu, c);
    if (lo == INT32_MAX) break;
    if (n == 32) return 33;
    if (c == lo) {
      m |= 1u << n;
      ++j;
    }
    if (pool && lane == 0) pool[n] = lo;
    ++n;
  }
  if (mk) *mk = m;
  return n;
}

// One warp per slice: w[s] = its longest row; u[s] = the size of its rows'
// offset union (33: more than 32, or patterns not built).
__global__ void k_slice_shape(int64_t nslices, const int32_t *__restrict__ srow0,
                              const int32_t *__restrict__ row_ptr,
                              const int32_t *__restrict__ col, int32_t patterns,
                              int32_t *__restrict__ w, int32_t *__restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nslices; s += nw) {
    const int32_t r = srow0[s] + lane;
    const bool live = r < srow0[s + 1];
    const int32_t rs = live ? row_ptr[r] : 0, re = live ? row_ptr[r + 1] : 0;
    const int32_t m = __reduce_max_sync(0xffffffffu, re - rs);
    const int n = patterns ? slice_union(col, r, rs, re, lane, nullptr, nullptr) : 33;
    if (lane == 0) {
      w[s] = m;
      u[s] = n;
    }
  }
}

// Position of entry k of a lane's row in slice storage from b on (pair
// layout; np = width / 2).
__device__ __forceinline__ int64_t sell_slot(int64_t b, int32_t k, int32_t np, int lane) {
  return k < 2 * np ? b + 64 * (k >> 1) + 2 * lane + (k & 1) : b + 64 * np + lane;
}

// Columns (SYM: with pat set each slice's pattern and row masks, else 32-bit
// columns or 16-bit offsets col - row, padding -1 / -32768) or values (0 in
// padding and in pattern entries a row lacks) of the sliced copy: one warp
// per slice, lane i on row i of the slice.
template <typename T, bool SYM>
__global__ void k_sell_fill(int64_t nslices, const int32_t *__restrict__ sptr,
                            const int32_t *__restrict__ srow0, const int32_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col, const T *__restrict__ val,
                            const int32_t *__restrict__ pat, int32_t *__restrict__ pool,
                            uint32_t *__restrict__ mask, int32_t *__restrict__ scol,
                            int16_t *__restrict__ soff, T *__restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nslices; s += nw) {
    const int32_t r = srow0[s] + lane;
    const bool live = r < srow0[s + 1];
    const int32_t rs = live ? row_ptr[r] : 0, len = live ? row_ptr[r + 1] - rs : 0;
    const int64_t b = sptr[s];
    const int32_t w = (int32_t)((sptr[s + 1] - b) >> 5), np = w >> 1;
    if (pat) {
      if constexpr (SYM) {
        uint32_t mk = 0;
        slice_union(col, r, rs, rs + len, lane, pool + pat[s], &mk);
        mask[32 * s + lane] = mk;
      } else {
        const uint32_t mk = mask[32 * s + lane];
        int32_t j = rs;
        for (int32_t k = 0; k < w; ++k) {
          const bool has = (mk >> k) & 1u;
          sval[sell_slot(b, k, np, lane)] = has ? val[j] : T(0);
          j += has ? 1 : 0;
        }
      }
      continue;
    }
    for (int32_t k = 0; k < w; ++k) {
      const bool ok = k < len;
      const int64_t q = sell_slot(b, k, np, lane);
      if constexpr (SYM) {
        if (scol) scol[q] = ok ? col[rs + k] : -1;
        if (soff) soff[q] = ok ? (int16_t)(col[rs + k] - r) : (int16_t)-32768;
      } else {
        sval[q] = ok ? val[rs + k] : T(0);
      }
    }
  }
}

// FP32 values of the sliced copy, RN(FP64 values), padding stays 0.
__global__ void k_sell_to_fp32(int64_t n, const double *__restrict__ v, float *__restrict__ v32) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    v32[p] = __double2float_rn(v[p]);
}

void free_sell(gbs_mat A) {
  for (void *p : {(void *)A->sell_ptr, (void *)A->sell_row0, (void *)A->sell_col,
                  (void *)A->sell_off16, (void *)A->sell_val, (void *)A->sell_val32,
                  (void *)A->sell_pat, (void *)A->sell_pool, (void *)A->sell_mask})
    dev_free(p, nullptr);
  A->sell_pat = nullptr;
  A->sell_pool = nullptr;
  A->sell_mask = nullptr;
  A->sell_npat = 0;
  A->sell_nnz_rows = 0;
  A->sell_ptr = nullptr;
  A->sell_row0 = nullptr;
  A->sell_col = nullptr;
  A->sell_off16 = nullptr;
  A->sell_val = nullptr;
  A->sell_val32 = nullptr;
  A->nslices = A->sell_nnz = 0;
}

// Slice table, column patterns chosen and padded size (no entries yet); when
// the padded size reaches 2^31 only the size is recorded.  Idempotent.
// Synchronises s once (the slice widths decide the sizes).
int sell_shape(gbs_mat A, cudaStream_t st) {
  if (A->sell_row0) return GBS_OK;
  std::vector<int32_t> srow0;
  for (int32_t q = 0; q < A->nsys; ++q)
    for (int64_t r = A->row_off_h[q]; r < A->row_off_h[q + 1]; r += 32) srow0.push_back((int32_t)r);
  const int64_t ns = (int64_t)srow0.size();
  srow0.push_back((int32_t)A->nrows);
  std::vector<int32_t> w(std::max<int64_t>(ns, 1), 0), u(std::max<int64_t>(ns, 1), 33);
  GBS_TRY(dev_alloc(&A->sell_row0, ns + 1, st));
  GBS_TRY_CUDA(cudaMemcpyAsync(A->sell_row0, srow0.data(), sizeof(int32_t) * (ns + 1),
                               cudaMemcpyHostToDevice, st));
  if (ns > 0) {
    int32_t *dw = nullptr;
    GBS_TRY(dev_alloc(&dw, 2 * ns, st));
    k_slice_shape<<<grid_of(ns * 32, 256), 256, 0, st>>>(
        ns, A->sell_row0, A->row_ptr, A->col, A->sell_patterns ? 1 : 0, dw, dw + ns);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.data(), dw, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(u.data(), dw + ns, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(dw, st);
    count_launches(1);
    GBS_TRY_CUDA(e);
  }
  // patterns when every slice has at most 32 offsets and they add at most a
  // quarter to the entries; pattern starts are even (pair loads)
  int64_t sum_w = 0, sum_u = 0;
  bool fit = A->sell_patterns && ns > 0;
  for (int64_t s = 0; s < ns; ++s) {
    sum_w += w[s];
    sum_u += u[s];
    fit = fit && u[s] <= 32;
  }
  fit = fit && 4 * sum_u <= 5 * sum_w;
  std::vector<int32_t> pat(std::max<int64_t>(ns, 1), 0);
  int64_t total = 0, pool_n = 0;
  for (int64_t s = 0; s < ns; ++s) {
    if (fit) {
      pat[s] = (int32_t)pool_n;
      pool_n += (u[s] + 1) & ~1;
      w[s] = u[s];
    }
    total += 32 * (int64_t)w[s];
  }
  const int64_t npat = fit ? ns : 0;
  A->sell_nnz_rows = 32 * sum_w;
  A->nslices = ns;
  A->sell_nnz = total;
  if (total > 2147483647LL) return GBS_OK;  // too large for 32-bit offsets: no copy
  std::vector<int32_t> sptr(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) sptr[s + 1] = sptr[s] + 32 * w[s];
  GBS_TRY(dev_alloc(&A->sell_ptr, ns + 1, st));
  GBS_TRY_CUDA(cudaMemcpyAsync(A->sell_ptr, sptr.data(), sizeof(int32_t) * (ns + 1),
                               cudaMemcpyHostToDevice, st));
  if (npat > 0) {
    GBS_TRY(dev_alloc(&A->sell_pat, ns, st));
    GBS_TRY(dev_alloc(&A->sell_pool, std::max<int64_t>(pool_n, 2), st));
    GBS_TRY(dev_alloc(&A->sell_mask, 32 * ns, st));
    GBS_TRY_CUDA(cudaMemcpyAsync(A->sell_pat, pat.data(), sizeof(int32_t) * ns,
                                 cudaMemcpyHostToDevice, st));
  }
  A->sell_npat = npat;
  A->sell_slice0_h.assign(A->nsys + 1, 0);
  for (int32_t q = 0; q < A->nsys; ++q)
    A->sell_slice0_h[q + 1] =
        A->sell_slice0_h[q] + (int32_t)((A->row_off_h[q + 1] - A->row_off_h[q] + 31) / 32);
  return GBS_OK;
}

// Column patterns or column indices and, if the values are set, FP64 values
// of the sliced copy.  Column indices are stored as 16-bit offsets col - row
// when every column lies within 2^15 - 1 of its row (the symbolic stage
// measured the span), else as 32-bit columns.
int sell_build(gbs_mat A, cudaStream_t s) {
  GBS_TRY(sell_shape(A, s));
  if (!A->sell_ptr) {
    set_error("the sliced-ELL copy would hold %lld entries (limit 2^31 - 1)",
              (long long)A->sell_nnz);
    return GBS_ERR_ARG;
  }
  if (!A->sell_val) {
    const size_t m = (size_t)std::max<int64_t>(A->sell_nnz, 1);
    GBS_TRY(dev_alloc(&A->sell_val, m, s));
    if (A->sell_npat == 0) {
      if (A->col_span <= 32767) GBS_TRY(dev_alloc(&A->sell_off16, m, s));
      else GBS_TRY(dev_alloc(&A->sell_col, m, s));
    }
    if (A->nslices > 0) {
      k_sell_fill<double, true><<<grid_of(A->nslices * 32, 256), 256, 0, s>>>(
          A->nslices, A->sell_ptr, A->sell_row0, A->row_ptr, A->col, (const double *)nullptr,
          A->sell_npat ? A->sell_pat : nullptr, A->sell_pool, A->sell_mask, A->sell_col,
          A->sell_off16, (double *)nullptr);
      GBS_LAUNCHED(1);
    }
    if (A->values_set) GBS_TRY(sell_values(A, s));
  }
  return GBS_OK;
}

// FP64 values of the sliced copy from the CSR values (after every numeric
// stage); the FP32 copy is refreshed by sell_values32 when a refined solve
// needs it.
int sell_values(gbs_mat A, cudaStream_t s) {
  if (!A->sell_val || A->nslices == 0) return GBS_OK;
  k_sell_fill<double, false><<<grid_of(A->nslices * 32, 256), 256, 0, s>>>(
      A->nslices, A->sell_ptr, A->sell_row0, A->row_ptr, A->col, A->val,
      A->sell_npat ? A->sell_pat : nullptr, A->sell_pool, A->sell_mask, (int32_t *)nullptr,
      (int16_t *)nullptr, A->sell_val);
  GBS_LAUNCHED(1);
  return GBS_OK;
}

int sell_values32(gbs_mat A, cudaStream_t s) {
  if (!A->sell_val) return GBS_OK;
  if (!A->sell_val32) GBS_TRY(dev_alloc(&A->sell_val32, std::max<int64_t>(A->sell_nnz, 1), s));
  if (A->sell_nnz > 0) {
    k_sell_to_fp32<<<grid_of(A->sell_nnz, 256), 256, 0, s>>>(A->sell_nnz, A->sell_val,
                                                             A->sell_val32);
    GBS_LAUNCHED(1);
  }
  return GBS_OK;
}

SellView sell_view(gbs_mat A) {
  SellView v;
  v.ptr = A->sell_ptr;
  v.row0 = A->sell_row0;
  v.col = A->sell_off16 ? nullptr : A->sell_col;
  v.off = A->sell_off16;
  v.pat = A->sell_npat ? A->sell_pat : nullptr;
  v.pool = A->sell_pool;
  v.mask = A->sell_mask;
  return v;
}

// Rebuilds a sliced copy that exists (and its transpose's) with or without
// column patterns; the cached graphs hold the old arrays and are dropped.
int set_slice_patterns(gbs_mat A, bool on, cudaStream_t s) {
  if (A->At && A->At->sell_patterns != on) {
    GBS_TRY(set_slice_patterns(A->At, on, s));
    drop_graphs(A);  // A's BiCG graphs hold the transpose's arrays
  }
  if (A->sell_patterns == on) return GBS_OK;
  A->sell_patterns = on;
  if (!A->sell_row0) return GBS_OK;
  const bool built = A->sell_val != nullptr, fp32 = A->sell_val32 != nullptr;
  GBS_TRY_CUDA(cudaStreamSynchronize(s));  // the old copy may be in use
  drop_graphs(A);
  free_sell(A);
  GBS_TRY(sell_shape(A, s));
  if (built) GBS_TRY(sell_build(A, s));
  if (fp32) GBS_TRY(sell_values32(A, s));
  return GBS_OK;
}

}  // namespace gbs
