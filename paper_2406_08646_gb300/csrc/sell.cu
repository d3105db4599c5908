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
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

static unsigned grid_of(int64_t n, int tpb) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + tpb - 1) / tpb, 1 << 20));
}

// w_s = longest row of slice s.
__global__ void k_slice_width(int64_t nslices, const int32_t *__restrict__ srow0,
                              const int32_t *__restrict__ row_ptr, int32_t *__restrict__ w) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nslices;
       s += (int64_t)gridDim.x * blockDim.x) {
    int32_t m = 0;
    for (int32_t r = srow0[s]; r < srow0[s + 1]; ++r) m = max(m, row_ptr[r + 1] - row_ptr[r]);
    w[s] = m;
  }
}

// Columns (and, with val != nullptr, values; with soff != nullptr, the 16-bit
// offsets col - row, padding -32768) of the sliced copy: one warp per slice,
// lane i on row i of the slice, padding written as (-1, 0).
template <typename T>
__global__ void k_sell_fill(int64_t nslices, const int32_t *__restrict__ sptr,
                            const int32_t *__restrict__ srow0, const int32_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col, const T *__restrict__ val,
                            int32_t *__restrict__ scol, int16_t *__restrict__ soff,
                            T *__restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nslices; s += nw) {
    const int32_t r = srow0[s] + lane;
    const bool live = r < srow0[s + 1];
    const int32_t rs = live ? row_ptr[r] : 0, len = live ? row_ptr[r + 1] - rs : 0;
    const int64_t b = sptr[s];
    const int32_t w = (int32_t)((sptr[s + 1] - b) >> 5), np = w >> 1;
    for (int32_t k = 0; k < w; ++k) {
      const bool ok = k < len;
      const int64_t q = k < 2 * np ? b + 64 * (k >> 1) + 2 * lane + (k & 1) : b + 64 * np + lane;
      if (scol) scol[q] = ok ? col[rs + k] : -1;
      if (soff) soff[q] = ok ? (int16_t)(col[rs + k] - r) : (int16_t)-32768;
      if (sval) sval[q] = ok ? val[rs + k] : T(0);
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
                  (void *)A->sell_off16, (void *)A->sell_val, (void *)A->sell_val32})
    dev_free(p, nullptr);
  A->sell_ptr = nullptr;
  A->sell_row0 = nullptr;
  A->sell_col = nullptr;
  A->sell_off16 = nullptr;
  A->sell_val = nullptr;
  A->sell_val32 = nullptr;
  A->nslices = A->sell_nnz = 0;
}

// Slice table and padded size (no entries yet); when the padded size reaches
// 2^31 only the size is recorded.  Idempotent.  Synchronises s once (the
// slice widths decide the sizes).
int sell_shape(gbs_mat A, cudaStream_t st) {
  if (A->sell_row0) return GBS_OK;
  std::vector<int32_t> srow0;
  for (int32_t q = 0; q < A->nsys; ++q)
    for (int64_t r = A->row_off_h[q]; r < A->row_off_h[q + 1]; r += 32) srow0.push_back((int32_t)r);
  const int64_t ns = (int64_t)srow0.size();
  srow0.push_back((int32_t)A->nrows);
  std::vector<int32_t> w(std::max<int64_t>(ns, 1), 0);
  GBS_TRY(dev_alloc(&A->sell_row0, ns + 1, st));
  GBS_TRY_CUDA(cudaMemcpyAsync(A->sell_row0, srow0.data(), sizeof(int32_t) * (ns + 1),
                               cudaMemcpyHostToDevice, st));
  if (ns > 0) {
    int32_t *dw = nullptr;
    GBS_TRY(dev_alloc(&dw, ns, st));
    k_slice_width<<<grid_of(ns, 256), 256, 0, st>>>(ns, A->sell_row0, A->row_ptr, dw);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.data(), dw, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(dw, st);
    count_launches(1);
    GBS_TRY_CUDA(e);
  }
  int64_t total = 0;
  for (int64_t s = 0; s < ns; ++s) total += 32 * (int64_t)w[s];
  A->nslices = ns;
  A->sell_nnz = total;
  if (total > 2147483647LL) return GBS_OK;  // too large for 32-bit offsets: no copy
  std::vector<int32_t> sptr(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) sptr[s + 1] = sptr[s] + 32 * w[s];
  GBS_TRY(dev_alloc(&A->sell_ptr, ns + 1, st));
  GBS_TRY_CUDA(cudaMemcpyAsync(A->sell_ptr, sptr.data(), sizeof(int32_t) * (ns + 1),
                               cudaMemcpyHostToDevice, st));
  A->sell_slice0_h.assign(A->nsys + 1, 0);
  for (int32_t q = 0; q < A->nsys; ++q)
    A->sell_slice0_h[q + 1] =
        A->sell_slice0_h[q] + (int32_t)((A->row_off_h[q + 1] - A->row_off_h[q] + 31) / 32);
  return GBS_OK;
}

// Columns and (if the values are set) FP64 values of the sliced copy.  The
// columns are stored as 16-bit offsets col - row when every column lies within
// 2^15 - 1 of its row (the symbolic stage measured the span), else as 32-bit
// columns.
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
    if (A->col_span <= 32767) GBS_TRY(dev_alloc(&A->sell_off16, m, s));
    else GBS_TRY(dev_alloc(&A->sell_col, m, s));
    if (A->nslices > 0) {
      k_sell_fill<double><<<grid_of(A->nslices * 32, 256), 256, 0, s>>>(
          A->nslices, A->sell_ptr, A->sell_row0, A->row_ptr, A->col, (const double *)nullptr,
          A->sell_col, A->sell_off16, (double *)nullptr);
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
  k_sell_fill<double><<<grid_of(A->nslices * 32, 256), 256, 0, s>>>(
      A->nslices, A->sell_ptr, A->sell_row0, A->row_ptr, A->col, A->val, (int32_t *)nullptr,
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

}  // namespace gbs
