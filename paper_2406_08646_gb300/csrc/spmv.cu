// MatMult (Sec. 6.1): y = A x on the assembled CSR, FP64, and the launch plan
// (work blocks of rows) shared with the persistent solves.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

constexpr int CAP_MAX = 8192;  // staged products per chunk (64 KB of FP64)

// One CTA per work block: staged CSR product, one row per thread.
__global__ void __launch_bounds__(512) k_spmv(const int32_t *__restrict__ row_ptr,
                                               const int32_t *__restrict__ col,
                                               const double *__restrict__ val,
                                               const double *__restrict__ x,
                                               double *__restrict__ y,
                                               const int32_t *__restrict__ blk_row0, int cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *prod = reinterpret_cast<double *>(smem_raw);
  const int b = blockIdx.x;
  const int32_t r0 = __ldg(blk_row0 + b), r1 = __ldg(blk_row0 + b + 1);
  const double s = staged_row_product<double>(row_ptr, col, val, x, r0, r1, prod, cap);
  const int32_t r = r0 + threadIdx.x;
  if (r < r1) y[r] = s;
}

int launch_spmv(gbs_mat A, const double *x, double *y, cudaStream_t s) {
  if (A->nblocks == 0) return GBS_OK;
  static int configured = 0;
  const size_t smem = (size_t)A->cap * sizeof(double);
  if ((int)smem > configured) {
    GBS_TRY_CUDA(cudaFuncSetAttribute(k_spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = (int)smem;
  }
  k_spmv<<<(unsigned)A->nblocks, A->tpb, smem, s>>>(A->row_ptr, A->col, A->val, x, y,
                                                   A->blk_row0, A->cap);
  GBS_LAUNCHED(1);
  return GBS_OK;
}

// Work blocks: each system's rows cut into ceil(n_s / R) blocks of R rows (the
// last one ragged); blocks never straddle systems.  cap = R * max row length,
// clamped to [256, CAP_MAX]; longer blocks are processed in chunks of cap.
int build_plan(gbs_mat A, int32_t R, int32_t tpb) {
  if (R < 32 || R > 1024 || (R & (R - 1)) != 0 || tpb < 64 || tpb > 512 || (tpb % 32) != 0 ||
      tpb < R) {
    set_error("plan: rows_per_block %d must be a power of two in [32,1024] and "
              "threads_per_block %d a multiple of 32 in [64,512], >= rows_per_block",
              R, tpb);
    return GBS_ERR_ARG;
  }
  std::vector<int32_t> row0, sys, sb0(A->nsys + 1, 0);
  for (int32_t q = 0; q < A->nsys; ++q) {
    const int64_t a = A->row_off_h[q], e = A->row_off_h[q + 1];
    for (int64_t r = a; r < e; r += R) {
      row0.push_back((int32_t)r);
      sys.push_back(q);
    }
    sb0[q + 1] = (int32_t)row0.size();
  }
  row0.push_back((int32_t)A->nrows);
  const int32_t nb = (int32_t)sys.size();
  if (A->blk_row0) cudaFree(A->blk_row0);
  if (A->blk_sys) cudaFree(A->blk_sys);
  if (A->sys_blk0) cudaFree(A->sys_blk0);
  A->blk_row0 = A->blk_sys = A->sys_blk0 = nullptr;
  GBS_TRY_CUDA(cudaMalloc(&A->blk_row0, sizeof(int32_t) * (nb + 1)));
  GBS_TRY_CUDA(cudaMalloc(&A->blk_sys, sizeof(int32_t) * std::max(nb, 1)));
  GBS_TRY_CUDA(cudaMalloc(&A->sys_blk0, sizeof(int32_t) * (A->nsys + 1)));
  GBS_TRY_CUDA(cudaMemcpy(A->blk_row0, row0.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice));
  if (nb > 0)
    GBS_TRY_CUDA(cudaMemcpy(A->blk_sys, sys.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
  GBS_TRY_CUDA(cudaMemcpy(A->sys_blk0, sb0.data(), sizeof(int32_t) * (A->nsys + 1), cudaMemcpyHostToDevice));
  A->sys_blk0_h = sb0;
  A->nblocks = nb;
  A->rows_per_block = R;
  A->tpb = tpb;
  const int64_t want = (int64_t)R * std::max<int32_t>(A->max_row_nnz, 1);
  A->cap = (int32_t)std::min<int64_t>(std::max<int64_t>(want, 256), CAP_MAX);
  A->slot_grid = -1;
  A->grid_fp64 = A->grid_fp32 = 0;
  if (A->graph) {
    cudaGraphExecDestroy(A->graph);
    A->graph = nullptr;
  }
  return GBS_OK;
}

}  // namespace gbs
