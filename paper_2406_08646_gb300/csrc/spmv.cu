// MatMult (Sec. 6.1): y = A x on the assembled CSR, FP64, and the launch plan
// (block tables, warps, pipeline stages) shared with the persistent solves.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"
#include "pipe.cuh"

namespace gbs {

constexpr int SMEM_BUDGET = 232448 - 1024;  // dynamic shared memory per CTA we plan for

// Persistent SpMV: every warp streams its SpMV blocks through its own
// bulk-copy pipeline (CSR values, columns and row pointers staged in shared
// memory) and sums each row lane by lane with one FMA per nonzero.
__global__ void __launch_bounds__(512) k_spmv(const int32_t *__restrict__ row_ptr,
                                              const int32_t *__restrict__ col,
                                              const double *__restrict__ val,
                                              const double *__restrict__ x,
                                              double *__restrict__ y, BlockTable t, int cap,
                                              int Ra, int Re, int ns, int64_t stage_bytes,
                                              int32_t *err, int64_t timeout_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)nw * ns * stage_bytes);
  WarpPipe P{smem_raw + (size_t)warp * ns * stage_bytes, bars + warp * ns, ns, cap, Ra, Re,
             stage_bytes, 0u, err, timeout_ns, policy_evict_first(), policy_evict_last()};
  if (lane == 0) P.init_barriers();
  __syncwarp();
  auto want = [](int) -> bool { return true; };
  auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
    if (arrive_for(bar, csr_bytes<double>(d, P.cap)))
      csr_copy<double>(P, st, d, row_ptr, col, val, bar);
  };
  auto work = [&](int b, const BlkDesc &d, unsigned char *st) {
    auto f = [&](int r, double s) { y[r] = s; };
    block_rows<double>(P, st, d, row_ptr, col, val, x, f);
  };
  warp_stream(P, t, blockIdx.x * nw + warp, gridDim.x * nw, want, issue, work);
}

static size_t spmv_smem(gbs_mat A) {
  return (size_t)A->nwarps * A->nstages * (size_t)A->stage_bytes +
         (size_t)A->nwarps * A->nstages * 8;
}

static BlockTable table_view(const TableDev &t) {
  return BlockTable{t.nblocks, t.row0, t.nz0, t.sys, t.sys_blk0, t.sys_slot0};
}

int launch_spmv(gbs_mat A, const double *x, double *y, cudaStream_t s) {
  if (A->ta.nblocks == 0) return GBS_OK;
  const size_t smem = spmv_smem(A);
  cudaFuncAttributes fa;
  GBS_TRY_CUDA(cudaFuncGetAttributes(&fa, k_spmv));
  if (fa.maxDynamicSharedSizeBytes < (int)smem)
    GBS_TRY_CUDA(cudaFuncSetAttribute(k_spmv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (A->grid_spmv <= 0) {
    int per_sm = 0, nsm = 0;
    GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv, A->tpb, smem));
    GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device));
    if (per_sm < 1) {
      set_error("SpMV kernel does not fit on an SM (tpb %d, smem %zu)", A->tpb, smem);
      return GBS_ERR_LAUNCH;
    }
    const int64_t warps_needed = A->ta.nblocks;
    A->grid_spmv = (int32_t)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)per_sm * nsm, (warps_needed + A->nwarps - 1) / A->nwarps));
  }
  k_spmv<<<(unsigned)A->grid_spmv, A->tpb, smem, s>>>(
      A->row_ptr, A->col, A->val, x, y, table_view(A->ta), A->cap, A->Ra, A->Re, A->nstages,
      A->stage_bytes, A->err_word, 2000000000LL);
  GBS_LAUNCHED(1);
  return GBS_OK;
}

void free_table(TableDev &t) {
  for (int32_t *p : {t.row0, t.nz0, t.sys, t.sys_blk0, t.sys_slot0})
    if (p) cudaFree(p);
  t.row0 = t.nz0 = t.sys = t.sys_blk0 = t.sys_slot0 = nullptr;
  t.nblocks = 0;
  t.sys_blk0_h.clear();
}

// Each system's rows cut into ceil(n_s / R) blocks of R rows (the last one
// ragged); blocks never straddle systems.
static int build_table(gbs_mat A, const std::vector<int32_t> &rp, int32_t R, TableDev &t) {
  std::vector<int32_t> row0, sys, sb0(A->nsys + 1, 0), nz0;
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
  nz0.resize(nb + 1);
  for (int32_t b = 0; b <= nb; ++b) nz0[b] = rp[row0[b]];
  free_table(t);
  GBS_TRY_CUDA(cudaMalloc(&t.row0, sizeof(int32_t) * (nb + 1)));
  GBS_TRY_CUDA(cudaMalloc(&t.nz0, sizeof(int32_t) * (nb + 1)));
  GBS_TRY_CUDA(cudaMalloc(&t.sys, sizeof(int32_t) * std::max(nb, 1)));
  GBS_TRY_CUDA(cudaMalloc(&t.sys_blk0, sizeof(int32_t) * (A->nsys + 1)));
  GBS_TRY_CUDA(cudaMalloc(&t.sys_slot0, sizeof(int32_t) * (A->nsys + 1)));
  GBS_TRY_CUDA(cudaMemcpy(t.row0, row0.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice));
  GBS_TRY_CUDA(cudaMemcpy(t.nz0, nz0.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice));
  if (nb > 0)
    GBS_TRY_CUDA(cudaMemcpy(t.sys, sys.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
  GBS_TRY_CUDA(cudaMemcpy(t.sys_blk0, sb0.data(), sizeof(int32_t) * (A->nsys + 1),
                          cudaMemcpyHostToDevice));
  t.sys_blk0_h = sb0;
  t.nblocks = nb;
  return GBS_OK;
}

// Plan: SpMV blocks of Ra rows (a multiple of 32: lanes own rows), update
// blocks of Re rows, nwarps independent warps per CTA, ns pipeline stages per
// warp.  A warp stage holds a whole SpMV block (Ra rows of the longest row,
// plus 16-byte rounding slack) or an update block (5 vector slices); when the
// stages would not fit in shared memory the SpMV capacity shrinks and longer
// blocks are read with plain loads instead.
int build_plan(gbs_mat A, int32_t Ra, int32_t Re, int32_t nw, int32_t ns) {
  if (Ra < 32 || Ra > 512 || (Ra % 32) != 0 || Re < 32 || Re > 4096 || (Re % 32) != 0 ||
      nw < 1 || nw > 16 || ns < 2 || ns > PIPE_MAX_STAGES) {
    set_error("plan: spmv_rows %d and update_rows %d must be multiples of 32 (<= 512, <= 4096), "
              "warps %d in [1,16], stages %d in [2,%d]",
              Ra, Re, nw, ns, PIPE_MAX_STAGES);
    return GBS_ERR_ARG;
  }
  std::vector<int32_t> rp(A->nrows + 1);
  GBS_TRY_CUDA(cudaMemcpy(rp.data(), A->row_ptr, sizeof(int32_t) * (A->nrows + 1),
                          cudaMemcpyDeviceToHost));
  const int64_t upd = (upd_stage_bytes(Re) + 15) & ~15LL;
  const int64_t per_stage_budget = (SMEM_BUDGET - 64) / ((int64_t)nw * ns) - 8;
  if (upd > per_stage_budget) {
    set_error("plan: %d warps x %d stages of %d-row update blocks exceed shared memory", nw, ns,
              Re);
    return GBS_ERR_ARG;
  }
  int64_t cap = ((int64_t)Ra * std::max<int32_t>(A->max_row_nnz, 1) + 4 + 3) & ~3LL;
  while (cap > 64 && ((spmv_stage_bytes((int)cap, Ra) + 15) & ~15LL) > per_stage_budget)
    cap = (cap / 2) & ~3LL;
  const int64_t spm = (spmv_stage_bytes((int)cap, Ra) + 15) & ~15LL;
  if (spm > per_stage_budget) {
    set_error("plan: %d warps x %d stages of %d-row SpMV blocks exceed shared memory", nw, ns, Ra);
    return GBS_ERR_ARG;
  }
  GBS_TRY(build_table(A, rp, Ra, A->ta));
  GBS_TRY(build_table(A, rp, Re, A->te));
  if (!A->err_word) {
    GBS_TRY_CUDA(cudaMalloc(&A->err_word, sizeof(int32_t)));
    GBS_TRY_CUDA(cudaMemset(A->err_word, 0, sizeof(int32_t)));
  }
  A->Ra = Ra;
  A->Re = Re;
  A->nwarps = nw;
  A->tpb = 32 * nw;
  A->nstages = ns;
  A->cap = (int32_t)cap;
  A->stage_bytes = std::max(spm, upd);
  A->slot_workers = -1;
  A->grid_fp64 = A->grid_fp32 = A->grid_spmv = 0;
  if (A->graph) {
    cudaGraphExecDestroy(A->graph);
    A->graph = nullptr;
  }
  return GBS_OK;
}

}  // namespace gbs
