// Internal declarations shared by the translation units of libgbs.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <vector>

#include "gbs.h"

namespace gbs {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void count_launches(int64_t n);

#define GBS_TRY_CUDA(call)                                                       \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ::gbs::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                \
                       cudaGetErrorString(e_));                                  \
      return GBS_ERR_CUDA;                                                       \
    }                                                                            \
  } while (0)

#define GBS_TRY(call)                                                            \
  do {                                                                           \
    int s_ = (call);                                                             \
    if (s_ != GBS_OK) return s_;                                                 \
  } while (0)

// After a <<<>>> launch.
#define GBS_LAUNCHED(n)                                                          \
  do {                                                                           \
    ::gbs::count_launches(n);                                                    \
    GBS_TRY_CUDA(cudaGetLastError());                                            \
  } while (0)

// ---------------------------------------------------------------- device state

// Per-system solver state, written only by the CTA that completes a system's
// reduction ("last arriver") and read by every CTA after the next grid barrier.
struct SysState {
  double bb;        // ||b_s||^2
  double rho;       // r.z
  double rr;        // ||r||^2 (inner precision in refined mode)
  double alpha, beta;
  double rnorm0, rnorm;
  double scale;     // refined: s = ||r64||
  double prev_rn;   // refined: previous outer residual norm
  double r0in;      // refined: initial inner residual norm
  double tt;        // ||b - A x||^2 at exit
  int32_t status;
  int32_t active;   // 1 while the system still iterates
  int32_t iterations;
  int32_t outer;
  int32_t inner_it;
  int32_t mode;     // refined: see pcg.cu
  int32_t stall;
  int32_t first;    // refined: next p update is p = z
  int32_t zero_x;   // b == 0: x must be set to 0
  int32_t pad;
};

// Device-side error word plus counters used by the persistent kernels.
struct DevCtl {
  unsigned long long bar;  // grid-barrier arrival counter (monotonic)
  int32_t err;             // GBS_ERR_TIMEOUT etc., 0 = none
  int32_t n_active;        // systems still iterating
  int64_t phase_ns[5];     // CTA 0's time per phase: setup, A, B, C, final residual
};

// Device block table plus its host mirror (see BlockTable in pipe.cuh).
struct TableDev {
  int32_t nblocks = 0;
  int32_t *row0 = nullptr;       // nblocks + 1
  int32_t *nz0 = nullptr;        // nblocks + 1
  int32_t *sys = nullptr;        // nblocks
  int32_t *sys_blk0 = nullptr;   // nsys + 1
  int32_t *sys_slot0 = nullptr;  // nsys + 1 (for slot_workers workers)
  std::vector<int32_t> sys_blk0_h;
};

}  // namespace gbs

// ---------------------------------------------------------------- the handle
struct gbs_mat_s {
  int device = 0;
  int64_t nrows = 0, ncols = 0, ncoo = 0, nkept = 0, nnz = 0;
  int32_t nsys = 1;
  int32_t max_row_nnz = 0;
  bool batched = false;
  bool values_set = false;
  bool val32_valid = false;

  // CSR and COO maps (device)
  int32_t *row_ptr = nullptr, *col = nullptr;
  double *val = nullptr;
  float *val32 = nullptr;
  int32_t *perm = nullptr, *jmap = nullptr;
  int32_t *diag_pos = nullptr;
  double *dinv = nullptr;
  float *dinv32 = nullptr;

  // systems (host + device)
  std::vector<int64_t> row_off_h;  // nsys + 1
  std::vector<int32_t> max_row_sys_h;

  // launch plan: two block tables (SpMV phases, vector-update phases), warps
  // per CTA, pipeline stages and the per-warp stage size
  gbs::TableDev ta, te;
  int32_t Ra = 32, Re = 256;  // rows per SpMV block / per update block
  int32_t nwarps = 8, nstages = 2;
  int32_t tpb = 256;          // 32 * nwarps
  int32_t cap = 1024;         // staged nonzeros per SpMV block
  int64_t stage_bytes = 0;
  int32_t grid_fp64 = 0, grid_fp32 = 0, grid_spmv = 0;  // persistent grid sizes (per plan)
  int32_t *err_word = nullptr;  // device error word of the SpMV pipeline

  // solver workspace (device, allocated on first solve)
  double *r = nullptr, *p = nullptr, *q = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  double *part = nullptr;       // reduction slots (table A region, then table E)
  int64_t part_cap = 0;
  int32_t slot_workers = -1;    // worker count the slot offsets were built for
  unsigned *sys_cnt = nullptr;  // nsys arrival counters
  gbs::SysState *st = nullptr;  // nsys
  gbs::DevCtl *ctl = nullptr;
  gbs::SysState *st_host = nullptr;  // pinned copy for results
  int32_t last_count = 0;            // systems in the last solve's result
  bool last_ensemble = false;

  // cached CUDA graph of the batched launch
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_key[8] = {0};
};

namespace gbs {

int ensure_solver_workspace(gbs_mat A, bool refined);
int build_plan(gbs_mat A, int32_t spmv_rows, int32_t update_rows, int32_t nwarps,
               int32_t nstages);
void free_table(TableDev &t);
int launch_spmv(gbs_mat A, const double *x, double *y, cudaStream_t s);
int launch_set_values(gbs_mat A, const double *v, int mode, cudaStream_t s);
int launch_to_fp32(gbs_mat A, cudaStream_t s);
int launch_adjoint_scatter(gbs_mat A, const double *lambda, const double *x,
                           double *dLda, double *dLdv, cudaStream_t s);
int symbolic(gbs_mat A, const int32_t *i, const int32_t *j, const int64_t *coo_off_h,
             cudaStream_t s);
int solve(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
          bool use_graph, cudaStream_t s);
int read_results(gbs_mat A, ksp_result *res, int32_t count, cudaStream_t s);

}  // namespace gbs
