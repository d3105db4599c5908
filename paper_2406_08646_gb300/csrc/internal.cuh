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

// ---------------------------------------------------------------- device memory
// Every device buffer of the library (except the allocation-free solve's
// static array) comes from one stream-ordered memory pool per device that
// keeps up to POOL_KEEP_BYTES of freed memory for reuse, so that creating
// and destroying handles of the same sizes does not map and unmap device
// pages each time.  dev_alloc orders the allocation on stream s (GBS_ERR_ALLOC
// on failure, *p = nullptr); dev_free returns the block on stream s (nullptr:
// the legacy default stream).  A buffer used on other streams than s must be
// ordered after s's allocation (the calls that allocate handle buffers
// synchronise s before returning).
constexpr uint64_t POOL_KEEP_BYTES = 32ull << 30;

// The per-CTA solver's automatic size rule: systems of at most this many
// FP64 operations per iteration (nonzeros plus eight per row; pcg.cu).
constexpr int64_t CTA_AUTO_WORK = 40000;
int dev_alloc_bytes(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
template <typename T>
int dev_alloc(T **p, size_t n, cudaStream_t s) {
  return dev_alloc_bytes(reinterpret_cast<void **>(p), n * sizeof(T), s);
}

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
// reduction ("last arriver") and read by the kernels of the following phases.
struct SysState {
  double bb;        // ||b_s||^2
  double rho;       // r.z
  double rr;        // ||r||^2 (inner precision in refined mode)
  double alpha, beta;
  double rnorm0, rnorm;
  double scale;     // refined: s = ||r64||
  double prev_rn;   // refined: previous outer residual norm
  double r0in;      // refined: inner stopping threshold (target x initial norm)
  double tt;        // ||b - A x||^2 at exit
  double thr;       // rtol ||b_s||, the convergence threshold (set by the setup)
  double tau, theta, eta;  // TFQMR: quasi-residual recurrence (eta of the last half step)
  double coef;             // TFQMR: theta^2 eta / alpha for the next d update
  double gam;              // single-reduction CG: r.u of the start residual
  double thr2lo, thr2hi;   // bounds of thr^2 (set_thr): ||r|| <= thr decided from ||r||^2
  int32_t status;
  int32_t active;   // 1 while the system still iterates
  int32_t iterations;
  int32_t outer;
  int32_t inner_it;
  int32_t mode;     // refined: M_INNER / M_XUPD / M_START (phases.cuh)
  int32_t stall;
  int32_t first;    // refined: next p update is p = z
  int32_t zero_x;   // b == 0: x must be set to 0
  int32_t m;        // TFQMR: half steps taken
  int32_t pend;     // TFQMR: x += eta D^-1 d of the last half step not yet applied
  int32_t rn_stale; // rnorm not yet taken from rr (the closing kernel takes it)
};

// Work vectors of the solvers in krylov.cu (TFQMR: w, y1, y2, rt, v, B y1,
// B y2, d, t; BiCG uses the first six as r, rt, p, pt, q, qt; pipelined CG
// all nine as r, u, w, p, s, q, z and the two buffers of m).
constexpr int KRYLOV_NVEC = 9;

// Cached solve graphs of a handle, by loop kind.
enum { GBS_GRAPH_CG = 0, GBS_GRAPH_CG32 = 1, GBS_GRAPH_BICG = 2, GBS_GRAPH_TFQMR = 3,
       GBS_GRAPH_PIPECG = 4, GBS_GRAPH_CGSR = 5, GBS_GRAPH_CGSR1 = 6, GBS_GRAPH_KINDS = 7 };

// Per-solve control words (device).  Zeroed before every solve.
struct DevCtl {
  int32_t n_active;        // systems still iterating
  int32_t err;             // GBS_ERR_TIMEOUT, 0 = none
  int32_t stop[2];         // host-stepped loop: trip t is skipped iff stop[t & 1]
  int64_t trips;           // loop trips completed
  int64_t t_start;         // globaltimer at the start of the solve
  int64_t stamp;           // globaltimer when the last phase kernel started
  int32_t last_phase;      // index of that phase, -1 before the first
  int32_t queue;           // per-CTA solver: systems taken beyond the grid's first ones
  int64_t phase_ns[5];     // setup, A, B, C, final: start-to-next-start time
};

// Per-call solve arguments, copied to the device before each solve so that a
// cached graph serves every call with the same shape.
struct CallArgs {
  const double *b;
  double *x;
  double rtol, inner_rtol;
  int32_t maxit, inner_maxit, max_outer, nonzero_guess;
  int64_t max_trips;   // cap on loop trips (a safety net; see solve())
  int64_t timeout_ns;  // wall-clock limit of the loop, 0 = none
};

// Device block table plus its host mirror (BlockTable in phases.cuh).
struct TableDev {
  int32_t nblocks = 0;
  int32_t *row0 = nullptr;       // nblocks + 1
  int32_t *sys = nullptr;        // nblocks
  int32_t *sys_blk0 = nullptr;   // nsys + 1
  int32_t *sys_slot0 = nullptr;  // nsys + 1 (for the table's grid)
  int32_t *slice0 = nullptr;     // nblocks + 1: first 32-row slice of each block
  int32_t *row1 = nullptr, *slice1 = nullptr;  // block ends (tables with gaps only)
  std::vector<int32_t> sys_blk0_h;
  int32_t grid = 0;              // CTAs of the kernels that walk this table
  int64_t nslots = 0;            // reduction slots: sum over systems of min(blocks, grid)
};

// The sliced-ELL copy as the row products read it (sell.cu, sell_rows).
// With column patterns (pat set) every slice takes its columns from its
// pattern: pool[pat[s] + k] is the pattern's k-th offset col - row
// (ascending) and bit k of mask[32 s + i] says whether row i of the slice
// holds it.  Without, the columns come from col (32-bit columns) or off
// (16-bit offsets), exactly one of which is set.
struct SellView {
  const int32_t *ptr, *row0;  // nslices + 1 entry offsets and first rows
  const int32_t *col;
  const int16_t *off;
  const int32_t *pat;
  const int32_t *pool;
  const uint32_t *mask;
};

}  // namespace gbs

// ---------------------------------------------------------------- the handle
struct gbs_mat_s {
  int device = 0;
  int64_t nrows = 0, ncols = 0, ncoo = 0, nkept = 0, nnz = 0;
  int32_t nsys = 1;
  int32_t max_row_nnz = 0;
  int32_t col_span = 0;         // largest |col - row| of the pattern (capped at 2^30)
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

  // sliced-ELL copy used by the row products (sell.cu), built on demand
  int64_t nslices = 0, sell_nnz = 0;
  int32_t *sell_ptr = nullptr;     // nslices + 1 entry offsets (< 2^31)
  int32_t *sell_row0 = nullptr;    // nslices + 1 first rows
  int32_t *sell_col = nullptr;     // sell_nnz, -1 = padding
  int16_t *sell_off16 = nullptr;   // sell_nnz column offsets col - row when they all fit
                                   // in 16 bits (padding -32768); the kernels read these then
  double *sell_val = nullptr;      // sell_nnz
  float *sell_val32 = nullptr;     // sell_nnz (refined solves)
  int32_t *sell_pat = nullptr;     // nslices: first offset of each slice's pattern in sell_pool
  int32_t *sell_pool = nullptr;    // the patterns' offsets col - row
  uint32_t *sell_mask = nullptr;   // 32 nslices: pattern entries each row holds
  int64_t sell_npat = 0;           // slices with a pattern (0 or nslices)
  int64_t sell_nnz_rows = 0;       // 32 x the slices' longest rows (the size without
                                   // patterns: the automatic plan's padding rule)
  bool sell_patterns = true;       // build column patterns when they fit
  std::vector<int32_t> sell_slice0_h;  // nsys + 1 first slice of each system

  // launch plan: two block tables (SpMV phases, vector-update phases), the
  // row-product kernel (0: sliced ELL; 1, 2, 4, 8, 32: CSR-vector with that
  // many lanes per row), CTAs per SM cap of the grids
  gbs::TableDev ta, te;
  int32_t Ra = 256, Re = 512;   // rows per SpMV block / per update block
  int32_t lanes = 0;
  int32_t ctas_per_sm = 0;      // grid cap per SM, 0 = as many as fit (one wave)
  int32_t solver = 0;           // GBS_SOLVER_AUTO / PHASES / CTA / SPLIT
  int64_t split_rows = 1;       // GBS_SOLVER_SPLIT: systems of at least this many rows on
                                // the phase kernels, the rest on the per-CTA solver
  bool solver_batched_only = false;  // the autotuner chose `solver` for batched solves
  gbs::TableDev sa, se;         // the size split's block tables (its large systems only)
  int64_t split_built = 0;      // split_rows the tables were built for (0: none)
  int32_t cg_form = 0;          // GBS_CG_TEXTBOOK / _SINGLE_REDUCTION / _SINGLE_KERNEL
  // one-kernel single-reduction CG: table A's CTA c waits, before its row
  // products, for CTAs c - halo_lo .. c - halo_lo + halo_n - 1 (mod grid) to
  // have updated their rows of u (set by build_plan from col_span)
  int32_t halo_lo = 0, halo_n = 0;
  int32_t *cta_order = nullptr; // nsys: systems by decreasing rows (per-CTA solver)
  int64_t max_sys_rows = 0, max_sys_nnz = 0;

  // solver workspace (device, allocated on first solve)
  double *r = nullptr, *p = nullptr, *q = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  double *part = nullptr;       // reduction slots (table A region, then table E)
  int64_t part_cap = 0;
  unsigned *sys_cnt = nullptr;  // nsys arrival counters
  int32_t *halo_flags = nullptr;  // table A grid: last iteration each CTA published
  int32_t halo_cap = 0;
  gbs::SysState *st = nullptr;  // nsys
  gbs::DevCtl *ctl = nullptr;
  gbs::CallArgs *call = nullptr;
  gbs::SysState *st_host = nullptr;  // pinned copy for results
  int32_t last_count = 0;            // systems in the last solve's result
  bool last_ensemble = false;
  bool trips_counted = true;         // launch counter already holds the last loop
  int32_t last_solver = 0;           // solver the last solve ran

  // cached executable graphs [loop kind][per_system] of the solve loop
  cudaGraphExec_t graph[gbs::GBS_GRAPH_KINDS][2] = {};
  int32_t loop_body = 3;             // kernels per trip of the last phase-kernel loop

  // nonsymmetric solvers (krylov.cu): the transpose as an internal handle
  // (its CSR and sliced copy), refreshed when the values change; the work
  // vectors; per-system first rows and first slices (device, nsys + 1)
  int64_t values_version = 0;       // bumped by every numeric stage
  gbs_mat_s *At = nullptr;
  int64_t at_version = -1;          // values_version the transpose holds
  double *kv = nullptr;             // gbs::KRYLOV_NVEC vectors of nrows
  int32_t *sys_row0 = nullptr, *sys_slice0 = nullptr;  // one allocation (sys_row0)
};

namespace gbs {

int ensure_solver_workspace(gbs_mat A, bool refined, cudaStream_t s);
// The solver setting that applies to a solve: the handle's, except that a
// choice the autotuner made for a batched handle's batched solves leaves its
// ensemble solves (the stacked system) to the automatic choice.
inline int32_t solver_for(gbs_mat A, bool per_system) {
  return (A->solver_batched_only && !per_system) ? GBS_SOLVER_AUTO : A->solver;
}
int build_plan(gbs_mat A, int32_t spmv_rows, int32_t update_rows, int32_t lanes,
               int32_t ctas_per_sm, cudaStream_t s);
int build_split_tables(gbs_mat A, cudaStream_t s);
void free_table(TableDev &t);
void drop_graphs(gbs_mat A);
int launch_spmv(gbs_mat A, const double *x, double *y, cudaStream_t s);
int launch_set_values(gbs_mat A, const double *v, int mode, cudaStream_t s);
int launch_vec_set_values(gbs_mat A, const double *v, int mode, double *y, cudaStream_t s);
int launch_to_fp32(gbs_mat A, cudaStream_t s);
int launch_adjoint_scatter(gbs_mat A, const double *lambda, const double *x,
                           double *dLda, double *dLdv, cudaStream_t s);
int symbolic(gbs_mat A, const int32_t *i, const int32_t *j, const int64_t *coo_off_h,
             cudaStream_t s);
int solve(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
          cudaStream_t s);
void free_handle(gbs_mat A);
int solve_krylov(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
                 cudaStream_t s);
CallArgs call_args(const double *b, double *x, const ksp_opts &o);
int put_call(CallArgs *dst, const CallArgs &c, cudaStream_t s, DevCtl *ctl = nullptr);
int read_results(gbs_mat A, ksp_result *res, int32_t count, cudaStream_t s);
int read_phase_ns(gbs_mat A, int64_t *phase_ns, cudaStream_t s);
int auto_lanes(int64_t nnz, int64_t nrows);
int phase_occupancy(int lanes, int *rows, int *upd);
int32_t stream_matrix(gbs_mat A, int bytes_per_entry);
void free_sell(gbs_mat A);
int sell_shape(gbs_mat A, cudaStream_t s);
int sell_build(gbs_mat A, cudaStream_t s);
int sell_values(gbs_mat A, cudaStream_t s);
int sell_values32(gbs_mat A, cudaStream_t s);
SellView sell_view(gbs_mat A);
int set_slice_patterns(gbs_mat A, bool on, cudaStream_t s);

}  // namespace gbs
