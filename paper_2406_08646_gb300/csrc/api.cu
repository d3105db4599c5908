// C-ABI entry points of libgbs.so (declared in include/gbs.h): argument
// checks, handle lifetime, option defaults, the autotuner, and dispatch to the
// kernels in coo.cu, spmv.cu and pcg.cu.
#include <cuda_runtime.h>

#include <fcntl.h>
#include <sys/file.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace gbs {

static thread_local char g_err[1024] = "";
static std::atomic<int64_t> g_launches{0};

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// The library's memory pool of the current device, created on first use.
static constexpr int kMaxPoolDevices = 256;
static cudaMemPool_t g_pools[kMaxPoolDevices] = {};
static std::mutex g_pool_mu;

static int device_pool(cudaMemPool_t *out) {
  int dev = 0;
  GBS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxPoolDevices) {
    set_error("device ordinal %d out of range", dev);
    return GBS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    GBS_TRY_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = POOL_KEEP_BYTES;
    GBS_TRY_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return GBS_OK;
}

int dev_alloc_bytes(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  GBS_TRY(device_pool(&pool));
  const cudaError_t e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GBS_ERR_ALLOC : GBS_ERR_CUDA;
  }
  return GBS_OK;
}

void dev_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

static constexpr int64_t kMaxIndex = 2147483647LL;

void free_handle(gbs_mat A) {
  if (!A) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(A->device);
  cudaDeviceSynchronize();  // the buffers may be in use on any stream
  drop_graphs(A);
  free_handle(A->At);
  void *dev[] = {A->row_ptr, A->col, A->val, A->val32, A->perm, A->jmap, A->diag_pos,
                 A->dinv, A->dinv32, A->r, A->p, A->q, A->r32, A->p32, A->q32, A->d32,
                 A->part, A->sys_cnt, A->st, A->ctl, A->call, A->cta_order,
                 A->kv, A->sys_row0, A->halo_flags};  // sys_slice0 lies inside sys_row0's
  for (void *p : dev) dev_free(p, nullptr);
  free_table(A->ta);
  free_table(A->sa);
  free_table(A->se);
  free_table(A->te);
  free_sell(A);
  if (A->st_host) cudaFreeHost(A->st_host);
  cudaSetDevice(cur);
  delete A;
}

// Default plan: everything automatic -- the row-product kernel chosen from
// the matrix, one wave of CTAs per phase kernel, about one block per CTA.
static int default_plan(gbs_mat A, cudaStream_t s) {
  return build_plan(A, 0, 0, GBS_SPMV_AUTO, 0, s);
}

static int64_t max_system_rows(gbs_mat A, bool per_system) {
  if (!per_system) return A->nrows;
  int64_t m = 0;
  for (int32_t q = 0; q < A->nsys; ++q) m = std::max(m, A->row_off_h[q + 1] - A->row_off_h[q]);
  return m;
}

static int fill_opts(gbs_mat A, const ksp_opts *in, ksp_opts &o, bool per_system) {
  ksp_opts_default(&o);
  if (in) o = *in;
  if (!(o.rtol >= 0.0) || !std::isfinite(o.rtol)) {
    set_error("ksp opts: rtol must be finite and >= 0");
    return GBS_ERR_ARG;
  }
  if (o.precision != GBS_FP64 && o.precision != GBS_FP32_REFINED) {
    set_error("ksp opts: precision must be GBS_FP64 or GBS_FP32_REFINED");
    return GBS_ERR_ARG;
  }
  if (o.host_loop != 0 && o.host_loop != 1) {
    set_error("ksp opts: host_loop must be 0 or 1");
    return GBS_ERR_ARG;
  }
  if (o.method < GBS_KSP_CG || o.method > GBS_KSP_CGSR) {
    set_error("ksp opts: method must be GBS_KSP_CG, GBS_KSP_CGSR, GBS_KSP_BICG, "
              "GBS_KSP_TFQMR or GBS_KSP_PIPECG");
    return GBS_ERR_ARG;
  }
  if (o.method != GBS_KSP_CG && o.precision != GBS_FP64) {
    set_error("ksp opts: BiCG, TFQMR, pipelined and single-reduction CG run in FP64 only "
              "(precision GBS_FP64)");
    return GBS_ERR_ARG;
  }
  const int64_t n = max_system_rows(A, per_system);
  const int32_t dflt = (int32_t)std::min<int64_t>(10 * std::max<int64_t>(n, 1), 100000);
  if (o.maxit < 0) o.maxit = dflt;
  if (o.inner_maxit < 0) o.inner_maxit = dflt;
  if (!(o.inner_rtol > 0.0)) o.inner_rtol = 1e-4;
  if (o.max_outer < 0) o.max_outer = 30;
  if (o.timeout_ns < 0) o.timeout_ns = 0;
  return GBS_OK;
}

static int check_mat(gbs_mat A, const char *fn) {
  if (!A) {
    set_error("%s: null matrix handle", fn);
    return GBS_ERR_ARG;
  }
  return GBS_OK;
}

static int use_device(gbs_mat A) {
  GBS_TRY_CUDA(cudaSetDevice(A->device));
  return GBS_OK;
}

static int create_common(gbs_mat *out, gbs_mat A, const int32_t *i, const int32_t *j,
                         const int64_t *coo_off_h, cudaStream_t s) {
  int st = symbolic(A, i, j, coo_off_h, s);
  if (st == GBS_OK) st = default_plan(A, s);
  if (st == GBS_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("mat_create_coo: synchronising the stream failed");
    st = GBS_ERR_CUDA;
  }
  if (st != GBS_OK) {
    free_handle(A);
    return st;
  }
  *out = A;
  return GBS_OK;
}

}  // namespace gbs

using namespace gbs;

extern "C" {

void ksp_opts_default(ksp_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->rtol = 1e-8;
  o->maxit = -1;
  o->precision = GBS_FP64;
  o->inner_rtol = 1e-4;
  o->max_outer = 30;
  o->inner_maxit = -1;
  o->timeout_ns = 0;
  o->nonzero_guess = 0;
  o->host_loop = 0;
}

int mat_create_coo(int64_t nrows, int64_t ncols, int64_t ncoo, const int32_t *i,
                   const int32_t *j, void *stream, gbs_mat *out) {
  if (!out) {
    set_error("mat_create_coo: out is null");
    return GBS_ERR_ARG;
  }
  *out = nullptr;
  if (nrows < 0 || ncols < 0 || ncoo < 0 || nrows > kMaxIndex || ncols > kMaxIndex ||
      ncoo > kMaxIndex) {
    set_error("mat_create_coo: sizes must be in [0, 2^31)");
    return GBS_ERR_ARG;
  }
  if (ncoo > 0 && (!i || !j)) {
    set_error("mat_create_coo: null i or j");
    return GBS_ERR_ARG;
  }
  gbs_mat A = new (std::nothrow) gbs_mat_s();
  if (!A) return GBS_ERR_ALLOC;
  cudaGetDevice(&A->device);
  A->nrows = nrows;
  A->ncols = ncols;
  A->ncoo = ncoo;
  A->nsys = 1;
  A->row_off_h = {0, nrows};
  return create_common(out, A, i, j, nullptr, (cudaStream_t)stream);
}

int mat_create_coo_batched(int32_t nsys, const int64_t *nrows_h, const int64_t *ncoo_h,
                           const int32_t *i, const int32_t *j, void *stream, gbs_mat *out) {
  if (!out) {
    set_error("mat_create_coo_batched: out is null");
    return GBS_ERR_ARG;
  }
  *out = nullptr;
  if (nsys < 1 || !nrows_h || !ncoo_h) {
    set_error("mat_create_coo_batched: need nsys >= 1 and host size arrays");
    return GBS_ERR_ARG;
  }
  std::vector<int64_t> row_off(nsys + 1, 0), coo_off(nsys + 1, 0);
  for (int32_t s = 0; s < nsys; ++s) {
    if (nrows_h[s] < 0 || ncoo_h[s] < 0) {
      set_error("mat_create_coo_batched: negative size for system %d", s);
      return GBS_ERR_ARG;
    }
    row_off[s + 1] = row_off[s] + nrows_h[s];
    coo_off[s + 1] = coo_off[s] + ncoo_h[s];
  }
  if (row_off[nsys] > kMaxIndex || coo_off[nsys] > kMaxIndex) {
    set_error("mat_create_coo_batched: total rows and COO entries must be < 2^31");
    return GBS_ERR_ARG;
  }
  if (coo_off[nsys] > 0 && (!i || !j)) {
    set_error("mat_create_coo_batched: null i or j");
    return GBS_ERR_ARG;
  }
  gbs_mat A = new (std::nothrow) gbs_mat_s();
  if (!A) return GBS_ERR_ALLOC;
  cudaGetDevice(&A->device);
  A->nrows = A->ncols = row_off[nsys];
  A->ncoo = coo_off[nsys];
  A->nsys = nsys;
  A->batched = true;
  A->row_off_h = row_off;
  return create_common(out, A, i, j, coo_off.data(), (cudaStream_t)stream);
}

int mat_set_values_coo(gbs_mat A, const double *v, int mode, void *stream) {
  GBS_TRY(check_mat(A, "mat_set_values_coo"));
  if (mode != GBS_INSERT && mode != GBS_ADD) {
    set_error("mat_set_values_coo: mode must be GBS_INSERT or GBS_ADD");
    return GBS_ERR_ARG;
  }
  if (A->nkept > 0 && !v) {
    set_error("mat_set_values_coo: v is null");
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(A));
  return launch_set_values(A, v, mode, (cudaStream_t)stream);
}

int mat_mult(gbs_mat A, const double *x, double *y, void *stream) {
  GBS_TRY(check_mat(A, "mat_mult"));
  if (A->nrows > 0 && (!x || !y)) {
    set_error("mat_mult: null x or y");
    return GBS_ERR_ARG;
  }
  if (x == y && x) {
    set_error("mat_mult: x and y must not overlap");
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(A));
  return launch_spmv(A, x, y, (cudaStream_t)stream);
}

// any_method: the generic entry points (ksp_solve*); the CG ones accept CG only.
static int solve_entry(gbs_mat A, const double *b, double *x, const ksp_opts *o,
                       ksp_result *res, void *stream, bool per_system, bool any_method,
                       const char *fn) {
  GBS_TRY(check_mat(A, fn));
  if (A->nrows != A->ncols) {
    set_error("%s: matrix is not square", fn);
    return GBS_ERR_ARG;
  }
  if (A->nrows > 0 && (!b || !x)) {
    set_error("%s: null b or x", fn);
    return GBS_ERR_ARG;
  }
  if (!A->values_set) {
    set_error("%s: mat_set_values_coo has not been called", fn);
    return GBS_ERR_ARG;
  }
  if ((((uintptr_t)b | (uintptr_t)x) & 7u) != 0) {
    set_error("%s: b and x must be 8-byte aligned device pointers", fn);
    return GBS_ERR_ARG;
  }
  ksp_opts oo;
  GBS_TRY(fill_opts(A, o, oo, per_system));
  if (!any_method && oo.method != GBS_KSP_CG && oo.method != GBS_KSP_CGSR) {
    set_error("%s: o->method must be GBS_KSP_CG or GBS_KSP_CGSR (ksp_solve takes the others)",
              fn);
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(A));
  cudaStream_t s = (cudaStream_t)stream;
  if (oo.method == GBS_KSP_CG) GBS_TRY(solve(A, b, x, oo, per_system, s));
  else GBS_TRY(solve_krylov(A, b, x, oo, per_system, s));
  if (res) return read_results(A, res, per_system ? A->nsys : 1, s);
  return GBS_OK;
}

int ksp_solve_cg(gbs_mat A, const double *b, double *x, const ksp_opts *o, ksp_result *res,
                 void *stream) {
  return solve_entry(A, b, x, o, res, stream, false, false, "ksp_solve_cg");
}

int ksp_solve_cg_batched(gbs_mat A, const double *b, double *x, const ksp_opts *o,
                         ksp_result *res_h, void *stream) {
  return solve_entry(A, b, x, o, res_h, stream, true, false, "ksp_solve_cg_batched");
}

int ksp_solve(gbs_mat A, const double *b, double *x, const ksp_opts *o, ksp_result *res,
              void *stream) {
  return solve_entry(A, b, x, o, res, stream, false, true, "ksp_solve");
}

int ksp_solve_batched(gbs_mat A, const double *b, double *x, const ksp_opts *o,
                      ksp_result *res_h, void *stream) {
  return solve_entry(A, b, x, o, res_h, stream, true, true, "ksp_solve_batched");
}

static int adjoint_entry(gbs_mat A, const double *x, const double *dLdx, double *lambda,
                         double *dLda, double *dLdv, const ksp_opts *o, ksp_result *res,
                         void *stream, bool per_system, const char *fn) {
  GBS_TRY(check_mat(A, fn));
  if (A->nrows > 0 && (!x || !dLdx || !lambda)) {
    set_error("%s: null x, dLdx or lambda", fn);
    return GBS_ERR_ARG;
  }
  ksp_opts oo;
  ksp_opts_default(&oo);
  if (o) oo = *o;
  oo.nonzero_guess = 0;
  // the adjoint system is solved in the precision the caller asked for
  int st = solve_entry(A, dLdx, lambda, &oo, nullptr, stream, per_system, false, fn);
  if (st != GBS_OK) return st;
  st = launch_adjoint_scatter(A, lambda, x, dLda, dLdv, (cudaStream_t)stream);
  if (st != GBS_OK) return st;
  if (res) return read_results(A, res, per_system ? A->nsys : 1, (cudaStream_t)stream);
  return GBS_OK;
}

int ksp_adjoint(gbs_mat A, const double *x, const double *dLdx, double *lambda, double *dLda,
                double *dLdv, const ksp_opts *o, ksp_result *res, void *stream) {
  return adjoint_entry(A, x, dLdx, lambda, dLda, dLdv, o, res, stream, false, "ksp_adjoint");
}

int ksp_adjoint_batched(gbs_mat A, const double *x, const double *dLdx, double *lambda,
                        double *dLda, double *dLdv, const ksp_opts *o, ksp_result *res_h,
                        void *stream) {
  return adjoint_entry(A, x, dLdx, lambda, dLda, dLdv, o, res_h, stream, true,
                       "ksp_adjoint_batched");
}

int ksp_get_result(gbs_mat A, ksp_result *res, int32_t count, void *stream) {
  GBS_TRY(check_mat(A, "ksp_get_result"));
  if (!res) {
    set_error("ksp_get_result: res is null");
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(A));
  return read_results(A, res, count, (cudaStream_t)stream);
}

int ksp_get_phase_ns(gbs_mat A, int64_t *phase_ns, void *stream) {
  GBS_TRY(check_mat(A, "ksp_get_phase_ns"));
  if (!phase_ns || !A->ctl) {
    set_error("ksp_get_phase_ns: no solve has run on this matrix, or null output");
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(A));
  return read_phase_ns(A, phase_ns, (cudaStream_t)stream);
}

int mat_get_info(gbs_mat A, int64_t *nrows, int64_t *ncols, int64_t *nnz, int64_t *ncoo,
                 int32_t *nsys) {
  GBS_TRY(check_mat(A, "mat_get_info"));
  if (nrows) *nrows = A->nrows;
  if (ncols) *ncols = A->ncols;
  if (nnz) *nnz = A->nnz;
  if (ncoo) *ncoo = A->ncoo;
  if (nsys) *nsys = A->nsys;
  return GBS_OK;
}

int mat_get_csr(gbs_mat A, const int32_t **row_ptr, const int32_t **col, const double **val,
                int64_t *nnz) {
  GBS_TRY(check_mat(A, "mat_get_csr"));
  if (row_ptr) *row_ptr = A->row_ptr;
  if (col) *col = A->col;
  if (val) *val = A->val;
  if (nnz) *nnz = A->nnz;
  return GBS_OK;
}

int mat_get_coo_maps(gbs_mat A, const int32_t **perm, const int32_t **jmap, int64_t *nkept) {
  GBS_TRY(check_mat(A, "mat_get_coo_maps"));
  if (perm) *perm = A->perm;
  if (jmap) *jmap = A->jmap;
  if (nkept) *nkept = A->nkept;
  return GBS_OK;
}

int mat_set_plan(gbs_mat A, int32_t spmv_rows, int32_t update_rows, int32_t kernel,
                 int32_t ctas_per_sm) {
  GBS_TRY(check_mat(A, "mat_set_plan"));
  GBS_TRY(use_device(A));
  GBS_TRY_CUDA(cudaDeviceSynchronize());  // the old tables may be in use
  GBS_TRY(build_plan(A, spmv_rows, update_rows, kernel, ctas_per_sm, nullptr));
  GBS_TRY_CUDA(cudaDeviceSynchronize());
  return GBS_OK;
}

int mat_set_slice_patterns(gbs_mat A, int32_t on) {
  GBS_TRY(check_mat(A, "mat_set_slice_patterns"));
  if (on != 0 && on != 1) {
    set_error("mat_set_slice_patterns: on = %d must be 0 or 1", on);
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(A));
  GBS_TRY_CUDA(cudaDeviceSynchronize());  // the old copy may be in use
  GBS_TRY(set_slice_patterns(A, on != 0, nullptr));
  GBS_TRY_CUDA(cudaDeviceSynchronize());
  return GBS_OK;
}

int mat_get_slices(gbs_mat A, int64_t *nslices, int64_t *pattern_slices, int64_t *entries) {
  GBS_TRY(check_mat(A, "mat_get_slices"));
  const bool built = A->sell_val != nullptr;
  if (nslices) *nslices = built ? A->nslices : 0;
  if (pattern_slices) *pattern_slices = built ? A->sell_npat : 0;
  if (entries) *entries = built ? A->sell_nnz : 0;
  return GBS_OK;
}

int mat_set_solver(gbs_mat A, int32_t solver) {
  GBS_TRY(check_mat(A, "mat_set_solver"));
  if (solver < GBS_SOLVER_AUTO || solver > GBS_SOLVER_SPLIT) {
    set_error("mat_set_solver: solver must be GBS_SOLVER_AUTO, _PHASES, _CTA or _SPLIT");
    return GBS_ERR_ARG;
  }
  if (solver != A->solver) drop_graphs(A);  // a split loop's graph skips the small systems
  A->solver = solver;
  A->solver_batched_only = false;
  return GBS_OK;
}

int mat_set_split_rows(gbs_mat A, int64_t min_rows) {
  GBS_TRY(check_mat(A, "mat_set_split_rows"));
  if (min_rows < 1) {
    set_error("mat_set_split_rows: min_rows = %lld must be at least 1", (long long)min_rows);
    return GBS_ERR_ARG;
  }
  if (min_rows != A->split_rows) drop_graphs(A);
  A->split_rows = min_rows;
  return GBS_OK;
}

int mat_get_plan(gbs_mat A, int32_t *spmv_rows, int32_t *update_rows, int32_t *kernel,
                 int32_t *ctas_per_sm, int32_t *spmv_grid) {
  GBS_TRY(check_mat(A, "mat_get_plan"));
  if (spmv_rows) *spmv_rows = A->Ra;
  if (update_rows) *update_rows = A->Re;
  if (kernel) *kernel = A->lanes;
  if (ctas_per_sm) *ctas_per_sm = A->ctas_per_sm;
  if (spmv_grid) *spmv_grid = A->ta.grid;
  return GBS_OK;
}

// ------------------------------------------------------------------ autotuner
//
// A candidate is a launch plan (SpMV rows, update rows, row-product kernel,
// CTAs per SM), a solver engine, a CG form and the column pattern setting.
// Each is timed on a fixed 30-iteration FP64 CG run (rtol 0, so every
// candidate does the same work; batched handles solve their systems each on
// their own): one untimed run (it builds the graph), then three timed back
// to back with CUDA events.  First the plans on the phase kernels (a single
// system's with the textbook and the single-reduction form and with the
// column patterns on and off; a batch's with the textbook form); then, with
// the best of them, the other CG forms and (sliced ELL) the per-CTA engine
// -- not for one system whose iteration is far beyond one SM's share -- and
// for a batch the size split and last the other pattern setting.  The three
// fastest are then solved to rtol 1e-8 once each, and the fastest of those
// wins.

namespace {
struct Tuning {
  int32_t Ra, Re, kernel, cpsm, solver, cg_form;
  int64_t split_rows;
  int32_t patterns;  // column patterns of the sliced copy (1 / 0; -1: as they are)
};

// Makes t the handle's plan (rebuilt only when it differs from the current
// one), solver, CG form and column patterns.
int apply_tuning(gbs_mat A, const Tuning &t, cudaStream_t s) {
  if (t.patterns >= 0) GBS_TRY(set_slice_patterns(A, t.patterns != 0, s));
  if (!(t.Ra == A->Ra && t.Re == A->Re && t.kernel == A->lanes && t.cpsm == A->ctas_per_sm))
    GBS_TRY(build_plan(A, t.Ra, t.Re, t.kernel, t.cpsm, s));
  if (t.solver != A->solver || t.split_rows != A->split_rows) drop_graphs(A);
  A->solver = t.solver;
  A->solver_batched_only = A->nsys > 1;  // tuned on the batched solve
  A->cg_form = t.cg_form;
  A->split_rows = t.split_rows;
  return GBS_OK;
}

// The resolved plan of the handle with its solver and form.
Tuning current_tuning(gbs_mat A) {
  return Tuning{A->Ra,     A->Re,         A->lanes,      A->ctas_per_sm,
                A->solver, A->cg_form,    A->split_rows, A->sell_patterns ? 1 : 0};
}

// 257 evenly spaced entries each of row_ptr and col (the cache key's sample).
__global__ void k_key_sample(const int32_t *row_ptr, const int32_t *col, int64_t n, int64_t nnz,
                             int32_t *out) {
  const int q = threadIdx.x;
  if (q < 257) {
    out[q] = row_ptr[n * q / 256];
    out[257 + q] = nnz > 0 ? col[(nnz - 1) * q / 256] : 0;
  }
}
}  // namespace

static int autotune(gbs_mat A, cudaStream_t s, Tuning *out, float *out_ms) {
  const bool per_system = A->nsys > 1;
  const int la = auto_lanes(A->nnz, A->nrows);
  const int sk = A->lanes;  // the kernel the current plan chose
  const int plans[][4] = {{0, 0, sk, 0},      {0, 0, la, 0},       {256, 512, sk, 0},
                          {512, 1024, sk, 0},  {0, 0, sk, 4},       {256, 2048, sk, 0},
                          {0, 0, sk, 2},       {0, 0, sk, 3},       {1024, 4096, sk, 0},
                          {2048, 4096, sk, 0}, {4096, 8192, sk, 0}, {2048, 4096, sk, 2},
                          {4096, 8192, sk, 2}};
  double *b = nullptr, *x = nullptr;
  GBS_TRY(dev_alloc(&b, A->nrows, s));
  GBS_TRY(dev_alloc(&x, A->nrows, s));
  // b = A * 1 (any nonzero right-hand side will do)
  std::vector<double> ones(A->nrows, 1.0);
  cudaMemcpyAsync(x, ones.data(), sizeof(double) * A->nrows, cudaMemcpyHostToDevice, s);
  ksp_opts o;
  ksp_opts_default(&o);
  o.rtol = 0.0;
  o.maxit = 30;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int32_t pat = A->sell_patterns ? 1 : 0;
  Tuning best{A->Ra, A->Re, A->lanes, A->ctas_per_sm, GBS_SOLVER_PHASES, GBS_CG_TEXTBOOK,
              A->split_rows, pat};
  float best_ms = 1e30f;
  int st = GBS_OK;
  std::vector<std::pair<float, Tuning>> tried;
  auto timed = [&](const Tuning &t) -> bool {
    if (apply_tuning(A, t, s) != GBS_OK) return false;
    if (launch_spmv(A, x, b, s) != GBS_OK) return false;
    if (solve(A, b, x, o, per_system, s) != GBS_OK) return false;  // warm-up (and graph build)
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3; ++rep) solve(A, b, x, o, per_system, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = GBS_ERR_CUDA;
      return false;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    tried.push_back({ms, t});
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
    return true;
  };
  // the plans on the phase kernels; a single system's with the textbook and
  // (sliced ELL) the single-reduction form, each with the column patterns as
  // they are and switched (unless the copy takes none): the best plan
  // depends on both
  const int npass = per_system || sk != GBS_SPMV_SELL ? 1 : 2;
  for (int pass = 0; pass < npass && st == GBS_OK; ++pass) {
    const int32_t pp = pass == 0 ? pat : 1 - pat;
    if (pass == 1) {
      if (set_slice_patterns(A, pp != 0, s) != GBS_OK) break;
      if (pp == 1 && A->sell_npat == 0) break;  // patterns do not fit this matrix
    }
    for (const auto &c : plans) {
      if (pass == 1 && c[2] != GBS_SPMV_SELL) continue;  // patterns concern the sliced copy
      for (int32_t form : {GBS_CG_TEXTBOOK, GBS_CG_SINGLE_REDUCTION}) {
        if (form != GBS_CG_TEXTBOOK && (per_system || c[2] != GBS_SPMV_SELL)) continue;
        timed(Tuning{c[0], c[1], c[2], c[3], GBS_SOLVER_PHASES, form, A->split_rows, pp});
        if (st != GBS_OK) break;
      }
      if (st != GBS_OK) break;
    }
  }
  if (st == GBS_OK && best.kernel == GBS_SPMV_SELL) {
    const Tuning base = best;
    Tuning t = base;
    if (per_system) {
      t.cg_form = GBS_CG_SINGLE_REDUCTION;
      timed(t);
    } else {  // the one-kernel form (where it fits, else two)
      t.cg_form = GBS_CG_SINGLE_KERNEL;
      timed(t);
    }
    t = base;
    const int64_t nz = per_system ? A->max_sys_nnz : A->nnz;
    const int64_t rows = per_system ? A->max_sys_rows : A->nrows;
    if (st == GBS_OK && (per_system || nz + 8 * rows <= 16 * CTA_AUTO_WORK)) {
      t = base;
      t.solver = GBS_SOLVER_CTA;
      timed(t);
      if (st == GBS_OK && per_system) {  // batches: also two CTAs per SM
        t.cpsm = 2;
        timed(t);
      }
    }
    // batches: the largest 1, 4, 16, 64 systems on the phase kernels, the
    // rest on the per-CTA solver
    if (per_system) {
      std::vector<int64_t> r(A->nsys);
      for (int32_t q = 0; q < A->nsys; ++q) r[q] = A->row_off_h[q + 1] - A->row_off_h[q];
      std::sort(r.begin(), r.end(), std::greater<int64_t>());
      for (int kth : {1, 4, 16, 64}) {
        if (st != GBS_OK || kth >= A->nsys) break;
        t = base;
        t.solver = GBS_SOLVER_SPLIT;
        t.split_rows = std::max<int64_t>(1, r[kth - 1]);
        timed(t);
      }
    }
  }
  // batches: the best candidate with the column patterns switched, unless
  // the copy takes none either way
  if (st == GBS_OK && per_system && best.kernel == GBS_SPMV_SELL &&
      apply_tuning(A, best, s) == GBS_OK && (best.patterns == 0 || A->sell_npat > 0)) {
    Tuning t = best;
    t.patterns = best.patterns ? 0 : 1;
    timed(t);
  }
  // the three fastest candidates again, each solved to rtol 1e-8 once: 30
  // iterations miss what happens once a batch's systems converge at
  // different iterations (on the C5 batch they ranked two per-CTA solver
  // CTAs per SM first, 2.35 s to convergence against 1.98 s for one)
  if (st == GBS_OK && tried.size() > 1) {
    std::stable_sort(tried.begin(), tried.end(),
                     [](const std::pair<float, Tuning> &p, const std::pair<float, Tuning> &q) {
                       return p.first < q.first;
                     });
    ksp_opts want, full;
    ksp_opts_default(&want);  // rtol 1e-8, the default iteration limit
    if (fill_opts(A, &want, full, per_system) != GBS_OK) full = o;
    full.maxit = std::min(full.maxit, 4096);  // bounds the tuning time of hard systems
    float best_full = 1e30f;
    for (size_t k = 0; k < tried.size() && k < 3 && st == GBS_OK; ++k) {
      const Tuning &t = tried[k].second;
      if (apply_tuning(A, t, s) != GBS_OK) continue;
      cudaMemcpyAsync(x, ones.data(), sizeof(double) * A->nrows, cudaMemcpyHostToDevice, s);
      if (launch_spmv(A, x, b, s) != GBS_OK) continue;             // b = A * 1
      if (solve(A, b, x, o, per_system, s) != GBS_OK) continue;   // warm-up (graph build)
      cudaEventRecord(e0, s);
      const int sst = solve(A, b, x, full, per_system, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = GBS_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (sst == GBS_OK && ms < best_full) {
        best_full = ms;
        best = t;
        best_ms = tried[k].first;
      }
    }
  }
  A->trips_counted = true;  // the timed solves' results are never read
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(b, s);
  dev_free(x, s);
  if (st != GBS_OK) {
    set_error("mat_autotune: a timed run failed");
    return st;
  }
  GBS_TRY(apply_tuning(A, best, s));
  GBS_TRY_CUDA(cudaStreamSynchronize(s));
  if (out) *out = current_tuning(A);  // with the plan's automatic sizes resolved
  if (out_ms) *out_ms = best_ms / 3.0f;
  return GBS_OK;
}

static int autotune_entry(gbs_mat A, const char *fn) {
  GBS_TRY(check_mat(A, fn));
  if (!A->values_set) {
    set_error("%s: mat_set_values_coo has not been called", fn);
    return GBS_ERR_ARG;
  }
  return GBS_OK;
}

int mat_autotune(gbs_mat A, void *stream) {
  GBS_TRY(autotune_entry(A, "mat_autotune"));
  if (A->nrows != A->ncols || A->nrows == 0) return GBS_OK;
  GBS_TRY(use_device(A));
  return autotune(A, (cudaStream_t)stream, nullptr, nullptr);
}

// The cache key of a handle: its sizes, a hash (FNV-1a) of its systems' row
// counts and of 257 evenly spaced entries of row_ptr and of col, and the
// device (name, SM count); the tuning is for FP64 CG.
static int tuning_key(gbs_mat A, cudaStream_t s, std::string *key) {
  const int K = 257;
  std::vector<int32_t> sample(2 * K);
  int32_t *d = nullptr;
  GBS_TRY(dev_alloc(&d, 2 * K, s));
  k_key_sample<<<1, 288, 0, s>>>(A->row_ptr, A->col, A->nrows, A->nnz, d);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sample.data(), d, sizeof(int32_t) * 2 * K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(d, s);
  GBS_TRY_CUDA(e);
  const int32_t *rp = sample.data(), *cl = sample.data() + K;
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t k = 0; k < n; ++k) {
      h ^= c[k];
      h *= 1099511628211ull;
    }
  };
  mix(A->row_off_h.data(), sizeof(int64_t) * A->row_off_h.size());
  mix(rp, sizeof(int32_t) * K);
  mix(cl, sizeof(int32_t) * K);
  cudaDeviceProp prop;
  GBS_TRY_CUDA(cudaGetDeviceProperties(&prop, A->device));
  char buf[512];
  std::string name(prop.name);
  for (char &c : name)
    if (c == ' ' || c == '|') c = '_';
  snprintf(buf, sizeof(buf), "fp64 n=%lld nnz=%lld nsys=%d sig=%016llx dev=%s sm=%d",
           (long long)A->nrows, (long long)A->nnz, A->nsys, (unsigned long long)h, name.c_str(),
           prop.multiProcessorCount);
  *key = buf;
  return GBS_OK;
}

int mat_autotune_file(gbs_mat A, const char *path, int32_t *from_cache, void *stream) {
  GBS_TRY(autotune_entry(A, "mat_autotune_file"));
  if (!path) {
    set_error("mat_autotune_file: null path");
    return GBS_ERR_ARG;
  }
  if (from_cache) *from_cache = 0;
  if (A->nrows != A->ncols || A->nrows == 0) return GBS_OK;
  GBS_TRY(use_device(A));
  cudaStream_t s = (cudaStream_t)stream;
  std::string key;
  GBS_TRY(tuning_key(A, s, &key));
  // one exclusive lock on the file for the lookup and, on a miss, the
  // tuning and the appended line, so concurrent processes tune a key once
  const int fd = open(path, O_RDWR | O_CREAT, 0644);
  if (fd < 0) {
    set_error("mat_autotune_file: cannot open %s", path);
    return GBS_ERR_ARG;
  }
  flock(fd, LOCK_EX);
  FILE *f = fdopen(fd, "r+");
  int st = GBS_OK;
  bool hit = false;
  if (!f) {
    set_error("mat_autotune_file: cannot read %s", path);
    st = GBS_ERR_ARG;
  } else {
    char line[1024];
    Tuning t{};
    while (fgets(line, sizeof(line), f)) {
      const char *bar = strchr(line, '|');
      if (!bar || (size_t)(bar - line) != key.size() + 1 || strncmp(line, key.c_str(), key.size()))
        continue;
      long long sr = 1;
      int pt = -1;
      const int nf = sscanf(bar + 1, " %d %d %d %d %d %d %lld %d", &t.Ra, &t.Re, &t.kernel,
                            &t.cpsm, &t.solver, &t.cg_form, &sr, &pt);
      if (nf >= 6) {  // the last matching line wins
        t.split_rows = nf >= 7 && sr >= 1 ? (int64_t)sr : 1;
        t.patterns = nf == 8 && (pt == 0 || pt == 1) ? pt : -1;
        hit = true;
      }
    }
    if (hit) {
      st = apply_tuning(A, t, s);
      if (st == GBS_OK && cudaStreamSynchronize(s) != cudaSuccess) st = GBS_ERR_CUDA;
      if (st == GBS_OK && from_cache) *from_cache = 1;
    } else {
      float ms = 0;
      st = autotune(A, s, &t, &ms);
      if (st == GBS_OK) {
        fseek(f, 0, SEEK_END);
        fprintf(f, "%s | %d %d %d %d %d %d %lld %d | %.4f ms per 30 iterations\n", key.c_str(),
                t.Ra, t.Re, t.kernel, t.cpsm, t.solver, t.cg_form, (long long)t.split_rows,
                t.patterns, ms);
        fflush(f);
      }
    }
  }
  flock(fd, LOCK_UN);
  if (f) fclose(f);
  else close(fd);
  return st;
}

int mat_set_cg_form(gbs_mat A, int32_t form) {
  GBS_TRY(check_mat(A, "mat_set_cg_form"));
  if (form != GBS_CG_TEXTBOOK && form != GBS_CG_SINGLE_REDUCTION && form != GBS_CG_SINGLE_KERNEL) {
    set_error("mat_set_cg_form: form must be GBS_CG_TEXTBOOK, GBS_CG_SINGLE_REDUCTION or "
              "GBS_CG_SINGLE_KERNEL");
    return GBS_ERR_ARG;
  }
  A->cg_form = form;
  return GBS_OK;
}

int mat_get_tuning(gbs_mat A, int32_t *solver, int32_t *cg_form, int64_t *split_rows) {
  GBS_TRY(check_mat(A, "mat_get_tuning"));
  if (solver) *solver = A->solver;
  if (cg_form) *cg_form = A->cg_form;
  if (split_rows) *split_rows = A->split_rows;
  return GBS_OK;
}

int mat_destroy(gbs_mat A) {
  free_handle(A);
  return GBS_OK;
}

// A vector COO handle is the symbolic stage of an n x 1 matrix whose COO
// column indices are all 0 (the pattern is then the set of distinct i).
struct gbs_vec_s {
  gbs_mat A = nullptr;
};

int vec_create_coo(int64_t n, int64_t ncoo, const int32_t *i, void *stream, gbs_vec *out) {
  if (!out) {
    set_error("vec_create_coo: out is null");
    return GBS_ERR_ARG;
  }
  *out = nullptr;
  if (n < 0 || ncoo < 0 || n > kMaxIndex || ncoo > kMaxIndex) {
    set_error("vec_create_coo: sizes must be in [0, 2^31)");
    return GBS_ERR_ARG;
  }
  if (ncoo > 0 && !i) {
    set_error("vec_create_coo: null i");
    return GBS_ERR_ARG;
  }
  gbs_vec V = new (std::nothrow) gbs_vec_s();
  if (!V) return GBS_ERR_ALLOC;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *zeros = nullptr;
  int st = GBS_OK;
  if (ncoo > 0) {
    if (dev_alloc(&zeros, ncoo, s) != GBS_OK ||
        cudaMemsetAsync(zeros, 0, sizeof(int32_t) * ncoo, s) != cudaSuccess) {
      set_error("vec_create_coo: allocating the column indices failed");
      st = GBS_ERR_ALLOC;
    }
  }
  if (st == GBS_OK) {
    gbs_mat A = new (std::nothrow) gbs_mat_s();
    if (!A) st = GBS_ERR_ALLOC;
    else {
      cudaGetDevice(&A->device);
      A->nrows = n;
      A->ncols = 1;
      A->ncoo = ncoo;
      A->nsys = 1;
      A->row_off_h = {0, n};
      st = symbolic(A, i, zeros, nullptr, s);
      if (st == GBS_OK) V->A = A;
      else free_handle(A);
    }
  }
  dev_free(zeros, s);
  if (st != GBS_OK) {
    delete V;
    return st;
  }
  *out = V;
  return GBS_OK;
}

int vec_set_values_coo(gbs_vec V, const double *v, int mode, double *y, void *stream) {
  if (!V || !V->A) {
    set_error("vec_set_values_coo: null vector handle");
    return GBS_ERR_ARG;
  }
  if (mode != GBS_INSERT && mode != GBS_ADD) {
    set_error("vec_set_values_coo: mode must be GBS_INSERT or GBS_ADD");
    return GBS_ERR_ARG;
  }
  if ((V->A->nkept > 0 && !v) || (V->A->nrows > 0 && !y)) {
    set_error("vec_set_values_coo: null v or y");
    return GBS_ERR_ARG;
  }
  GBS_TRY(use_device(V->A));
  return launch_vec_set_values(V->A, v, mode, y, (cudaStream_t)stream);
}

int vec_get_info(gbs_vec V, int64_t *n, int64_t *nentries, int64_t *ncoo) {
  if (!V || !V->A) {
    set_error("vec_get_info: null vector handle");
    return GBS_ERR_ARG;
  }
  if (n) *n = V->A->nrows;
  if (nentries) *nentries = V->A->nnz;
  if (ncoo) *ncoo = V->A->ncoo;
  return GBS_OK;
}

int vec_destroy(gbs_vec V) {
  if (!V) return GBS_OK;
  free_handle(V->A);
  delete V;
  return GBS_OK;
}

int64_t gbs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *gbs_last_error(void) { return g_err; }

}  // extern "C"
