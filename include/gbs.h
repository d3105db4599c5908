/*
 * gbs.h -- C-ABI of the GB300 sparse SPD solver library (libgbs.so).
 *
 * The library assembles a CSR matrix on the GPU from COO triples, summing
 * duplicates, and solves A x = b with a Jacobi-preconditioned conjugate
 * gradient whose iterations run inside one CUDA graph: SpMV fused with p.Ap,
 * the vector updates fused with their dot products, device-resident scalars,
 * and a loop condition set on the device.  On top of that sit an
 * FP32-inner / FP64-refined solve, a batched solve of many independent
 * systems in one graph launch, and the adjoint of the solve.
 *
 * Paper: "PETSc/TAO developments for GPU-based early exascale systems".
 *   - COO assembly: Sec. 5 (MatSetPreallocationCOO / MatSetValuesCOO).
 *   - CG with device-resident scalars and no host round trip: Sec. 6.1
 *     (CGAsync), Sec. 6.2.
 *   - Diagonal (Jacobi) preconditioning and batched solvers: Sec. 7.
 *   - Multiprecision (single-precision inner solver): Sec. 2, challenge A7.
 *   - Adjoint capability: Sec. 1.
 *   - One stream handle per call, device pointers in and out: Sec. 2.
 *
 * Conventions for every entry point:
 *   - Pointers are DEVICE pointers unless the comment says "host".  The
 *     vectors handed to the solves (b, x, dLdx, lambda) must be 8-byte
 *     aligned (GBS_ERR_ARG otherwise).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  All work is enqueued on that stream.  Unless stated otherwise a
 *     call is asynchronous: the caller keeps every borrowed buffer alive (and
 *     unmodified, for inputs) until the stream has passed the call.
 *   - Every function returns a status code (GBS_OK = 0).  No exception or
 *     signal crosses the ABI.  On failure gbs_last_error() returns a
 *     thread-local message.  Errors the host can see (bad arguments, CUDA API
 *     failures) are returned at once; errors found on the device (index out of
 *     range, bad diagonal, breakdown, NaN, iteration limit, time limit)
 *     are returned by the next call that synchronises (mat_create_coo*, or a
 *     solve given a non-NULL result pointer, or ksp_get_result).
 *   - Index type: int32 row/column indices, int32 CSR row pointers; so
 *     nrows, ncols, ncoo and nnz must each be < 2^31.
 *   - A matrix handle is used by one host thread at a time.
 */
#ifndef GBS_H
#define GBS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbs_mat_s *gbs_mat; /* opaque; owned by the library */
typedef struct gbs_vec_s *gbs_vec; /* opaque; owned by the library */

enum {
  GBS_OK = 0,
  GBS_ERR_ARG = 1,        /* invalid argument (host check) */
  GBS_ERR_INDEX = 2,      /* a kept COO index >= nrows / ncols */
  GBS_ERR_ALLOC = 3,      /* device or host allocation failed */
  GBS_ERR_CUDA = 4,       /* a CUDA runtime call failed */
  GBS_ERR_NOT_SPD = 5,    /* missing or non-positive diagonal, or r.z <= 0 */
  GBS_ERR_BREAKDOWN = 6,  /* p.Ap <= 0 (matrix not SPD) */
  GBS_ERR_NAN = 7,        /* NaN / Inf met in the iteration or in b */
  GBS_ERR_MAXIT = 8,      /* iteration limit reached before rtol */
  GBS_ERR_STAGNATION = 9, /* refined solve: residual stopped decreasing */
  GBS_ERR_TIMEOUT = 10,   /* the solve ran longer than ksp_opts.timeout_ns */
  GBS_ERR_LAUNCH = 11     /* a kernel or graph could not be launched */
};

enum { GBS_INSERT = 0, GBS_ADD = 1 };
enum { GBS_FP64 = 0, GBS_FP32_REFINED = 1 };
/* Row-product kernels of a launch plan (mat_set_plan); a positive value n in
 * {1, 2, 4, 8, 32} selects the CSR-vector kernel with n lanes per row. */
enum { GBS_SPMV_AUTO = -1, GBS_SPMV_SELL = 0 };
/* Solvers (mat_set_solver). */
enum { GBS_SOLVER_AUTO = 0, GBS_SOLVER_PHASES = 1, GBS_SOLVER_CTA = 2, GBS_SOLVER_SPLIT = 3 };
/* Forms of CG on the phase kernels (mat_set_cg_form, chosen by the autotuner). */
enum { GBS_CG_TEXTBOOK = 0, GBS_CG_SINGLE_REDUCTION = 1, GBS_CG_SINGLE_KERNEL = 2 };
/* Krylov methods (ksp_opts.method; Sec. 7 batched solvers, Sec. 6.2). */
enum { GBS_KSP_CG = 0, GBS_KSP_BICG = 1, GBS_KSP_TFQMR = 2, GBS_KSP_PIPECG = 3,
       GBS_KSP_CGSR = 4 };

/* Solver options (host struct).  Fill with ksp_opts_default(), then override. */
typedef struct {
  double rtol;          /* stop when ||r||_2 <= rtol ||b||_2 (default 1e-8) */
  int32_t maxit;        /* < 0: 10 n capped at 100000, n = largest system;
                           0 stops at once with GBS_ERR_MAXIT unless b = 0 */
  int32_t precision;    /* GBS_FP64 or GBS_FP32_REFINED */
  double inner_rtol;    /* refined: FP32 inner tolerance (<= 0: 1e-4); an inner
                           solve stops at max(inner_rtol, rtol ||b|| / (2 s))
                           times its initial residual, s = the FP64 residual
                           norm it corrects */
  int32_t max_outer;    /* refined: max refinement steps (< 0: 30) */
  int32_t inner_maxit;  /* refined: inner products per step (< 0: as maxit) */
  int64_t timeout_ns;   /* wall-clock limit of the iteration loop, checked
                           on the device once per iteration; systems still
                           iterating then end with GBS_ERR_TIMEOUT (<= 0:
                           no limit, the default).  The per-CTA solver and
                           the host-stepped loop stop at that iteration; the
                           graph-driven loop finishes its body of 8 trips,
                           so up to 7 more iterations may run */
  int32_t nonzero_guess;/* 1: x holds the initial guess; 0: start from x = 0 */
  int32_t host_loop;    /* 0 (default): one CUDA graph launch per solve, the
                           loop runs on the device.  1: no graph; the host
                           launches the iteration kernels in chunks of 16
                           and reads a 4-byte stop flag after each chunk
                           (synchronising the stream once per chunk), so
                           profilers that cannot follow device-side graph
                           loops see every kernel */
  int32_t method;       /* GBS_KSP_CG (default), GBS_KSP_CGSR, GBS_KSP_BICG,
                           GBS_KSP_TFQMR or GBS_KSP_PIPECG; the CG entry
                           points (ksp_solve_cg*, ksp_adjoint*) take the two
                           CG forms, ksp_solve / ksp_solve_batched all */
} ksp_opts;

/* Per-solve (or per-system) result, host struct. */
typedef struct {
  int32_t status;           /* GBS_OK or the GBS_ERR_* that ended the solve */
  int32_t iterations;       /* CG and BiCG: products q = A p (refined: total
                               inner ones); TFQMR: products with A D^-1;
                               pipelined CG: x updates (= CG's count) */
  int32_t outer_iterations; /* refined: refinement steps; FP64: 0 */
  int32_t solver;           /* GBS_SOLVER_PHASES, _CTA or _CLUSTER: which ran */
  double rnorm0;            /* ||b - A x0||_2 */
  double rnorm;             /* last recursively updated residual norm
                               (refined: last FP64 outer residual norm;
                               TFQMR: the quasi-residual bound tau sqrt(m+1)) */
  double true_rel_residual; /* ||b - A x||_2 / ||b||_2 recomputed at exit */
} ksp_result;

/* Fills *o with the defaults listed above. */
void ksp_opts_default(ksp_opts *o);

/*
 * Symbolic COO stage (Sec. 5, MatSetPreallocationCOO(A, n, i, j)).
 * i, j: int32[ncoo] device arrays; an entry with i[k] < 0 or j[k] < 0 is
 * ignored (Sec. 5 allows negative indices to mark entries to skip).  The
 * pattern is the set of distinct kept (i, j), rows ascending and columns
 * strictly ascending.  i and j are only read during this call and may be freed
 * after it returns.  Builds on the device: the CSR structure, the map from
 * sorted position to COO index (perm) and the segment offsets (jmap), the
 * diagonal positions and the launch plan.  Synchronises `stream` (nnz is
 * data-dependent).  Errors: GBS_ERR_ARG (sizes), GBS_ERR_INDEX (a kept index
 * out of range), GBS_ERR_ALLOC, GBS_ERR_CUDA.  On success *out is a new
 * handle, to be released with mat_destroy.
 */
int mat_create_coo(int64_t nrows, int64_t ncols, int64_t ncoo, const int32_t *i,
                   const int32_t *j, void *stream, gbs_mat *out);

/*
 * Batched symbolic stage (Sec. 7 batched systems; Sec. 5 COO per system).
 * nsys independent square systems; nrows_h[s], ncoo_h[s] are HOST arrays;
 * i, j are the systems' COO indices concatenated in system order, each LOCAL to
 * its system (0 <= i < nrows_h[s]; negative = ignored).  The handle holds one
 * block-diagonal CSR of sum(nrows_h) rows; ksp_solve_cg_batched solves the
 * systems independently, ksp_solve_cg solves the stacked ("ensemble", Sec. 7)
 * system with one global norm.  Same synchronisation and errors as
 * mat_create_coo.
 */
int mat_create_coo_batched(int32_t nsys, const int64_t *nrows_h, const int64_t *ncoo_h,
                           const int32_t *i, const int32_t *j, void *stream,
                           gbs_mat *out);

/*
 * Numeric COO stage (Sec. 5, MatSetValuesCOO(A, v, mode)).
 * v: double[ncoo] device array in the same order as the i/j given at creation
 * (entries that were ignored are not read).  Each nonzero a_p is the sum of its
 * contributions in increasing COO index order, computed by one thread with no
 * atomics; GBS_INSERT replaces the stored value, GBS_ADD adds to it.  Also
 * refreshes the Jacobi diagonal inverse used by the solves (a missing or
 * non-positive diagonal is reported as GBS_ERR_NOT_SPD by the next solve).
 * Asynchronous.
 */
int mat_set_values_coo(gbs_mat A, const double *v, int mode, void *stream);

/* y = A x (the MatMult of Sec. 6.1), FP64.  x: double[ncols], y: double[nrows],
 * must not overlap.  The row products are those of the launch plan (see
 * mat_set_plan).  Asynchronous. */
int mat_mult(gbs_mat A, const double *x, double *y, void *stream);

/*
 * Jacobi-preconditioned CG on the whole matrix (Sec. 6.1 CG without host
 * round trips; Sec. 7 diagonal preconditioner).  b, x: double[nrows]; x is the
 * initial guess when o->nonzero_guess, else overwritten from 0.  One CUDA
 * graph launch runs the solve: a setup kernel, a conditional WHILE node whose
 * body is three kernels per iteration (SpMV fused with p.Ap; the x/r updates
 * fused with r.z and ||r||^2; the p update, whose CTA 0 sets the loop
 * condition), and a closing true-residual kernel.  Reductions are
 * deterministic and the scalars stay on the device.  The graph is built on
 * the first solve of each shape (precision, batched or not) and replayed
 * afterwards; the call arguments are written to the device by a one-thread
 * kernel first.  o->precision =
 * GBS_FP32_REFINED runs FP32 inner PCG (FP32 values, vectors, reductions)
 * inside FP64 iterative refinement (Sec. 2, A7).  o may be NULL (defaults).
 * res (host): if non-NULL the call synchronises and fills it, and returns its
 * status; if NULL the call is asynchronous and the result can be fetched later
 * with ksp_get_result.  o->method must be GBS_KSP_CG or GBS_KSP_CGSR (the
 * single-reduction form described at ksp_solve; else GBS_ERR_ARG).
 */
int ksp_solve_cg(gbs_mat A, const double *b, double *x, const ksp_opts *o,
                 ksp_result *res, void *stream);

/*
 * Batched solve of a handle made by mat_create_coo_batched: every system runs
 * its own PCG (own alpha, beta, norms, stopping test ||r_s|| <= rtol ||b_s||)
 * in the same graph launch, each kernel covering all systems; converged
 * systems are frozen and the loop ends when none is left.  b, x: double[sum
 * nrows] in system order.  res_h: HOST array of nsys results or NULL
 * (asynchronous).  Returns the first non-OK system status when res_h is
 * given.
 */
int ksp_solve_cg_batched(gbs_mat A, const double *b, double *x, const ksp_opts *o,
                         ksp_result *res_h, void *stream);

/*
 * Krylov solve with the method o->method (Sec. 7: PETSc's batched solvers are
 * TFQMR and BiCG with diagonal preconditioning; CG as in ksp_solve_cg).
 * ksp_solve treats the whole matrix as one system (for a batched handle, the
 * stacked "ensemble" of Sec. 7); ksp_solve_batched solves each system of a
 * batched handle on its own, with its own scalars and stopping test.
 *
 *   GBS_KSP_CG: identical to ksp_solve_cg / ksp_solve_cg_batched.
 *   GBS_KSP_CGSR: the same Jacobi-PCG in Chronopoulos and Gear's
 *     single-reduction form (PCG's iterates in exact arithmetic): r.u, w.u
 *     and ||r||^2 are reduced together right after the product w = A u, and
 *     alpha, beta follow from them (alpha = r.u / (w.u - beta r.u /
 *     alpha_prev)), so an iteration is TWO kernels -- the product fused with
 *     the one reduction, then one element-wise update of p, s = A p, x, r and
 *     u = M^-1 r with no reduction -- against the textbook form's three and
 *     two.  Same stopping test, counts (x updates) and statuses as CG;
 *     traffic 12 nnz + 128 n bytes per iteration.  Runs on the phase kernels
 *     (any solver setting), FP64.
 *   GBS_KSP_BICG: biconjugate gradients with M = diag(A) on both sequences
 *     and shadow residual rt0 = r0; q = A p and qt = A^T pt each iteration,
 *     A^T from a transposed sliced-ELL copy built on the first BiCG solve
 *     (its values refreshed after every mat_set_values_coo).  Stops when
 *     ||r|| <= rtol ||b|| (tested before each iteration).  For symmetric A
 *     it performs PCG's operations.
 *   GBS_KSP_TFQMR: Freund's transpose-free QMR on A M^-1 u = b, x = M^-1 u,
 *     M = diag(A) (right preconditioning, so its bound refers to b - A x);
 *     stops when the quasi-residual bound tau sqrt(m + 1) <= rtol ||b||
 *     (m = half steps).  Two products with A per step.
 *   GBS_KSP_PIPECG: pipelined Jacobi-PCG (Ghysels-Vanroose): PCG's iterates
 *     in exact arithmetic, with the recurrences u = M^-1 r, w = A u, s = A p,
 *     q = M^-1 s, z = A q carried along so that an iteration needs ONE
 *     reduction (r.u, w.u, ||r||^2 together) and one product.  For the
 *     latency-bound regime where Sec. 6.2's asynchronous solvers gain most:
 *     it always runs on the phase kernels, one fused kernel per iteration
 *     (CG takes three, with two reductions), at the price of more vector
 *     traffic (152 n + 12 nnz bytes per iteration against CG's 112 n + 12
 *     nnz) and the method's larger drift between the recursive and the true
 *     residual.  Same stopping test and statuses as CG.
 *
 * BiCG, TFQMR, pipelined and single-reduction CG run in FP64 (o->precision
 * must be GBS_FP64).  BiCG and TFQMR run on the per-CTA solver (one 1024-thread CTA
 * per system, every iteration inside one kernel launch, systems largest
 * first) or on the grid-wide phase kernels in a CUDA graph, chosen as for CG
 * by mat_set_solver (automatic: per-CTA when the largest system has at most
 * 40000 nonzeros plus eight per row, or a batch has at least one system per
 * SM); o->host_loop applies to the phase kernels.  A zero or negative diagonal entry ends the solve
 * with GBS_ERR_NOT_SPD (the Jacobi preconditioner needs a positive diagonal);
 * rt.v = 0 or rho = 0 (TFQMR), rho = 0 or pt.q = 0 (BiCG) with
 * GBS_ERR_BREAKDOWN.  Arguments, results and synchronisation as in
 * ksp_solve_cg / ksp_solve_cg_batched (a handle made by mat_create_coo has
 * one system).  Workspace: 9 (TFQMR) or 6 (BiCG) FP64 vectors of
 * nrows (pipelined CG: 9), allocated on first use and kept with the handle.
 */
int ksp_solve(gbs_mat A, const double *b, double *x, const ksp_opts *o, ksp_result *res,
              void *stream);
int ksp_solve_batched(gbs_mat A, const double *b, double *x, const ksp_opts *o,
                      ksp_result *res_h, void *stream);

/*
 * Adjoint of x = A^{-1} b (Sec. 1 adjoint capability), for symmetric A:
 * solves A^T lambda = dLdx with the same CG kernels (o->rtol, default 1e-8),
 * then writes dL/db = lambda, dLda[p] = -lambda[row p] x[col p] over the
 * pattern (double[nnz], may be NULL) and dLdv[k] = dLda[p(k)] for every kept
 * COO entry, 0 for ignored ones (double[ncoo], may be NULL).  Symmetry is the
 * caller's contract (it is not checked).  res as in ksp_solve_cg.
 */
int ksp_adjoint(gbs_mat A, const double *x, const double *dLdx, double *lambda,
                double *dLda, double *dLdv, const ksp_opts *o, ksp_result *res,
                void *stream);

/* Batched adjoint: per-system lambda solves in one launch, then the same
 * scatters over the concatenated arrays.  res_h: HOST array of nsys or NULL. */
int ksp_adjoint_batched(gbs_mat A, const double *x, const double *dLdx, double *lambda,
                        double *dLda, double *dLdv, const ksp_opts *o,
                        ksp_result *res_h, void *stream);

/*
 * Allocation-free FP64 solve.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory -- code whose
 * device memory is budgeted and handed out by another allocator, or that
 * cannot afford the device-wide synchronisation cudaMalloc / cudaFree imply.
 * It runs the same Jacobi-PCG phase kernels as ksp_solve_cg, on a CSR
 * matrix the caller owns: row_ptr int32[n+1], col int32[nnz] (each < n),
 * val double[nnz]; b, x double[n]; all five 16-byte aligned.  All
 * its scratch lives in one fixed static device array (about 8.5 MB, resident
 * on every GPU that loads the library until the process exits), so n must be
 * <= 262144; a larger n returns
 * GBS_ERR_ARG without touching the GPU.  It calls no cudaMalloc, cudaFree or
 * other allocating routine, and builds no CUDA graph: the host launches the
 * iterations in chunks of 16 and reads a 4-byte stop flag after each chunk,
 * so the call synchronises `stream` once per chunk and once at the end, and
 * always returns the solve's status (GBS_ERR_NOT_SPD for a missing or
 * non-positive diagonal, GBS_ERR_MAXIT, ... as ksp_solve_cg).  Every call
 * shares that array, which keeps the last call's contents: calls that overlap
 * on the GPU (other streams or host threads) race, so the caller must
 * serialise them.  The first call on a device looks up the array's device
 * address and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point on a device
 * after a cudaDeviceReset of it (the kept address is then stale).  o: NULL
 * (defaults) or method GBS_KSP_CG with precision GBS_FP64 (GBS_ERR_ARG
 * otherwise; host_loop is ignored, the loop is always host-stepped).  res
 * (host): NULL or the result to fill.
 */
int ksp_solve_cg_noalloc(int64_t n, const int32_t *row_ptr, const int32_t *col,
                         const double *val, const double *b, double *x,
                         const ksp_opts *o, ksp_result *res, void *stream);

/* Synchronises `stream` and copies the results of the last solve on A into the
 * HOST array res (nsys entries for a batched solve, else 1).  Returns the first
 * non-OK status. */
int ksp_get_result(gbs_mat A, ksp_result *res, int32_t count, void *stream);

/* Diagnostic: wall time the last solve on A spent in each phase (ns, HOST
 * array of 5: setup, SpMV phase, x/r update phase, p update phase, closing
 * true residual), summed over iterations.  A phase's time runs from the start
 * of its kernel's CTA 0 to the start of the next phase kernel's CTA 0, so it
 * includes the launch gap after it.  Synchronises `stream`. */
int ksp_get_phase_ns(gbs_mat A, int64_t *phase_ns, void *stream);

/* Sizes (host outputs; any may be NULL). */
int mat_get_info(gbs_mat A, int64_t *nrows, int64_t *ncols, int64_t *nnz,
                 int64_t *ncoo, int32_t *nsys);

/* Borrowed device views of the CSR arrays, valid until mat_destroy (host
 * outputs; any may be NULL). */
int mat_get_csr(gbs_mat A, const int32_t **row_ptr, const int32_t **col,
                const double **val, int64_t *nnz);

/* Borrowed device views of the COO maps: perm[nkept] (sorted position ->
 * original COO index) and jmap[nnz+1] (segment offsets into perm). */
int mat_get_coo_maps(gbs_mat A, const int32_t **perm, const int32_t **jmap,
                     int64_t *nkept);

/*
 * Launch plan used by mat_mult and the solves.  Every phase kernel runs
 * 512-thread CTAs; a CTA walks blocks c, c + grid, ... of its phase's block
 * table.  spmv_rows: rows per block of the SpMV phases (a multiple of 32 in
 * [32, 65536], or 0: about one block per CTA, at least 256); update_rows:
 * rows per block of the vector-update phases (same).  kernel: the row
 * products --
 *   GBS_SPMV_SELL: a sliced-ELL copy of the matrix (32-row slices stored
 *     column-major, padding skipped), one lane per row, built on first use
 *     (at most (4 + 8) bytes per padded entry more device memory, plus 4
 *     bytes more once a refined solve needs FP32 values; column patterns,
 *     mat_set_slice_patterns, replace the column indices);
 *   1, 2, 4, 8 or 32: the CSR arrays read by that many lanes per row;
 *   GBS_SPMV_AUTO: sliced ELL when padding to the slices' longest rows adds
 *     at most 20% to the entries, else CSR-vector with lanes from the mean
 *     row length.
 * Every kernel sums each row in CSR order with one FMA per nonzero except
 * CSR-vector with more than one lane, which splits the row over the lanes
 * and adds the lane sums in a fixed tree.  ctas_per_sm: cap on the grids in
 * CTAs per SM (1..64), or 0 for as many as fit on an SM at once (each phase
 * kernel then runs in one wave and keeps one reduction slot per CTA); the
 * per-CTA CG solver (mat_set_solver) runs one CTA per SM, or two under a cap
 * of two or more when a batch has more systems than SMs.  mat_set_plan
 * synchronises the device (the old tables may be in use) and drops the
 * cached solve graphs.  mat_create_coo picks (0, 0, GBS_SPMV_AUTO, 0);
 * mat_autotune (below) picks among candidates by timing them.  mat_get_plan
 * returns the kernel in use (never AUTO) and the grid of the SpMV-phase
 * kernels.  Host outputs may be NULL.
 */
int mat_set_plan(gbs_mat A, int32_t spmv_rows, int32_t update_rows, int32_t kernel,
                 int32_t ctas_per_sm);

/*
 * Column patterns of the sliced-ELL copy (on = 1, the default, or 0).  With
 * patterns on, a 32-row slice whose rows draw their offsets col - row from a
 * common set of at most 32 (at most a quarter more than its longest row)
 * stores that set once, ascending, and one 32-bit mask per row instead of a
 * column index per entry; its width becomes the set's size and entries a
 * row lacks hold 0 and are skipped by the mask.  The row products sum the
 * same terms in the same (CSR) order either way, so every result is
 * bit-identical with patterns on or off; only the bytes read change (8 per
 * FP64 entry plus 4 per row, against 10 or 12 per entry).  A copy that
 * exists (and the transpose's, for BiCG) is rebuilt at once; cached graphs
 * are dropped.  Synchronises the device.  mat_get_slices returns the copy's
 * slices, how many of them have a pattern and its padded entries (host
 * outputs, each may be NULL; zeros while no copy is built).
 */
int mat_set_slice_patterns(gbs_mat A, int32_t on);
int mat_get_slices(gbs_mat A, int64_t *nslices, int64_t *pattern_slices, int64_t *entries);
int mat_get_plan(gbs_mat A, int32_t *spmv_rows, int32_t *update_rows, int32_t *kernel,
                 int32_t *ctas_per_sm, int32_t *spmv_grid);

/*
 * Which solver runs the solves on A (Sec. 6.1 device-side iteration either
 * way; both give the same iteration up to reduction order):
 *   GBS_SOLVER_PHASES: the grid-wide phase kernels in a CUDA graph (SpMV,
 *     vector update, direction update per iteration), for large systems;
 *   GBS_SOLVER_CTA: one 1024-thread CTA per system runs every iteration in
 *     one kernel with CTA barriers only -- the latency path for small systems,
 *     and for batches of many systems, which then run as concurrent CTAs,
 *     largest first (CG: a grid of one CTA per SM -- two under a plan
 *     cap of two or more -- each taking the next system when it is done).  Needs the sliced-ELL plan kernel (GBS_ERR_ARG from the
 *     solve otherwise); ignores host_loop; ksp_get_phase_ns reports zeros;
 *   GBS_SOLVER_SPLIT: CG (FP64 or refined) of a batched solve
 *     (ksp_solve_cg_batched, ksp_adjoint_batched) by size: the systems with
 *     at least mat_set_split_rows' row count run on the phase kernels (the
 *     whole GPU per iteration, one graph launch for all of them), then the
 *     others on the per-CTA solver, so that no large system ends the batch
 *     alone on one SM.  Needs the sliced-ELL plan kernel; a solve that is not
 *     batched, or another method, takes GBS_SOLVER_AUTO's choice;
 *   GBS_SOLVER_AUTO (default): CTA when the largest system solved has at
 *     most 40000 nonzeros plus eight per row (the FP64 work of one iteration
 *     that one SM does faster than the phase kernels' fixed cost per
 *     iteration), or a batched solve has at least 2 systems per SM.
 * ksp_result.solver tells which one ran.  No synchronisation.
 */
int mat_set_solver(gbs_mat A, int32_t solver);
/* The row count from which a system of a batched solve runs on the phase
 * kernels under GBS_SOLVER_SPLIT (>= 1; the autotuner sets it).  Cached
 * graphs are dropped.  No synchronisation. */
int mat_set_split_rows(gbs_mat A, int64_t min_rows);

/*
 * The form of FP64 CG (ksp_solve_cg*, ksp_adjoint*, method GBS_KSP_CG) on the
 * phase kernels: GBS_CG_TEXTBOOK (default; three kernels and two reductions
 * per iteration), GBS_CG_SINGLE_REDUCTION (the GBS_KSP_CGSR loop: two
 * kernels and one reduction, the same iterates in exact arithmetic) or
 * GBS_CG_SINGLE_KERNEL (the same loop as ONE kernel per iteration: each CTA
 * updates its rows, waits -- spinning on flags in device memory, bounded by
 * about a second, after which the solve ends with GBS_ERR_TIMEOUT -- until
 * the CTAs holding the rows its row products read have updated theirs, then
 * runs its row products; the grid is launched cooperatively, so all its
 * CTAs are resident together).  The single-reduction forms need the
 * sliced-ELL plan kernel (else the textbook form runs); the single-kernel
 * form also needs an ensemble solve (ksp_solve_cg, one system or a batch
 * solved as one), else the two-kernel form runs.  GBS_KSP_CGSR follows the
 * handle's form too: the single-kernel form where it applies, else two
 * kernels.  The per-CTA solver and the refined solve always use the
 * textbook form.  No synchronisation.  mat_get_tuning returns the solver
 * setting (mat_set_solver), the CG form and the split row count
 * (mat_set_split_rows) (host outputs, each may be NULL).
 */
int mat_set_cg_form(gbs_mat A, int32_t form);
int mat_get_tuning(gbs_mat A, int32_t *solver, int32_t *cg_form, int64_t *split_rows);

/*
 * Autotuner of the FP64 CG solve ("rows-per-warp and block shapes picked by a
 * project-written autotuner"): candidates are launch plans (as mat_set_plan:
 * block rows, row-product kernel, CTAs per SM) -- for a handle of one system
 * each with the textbook and the two-kernel single-reduction CG form and
 * with the column patterns of the sliced copy (mat_set_slice_patterns) on
 * and off, unless the copy takes none -- then, for the fastest of them, the
 * one-kernel form (one system) or the single-reduction form (batches), the
 * per-CTA engine (sliced ELL; batches, or systems within 16 times the
 * per-CTA size rule), and for batches the size split (GBS_SOLVER_SPLIT) at
 * the row counts of the 1st, 4th, 16th and 64th largest systems and last the
 * other pattern setting.  Each candidate runs a fixed 30-iteration FP64
 * CG (rtol 0, every candidate the same work; a batched handle solves its
 * systems each on its own) once untimed and three times under CUDA events
 * on `stream`; the three fastest then each solve A x = A 1 to rtol 1e-8
 * once (timed; at most 4096 iterations), which catches what 30 iterations miss (a batch's systems
 * converging at different iterations), and the fastest of those becomes the
 * handle's plan, solver (mat_set_solver), CG form (mat_set_cg_form), split
 * row count (mat_set_split_rows) and pattern setting; on a batched handle
 * the engine chosen for its
 * batched solves leaves its ensemble solves (ksp_solve on the stacked
 * system) to GBS_SOLVER_AUTO's choice.  Synchronises.
 *
 * mat_autotune_file: the same, persisted.  path names a text file (created if
 * missing) of one line per tuned key: "<key> | Ra Re kernel ctas_per_sm
 * solver cg_form split_rows patterns | <time>" (lines without the last one
 * or two fields leave those settings as they are).  The key holds the handle's sizes, a hash of its
 * systems' sizes and of 257 sampled entries each of row_ptr and col, the
 * device name and SM count, and "fp64".  A matching line is applied without
 * timing (*from_cache = 1); otherwise the handle is tuned and the line
 * appended (*from_cache = 0).  The file is held under an exclusive lock
 * (flock) meanwhile.  from_cache (host) may be NULL.  GBS_ERR_ARG if the
 * file cannot be opened.
 */
int mat_autotune(gbs_mat A, void *stream);
int mat_autotune_file(gbs_mat A, const char *path, int32_t *from_cache, void *stream);

/* Releases every device buffer the handle owns.  Synchronises the device
 * buffers' last stream first.  NULL is accepted. */
int mat_destroy(gbs_mat A);

/*
 * Vector COO assembly (Sec. 5's COO interface applied to vectors:
 * VecSetPreallocationCOO / VecSetValuesCOO).  vec_create_coo: i int32[ncoo]
 * device array of indices in [0, n) (negative = ignored; read only during
 * the call); builds the set of distinct kept indices and the maps with the
 * matrix symbolic stage (an n x 1 pattern).  Synchronises `stream`; errors as
 * mat_create_coo (GBS_ERR_INDEX for an index >= n).
 * vec_set_values_coo: v double[ncoo] in the same order; for every index r
 * that appears, y[r] becomes the in-order sum of its v[k] (GBS_INSERT) or
 * y[r] plus that sum (GBS_ADD); entries of y whose index does not appear are
 * left as they are.  y: double[n] device array.  Asynchronous.
 * vec_get_info: n, the number of distinct indices and ncoo (host outputs,
 * any may be NULL).  vec_destroy: releases the handle (NULL accepted).
 */
int vec_create_coo(int64_t n, int64_t ncoo, const int32_t *i, void *stream, gbs_vec *out);
int vec_set_values_coo(gbs_vec V, const double *v, int mode, double *y, void *stream);
int vec_get_info(gbs_vec V, int64_t *n, int64_t *nentries, int64_t *ncoo);
int vec_destroy(gbs_vec V);

/*
 * Device-side COO generation for the model problems: Sec. 3's pattern of a
 * user Jacobian kernel that fills the COO values on the device and hands
 * them to MatSetValuesCOO, with Sec. 5's per-element offsets (64 e for a Q1
 * hexahedron, 4 e for a graph edge).  All pointers are device pointers; the
 * calls are asynchronous on `stream`; errors: GBS_ERR_ARG (sizes, null or
 * misaligned pointers), GBS_ERR_CUDA.
 *
 * q1_hex_element_coo: the COO indices of ne^3 Q1 hexahedra of the unit cube
 *   (ne >= 1, 64 ne^3 < 2^31): entry 64 e + 8 a + b is (g(e, a), g(e, b)),
 *   node g = ix + (ne+1) (iy + (ne+1) iz), element e = ex + ne (ey + ne ez),
 *   local node a = ax + 2 ay + 4 az.  i, j: int32[64 ne^3], 16-byte aligned.
 * q1_hex_element_values: the matching values v[64 e + 8 a + b] =
 *   (kappa[e] h) K_ref[a][b], h = 1/ne, K_ref the Q1 reference stiffness
 *   (1/3 on the diagonal, 0 for nodes differing in one coordinate, -1/12 in
 *   two or three), each product rounded once after kappa[e] h; Dirichlet on
 *   the outer faces keeping every row: an off-diagonal entry touching a
 *   boundary node is 0 and a boundary node's diagonal entry is 1/m (m = 1,
 *   2, 4 elements at a corner, edge, face node), so its assembled diagonal
 *   is 1.  kappa: double[ne^3] (8-byte aligned); v: double[64 ne^3]
 *   (16-byte aligned).
 * edge_coo_values: the values of a variable-coefficient graph Laplacian
 *   given as 4 COO entries per edge, (a, a), (b, b), (a, b), (b, a): v[4 e ..
 *   4 e + 3] = (+kappa[e], +kappa[e], -kappa[e], -kappa[e]).  nedges in
 *   [0, 2^29); kappa: double[nedges]; v: double[4 nedges] (16-byte aligned).
 *   The indices (with -1 for a Dirichlet ghost) are the caller's.
 */
int q1_hex_element_coo(int32_t ne, int32_t *i, int32_t *j, void *stream);
int q1_hex_element_values(int32_t ne, const double *kappa, double *v, void *stream);
int edge_coo_values(int64_t nedges, const double *kappa, double *v, void *stream);

/* Number of kernels this library has launched in this process (a diagnostic
 * counter).  A solve graph counts its setup and closing kernels at launch and
 * its loop kernels (three per trip) when the solve's results are read. */
int64_t gbs_launch_count(void);

/* Thread-local message describing the last error ("" if none). */
const char *gbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GBS_H */
