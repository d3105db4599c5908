/*
 * Plain, slow, obviously-correct FP64 CPU oracle for the sparse SPD solver path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The product path never calls it,
 * and it shares no code, header, table or constant with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -std=c11 -fPIC -shared oracle.c -lm
 * (-ffp-contract=off matters: a fused multiply-add would change the rounding
 *  of every product-then-sum below, and gcc fuses by default on aarch64.)
 *
 * Functions and the passages they follow (paper: PETSc/TAO developments for
 * GPU-based early exascale systems):
 *   orc_coo_symbolic / orc_coo_numeric  -- Sec. 5, the COO definition: the
 *       assembled A is the sum of the contributions v[k] to a_{i[k],j[k]};
 *       negative indices mean "ignore this entry"; MatSetPreallocationCOO fixes
 *       the pattern, MatSetValuesCOO(v, mode) fills values.
 *   orc_spmv           -- the MatMult of Sec. 6.1: y = A x on CSR.
 *   orc_pcg            -- the KSP CG of Sec. 6.1 with the diagonal (Jacobi)
 *       preconditioner the batched solvers of Sec. 7 use; textbook
 *       Hestenes-Stiefel preconditioned CG (the paper relies on PETSc's CG and
 *       does not restate it).
 *   orc_pcg_refined    -- the single-precision inner solve under a double
 *       precision outer solve motivated in Sec. 2 (multiprecision, A7):
 *       FP32 PCG inside FP64 iterative refinement.
 *   orc_adjoint_*      -- the adjoint capability mentioned in Sec. 1, for a
 *       linear solve: A^T lambda = g, dL/da_ij = -lambda_i x_j, dL/db = lambda.
 *   orc_pcg_batched    -- Sec. 7: many independent systems, each solved on its
 *       own (per-system scalars and convergence).
 *   orc_bicg / orc_tfqmr / orc_krylov_batched -- Sec. 7's batched solvers
 *       for nonsymmetric systems (BiCG and TFQMR with the diagonal
 *       preconditioner), one system at a time.
 *   orc_pipecg         -- a CG whose iteration needs one global reduction,
 *       for the latency-bound (small-NNZ) regime where Sec. 6.2's
 *       asynchronous solvers gain most: the preconditioned pipelined CG of
 *       Ghysels and Vanroose (Parallel Computing 40, 2014), Jacobi
 *       preconditioner.  In exact arithmetic its iterates are PCG's.
 *   orc_pcg_sr         -- the same Jacobi-PCG in Chronopoulos and Gear's
 *       single-reduction form (J. Comput. Appl. Math. 25, 1989): PCG's
 *       iterates in exact arithmetic with the two inner products of an
 *       iteration taken in one reduction after the product -- the form the
 *       GPU's two-kernel CG iteration follows (Sec. 6.1's CG with the
 *       scalars kept on the device).
 *   orc_vec_set_values_coo -- Sec. 5's COO interface for vectors
 *       (VecSetPreallocationCOO / VecSetValuesCOO): y_r is the sum of the
 *       contributions v[k] with i[k] = r.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_*.py against
 * dense brute force, closed forms (Laplacian eigenpairs, the Q1 stencil),
 * finite differences and invariants; see those tests for the list.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Built twice: as it stands (one thread), and with -fopenmp for the timed
 * all-cores baseline, where ORC_PAR splits the row loops of the SpMV, the
 * numeric COO stage and the FP64 PCG's element-wise updates across threads.
 * Every split loop writes each element from one iteration alone, and the
 * inner products stay sequential, so both builds give the same bits. */
#ifdef _OPENMP
#define ORC_PAR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PAR
#endif

/* status codes (numerically the same values the public C-ABI documents) */
enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_INDEX = 2,
  ORC_ERR_ALLOC = 3,
  ORC_ERR_NOT_SPD = 5,
  ORC_ERR_BREAKDOWN = 6,
  ORC_ERR_NAN = 7,
  ORC_ERR_MAXIT = 8,
  ORC_ERR_STAGNATION = 9
};

typedef struct {
  int32_t status, iterations, outer_iterations, pad;
  double rnorm0, rnorm, true_rel_residual;
} orc_result;

/* ------------------------------------------------------------------------ */
/* O1: COO -> CSR, symbolic                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t i, j;
  int64_t k;
} orc_trip;

static int cmp_trip(const void *pa, const void *pb) {
  const orc_trip *a = (const orc_trip *)pa, *b = (const orc_trip *)pb;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->k != b->k) return a->k < b->k ? -1 : 1; /* keeps the sort stable */
  return 0;
}

/*
 * Kept set K = {k : i[k] >= 0 and j[k] >= 0}.  A kept index outside
 * [0,nrows) x [0,ncols) is an error.  The pattern is the set of distinct (i,j)
 * over K, rows ascending and columns strictly ascending within a row.
 * Outputs (caller-allocated):
 *   row_ptr[nrows+1], col[>= nnz], perm[>= nkept] (sorted position -> original
 *   COO index k), jmap[>= nnz+1] (segment p of the sorted kept entries is
 *   [jmap[p], jmap[p+1]) ).
 * Returns nnz >= 0, or -status on error.
 */
int64_t orc_coo_symbolic(int64_t nrows, int64_t ncols, int64_t ncoo,
                         const int32_t *ci, const int32_t *cj, int32_t *row_ptr,
                         int32_t *col, int32_t *perm, int32_t *jmap,
                         int64_t *nkept_out) {
  if (nrows < 0 || ncols < 0 || ncoo < 0) return -ORC_ERR_ARG;
  int64_t nkept = 0;
  for (int64_t k = 0; k < ncoo; ++k) {
    if (ci[k] < 0 || cj[k] < 0) continue;
    if ((int64_t)ci[k] >= nrows || (int64_t)cj[k] >= ncols) return -ORC_ERR_INDEX;
    ++nkept;
  }
  orc_trip *t = (orc_trip *)malloc((size_t)(nkept > 0 ? nkept : 1) * sizeof(orc_trip));
  if (!t) return -ORC_ERR_ALLOC;
  int64_t m = 0;
  for (int64_t k = 0; k < ncoo; ++k) {
    if (ci[k] < 0 || cj[k] < 0) continue;
    t[m].i = ci[k];
    t[m].j = cj[k];
    t[m].k = k;
    ++m;
  }
  qsort(t, (size_t)nkept, sizeof(orc_trip), cmp_trip);

  for (int64_t r = 0; r <= nrows; ++r) row_ptr[r] = 0;
  int64_t nnz = 0;
  for (int64_t s = 0; s < nkept; ++s) {
    int head = (s == 0) || t[s].i != t[s - 1].i || t[s].j != t[s - 1].j;
    if (head) {
      col[nnz] = t[s].j;
      jmap[nnz] = (int32_t)s;
      row_ptr[t[s].i + 1] += 1; /* count of pattern entries in row i */
      ++nnz;
    }
    perm[s] = (int32_t)t[s].k;
  }
  jmap[nnz] = (int32_t)nkept;
  for (int64_t r = 0; r < nrows; ++r) row_ptr[r + 1] += row_ptr[r];
  free(t);
  if (nkept_out) *nkept_out = nkept;
  return nnz;
}

/* ------------------------------------------------------------------------ */
/* O1: COO -> CSR, numeric                                                   */
/* ------------------------------------------------------------------------ */

/*
 * a_p = left fold of v over the segment's original indices, in increasing k,
 * starting from the first term (so a lone -0.0 stays -0.0).
 * mode 0 = INSERT (a_p replaces), mode 1 = ADD (a_p is added to val[p]).
 */
void orc_coo_numeric(int64_t nnz, const int32_t *jmap, const int32_t *perm,
                     const double *v, int mode, double *val) {
  ORC_PAR
  for (int64_t p = 0; p < nnz; ++p) {
    double s = v[perm[jmap[p]]];
    for (int64_t t = (int64_t)jmap[p] + 1; t < jmap[p + 1]; ++t) s = s + v[perm[t]];
    val[p] = (mode == 1) ? val[p] + s : s;
  }
}

/* dL/dv_k = dL/da_{p(k)} for kept k, 0 for ignored k (transpose of the above) */
void orc_coo_scatter(int64_t nnz, int64_t ncoo, const int32_t *jmap,
                     const int32_t *perm, const double *dlda, double *dldv) {
  for (int64_t k = 0; k < ncoo; ++k) dldv[k] = 0.0;
  for (int64_t p = 0; p < nnz; ++p)
    for (int64_t t = jmap[p]; t < jmap[p + 1]; ++t) dldv[perm[t]] = dlda[p];
}

/*
 * Vector COO assembly, straight from the definition: for every index r that
 * appears among the kept entries (i[k] >= 0), acc_r is the left fold of its
 * v[k] in increasing k starting from the first term; INSERT (mode 0) sets
 * y[r] = acc_r, ADD (mode 1) sets y[r] = y[r] + acc_r; indices that do not
 * appear leave y[r] unchanged.  An index >= n is an error (-ORC_ERR_INDEX).
 * Returns the number of distinct indices.
 */
int64_t orc_vec_set_values_coo(int64_t n, int64_t ncoo, const int32_t *ci, const double *v,
                               int mode, double *y) {
  for (int64_t k = 0; k < ncoo; ++k)
    if (ci[k] >= 0 && (int64_t)ci[k] >= n) return -ORC_ERR_INDEX;
  double *acc = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  unsigned char *seen = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!acc || !seen) {
    free(acc);
    free(seen);
    return -ORC_ERR_ALLOC;
  }
  int64_t distinct = 0;
  for (int64_t k = 0; k < ncoo; ++k) {
    if (ci[k] < 0) continue;
    const int64_t r = ci[k];
    if (!seen[r]) {
      seen[r] = 1;
      acc[r] = v[k];
      ++distinct;
    } else {
      acc[r] = acc[r] + v[k];
    }
  }
  for (int64_t r = 0; r < n; ++r)
    if (seen[r]) y[r] = (mode == 1) ? y[r] + acc[r] : acc[r];
  free(acc);
  free(seen);
  return distinct;
}

/* ------------------------------------------------------------------------ */
/* O2: SpMV                                                                  */
/* ------------------------------------------------------------------------ */

void orc_spmv(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
              const double *x, double *y) {
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += a[p] * x[ci[p]];
    y[i] = s;
  }
}

static void spmv32(int64_t n, const int32_t *rp, const int32_t *ci,
                   const float *a, const float *x, float *y) {
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += a[p] * x[ci[p]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double *x, const double *y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

/* FP32 inner product with FP32 accumulation, summed pairwise: halves of
 * n > 8 terms are summed recursively and added, runs of at most 8 terms left
 * to right.  Each product and each addition is rounded to FP32.  (Summed left
 * to right, the rounding error of n FP32 terms grows like n eps -- about 5%
 * for the million-row systems here -- and slows the inner solve for reasons
 * of order alone; pairwise it grows like eps log2 n, as any tree reduction's
 * does.) */
static float dot32(int64_t n, const float *x, const float *y) {
  if (n <= 8) {
    float s = 0.0f;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
  }
  const int64_t h = n / 2;
  return dot32(h, x, y) + dot32(n - h, x + h, y + h);
}

/* Jacobi: dinv_i = 1/a_ii; missing or non-positive diagonal is an error. */
static int jacobi(int64_t n, const int32_t *rp, const int32_t *ci,
                  const double *a, double *dinv) {
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    int found = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) {
        d = a[p];
        found = 1;
      }
    if (!found || !(d > 0.0)) return ORC_ERR_NOT_SPD;
    dinv[i] = 1.0 / d;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O3: Jacobi-preconditioned CG                                              */
/* ------------------------------------------------------------------------ */

static double true_rel(int64_t n, const int32_t *rp, const int32_t *ci,
                       const double *a, const double *b, const double *x,
                       double bnorm, double *work) {
  orc_spmv(n, rp, ci, a, x, work);
  for (int64_t i = 0; i < n; ++i) work[i] = b[i] - work[i];
  double rn = sqrt(dot(n, work, work));
  return bnorm > 0.0 ? rn / bnorm : rn;
}

/*
 * Solve A x = b.  x holds the initial guess when nonzero_guess, else starts at
 * 0.  Stops when ||r||_2 <= rtol ||b||_2 (r the recursively updated residual),
 * checked before every product q = A p; iterations = number of such products.
 */
int orc_pcg(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
            const double *b, double *x, double rtol, int64_t maxit,
            int nonzero_guess, orc_result *res) {
  memset(res, 0, sizeof(*res));
  double *dinv = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double) * 5);
  if (!dinv) return res->status = ORC_ERR_ALLOC;
  double *r = dinv + n, *z = r + n, *p = z + n, *q = p + n;
  int st = jacobi(n, rp, ci, a, dinv);
  if (st != ORC_OK) {
    free(dinv);
    return res->status = st;
  }
  if (!nonzero_guess)
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  double bnorm = sqrt(dot(n, b, b));
  if (!isfinite(bnorm)) {
    free(dinv);
    return res->status = ORC_ERR_NAN;
  }
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    free(dinv);
    return res->status = ORC_OK;
  }
  orc_spmv(n, rp, ci, a, x, r);
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
  ORC_PAR
  for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  double rho = dot(n, r, z);
  double rr = dot(n, r, r);
  res->rnorm0 = sqrt(rr);
  int64_t it = 0;
  st = ORC_OK;
  for (;;) {
    double rnorm = sqrt(rr);
    res->rnorm = rnorm;
    if (!isfinite(rnorm) || !isfinite(rho)) {
      st = ORC_ERR_NAN;
      break;
    }
    if (rnorm <= rtol * bnorm) break;
    if (it >= maxit) {
      st = ORC_ERR_MAXIT;
      break;
    }
    orc_spmv(n, rp, ci, a, p, q);
    double sigma = dot(n, p, q);
    ++it;
    if (isnan(sigma)) {
      st = ORC_ERR_NAN;
      break;
    }
    if (!(sigma > 0.0)) {
      st = ORC_ERR_BREAKDOWN;
      break;
    }
    double alpha = rho / sigma;
    ORC_PAR
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
    ORC_PAR
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    ORC_PAR
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    double rho_new = dot(n, r, z);
    rr = dot(n, r, r);
    double beta = rho_new / rho;
    ORC_PAR
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
  res->iterations = (int32_t)it;
  res->true_rel_residual = true_rel(n, rp, ci, a, b, x, bnorm, q);
  free(dinv);
  return res->status = st;
}

/* ------------------------------------------------------------------------ */
/* O4: FP32 inner PCG inside FP64 iterative refinement                       */
/* ------------------------------------------------------------------------ */

/*
 * Outer (FP64): r = b - A64 x; stop when ||r|| <= rtol ||b||; s = ||r||.
 * Inner (FP32 values, vectors and accumulation, inner products summed
 * pairwise, see dot32): Jacobi-PCG on A32 d = RN(r/s)
 * from d = 0 until ||r_in|| <= tgt ||r_in,0|| with tgt = max(inner_rtol,
 * rtol ||b|| / (2 s)) (the last correction only has to close the remaining
 * gap), inner_maxit products, or a non-positive / non-finite sigma.  Update
 * x += s * d in FP64.
 * Stagnation: ||r|| fails to halve on two consecutive outer steps.
 * A32 = RN(A64) elementwise; dinv32 = RN(1/a_ii) with the reciprocal in FP64.
 * inner_its (max_outer entries, or NULL) receives each outer step's inner
 * iteration count.
 */
int orc_pcg_refined(int64_t n, const int32_t *rp, const int32_t *ci,
                    const double *a, const double *b, double *x, double rtol,
                    double inner_rtol, int64_t inner_maxit, int32_t max_outer,
                    int nonzero_guess, orc_result *res, int32_t *inner_its) {
  memset(res, 0, sizeof(*res));
  int64_t nnz = rp[n];
  double *dinv = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double) * 2);
  float *f = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float) * 6 +
                             (size_t)(nnz > 0 ? nnz : 1) * sizeof(float));
  if (!dinv || !f) {
    free(dinv);
    free(f);
    return res->status = ORC_ERR_ALLOC;
  }
  double *r = dinv + n;
  float *dinv32 = f, *r32 = f + n, *z32 = r32 + n, *p32 = z32 + n, *q32 = p32 + n,
        *d32 = q32 + n, *a32 = d32 + n;
  int st = jacobi(n, rp, ci, a, dinv);
  if (st != ORC_OK) goto done;
  for (int64_t i = 0; i < n; ++i) dinv32[i] = (float)dinv[i];
  for (int64_t p = 0; p < nnz; ++p) a32[p] = (float)a[p];
  if (!nonzero_guess)
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  double bnorm = sqrt(dot(n, b, b));
  if (!isfinite(bnorm)) {
    st = ORC_ERR_NAN;
    goto done;
  }
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  double prev = INFINITY;
  int stall = 0;
  int32_t outer = 0;
  int64_t inner_total = 0;
  for (;;) {
    orc_spmv(n, rp, ci, a, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rn = sqrt(dot(n, r, r));
    if (outer == 0) res->rnorm0 = rn;
    res->rnorm = rn;
    if (!isfinite(rn)) {
      st = ORC_ERR_NAN;
      break;
    }
    if (rn <= rtol * bnorm) break;
    if (outer >= max_outer) {
      st = ORC_ERR_MAXIT;
      break;
    }
    if (outer > 0) {
      stall = (rn > 0.5 * prev) ? stall + 1 : 0;
      if (stall >= 2) {
        st = ORC_ERR_STAGNATION;
        break;
      }
    }
    prev = rn;
    double s = rn;
    /* inner target: inner_rtol, or the smaller reduction that already brings
       the outer residual to half of rtol ||b|| */
    const double tgt = fmax(inner_rtol, 0.5 * rtol * bnorm / s);
    for (int64_t i = 0; i < n; ++i) r32[i] = (float)(r[i] / s);
    /* inner FP32 Jacobi-PCG from d = 0 */
    for (int64_t i = 0; i < n; ++i) d32[i] = 0.0f;
    for (int64_t i = 0; i < n; ++i) z32[i] = dinv32[i] * r32[i];
    for (int64_t i = 0; i < n; ++i) p32[i] = z32[i];
    float rho = dot32(n, r32, z32);
    float rr = dot32(n, r32, r32);
    const double thr = tgt * (double)sqrtf(rr);
    int64_t it = 0;
    for (;;) {
      if (!((double)sqrtf(rr) > thr)) break; /* also ends on NaN */
      if (it >= inner_maxit) break;
      spmv32(n, rp, ci, a32, p32, q32);
      float sigma = dot32(n, p32, q32);
      if (!(sigma > 0.0f)) break;
      ++it;
      float alpha = rho / sigma;
      for (int64_t i = 0; i < n; ++i) d32[i] += alpha * p32[i];
      for (int64_t i = 0; i < n; ++i) r32[i] -= alpha * q32[i];
      for (int64_t i = 0; i < n; ++i) z32[i] = dinv32[i] * r32[i];
      float rho_new = dot32(n, r32, z32);
      rr = dot32(n, r32, r32);
      float beta = rho_new / rho;
      for (int64_t i = 0; i < n; ++i) p32[i] = z32[i] + beta * p32[i];
      rho = rho_new;
    }
    if (it == 0) {
      st = ORC_ERR_BREAKDOWN;
      break;
    }
    inner_total += it;
    if (inner_its) inner_its[outer] = (int32_t)it;
    for (int64_t i = 0; i < n; ++i) x[i] += s * (double)d32[i];
    ++outer;
  }
  res->iterations = (int32_t)inner_total;
  res->outer_iterations = outer;
  res->true_rel_residual = true_rel(n, rp, ci, a, b, x, bnorm, r);
done:
  free(dinv);
  free(f);
  return res->status = st;
}

/* ------------------------------------------------------------------------ */
/* Nonsymmetric solvers with the diagonal preconditioner (Sec. 7)            */
/* ------------------------------------------------------------------------ */

/* y = A^T x: y_j = sum_i a_ij x_i, each sum in increasing i. */
static void spmv_t(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                   const double *x, double *y) {
  for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) y[ci[p]] = y[ci[p]] + a[p] * x[i];
}

static int start_residual(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                          const double *b, double *x, int nonzero_guess, double *r,
                          double *bnorm, orc_result *res) {
  if (!nonzero_guess)
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  orc_spmv(n, rp, ci, a, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  *bnorm = sqrt(dot(n, b, b));
  res->rnorm0 = res->rnorm = sqrt(dot(n, r, r));
  if (!isfinite(*bnorm)) return ORC_ERR_NAN;
  return ORC_OK;
}

/*
 * Preconditioned BiCG with M = diag(A) (applied to both sequences, M^T = M)
 * and shadow residual rt_0 = r_0:
 *   z = M^-1 r, zt = M^-1 rt, rho = z.rt; p = z + beta p, pt = zt + beta pt
 *   (beta = rho / rho_prev; p = z, pt = zt first); q = A p, qt = A^T pt;
 *   alpha = rho / (pt.q); x += alpha p; r -= alpha q; rt -= alpha qt.
 * Stops when ||r|| <= rtol ||b|| (checked before each iteration);
 * iterations counts the products q = A p.  rho = 0 or pt.q = 0: BREAKDOWN.
 * For symmetric A, rt stays equal to r and the iteration is PCG's, operation
 * for operation.
 */
int orc_bicg(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
             const double *b, double *x, double rtol, int64_t maxit, int nonzero_guess,
             orc_result *res) {
  memset(res, 0, sizeof(*res));
  double *w = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double) * 9);
  if (!w) return res->status = ORC_ERR_ALLOC;
  double *dinv = w, *r = w + n, *rt = r + n, *z = rt + n, *zt = z + n, *p = zt + n,
         *pt = p + n, *q = pt + n, *qt = q + n;
  double bnorm = 0.0;
  int st = jacobi(n, rp, ci, a, dinv);
  if (st == ORC_OK) st = start_residual(n, rp, ci, a, b, x, nonzero_guess, r, &bnorm, res);
  if (st == ORC_OK && bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    res->rnorm0 = res->rnorm = 0.0;
  } else if (st == ORC_OK) {
    for (int64_t i = 0; i < n; ++i) rt[i] = r[i];
    double rho_prev = 0.0;
    int64_t it = 0;
    for (;;) {
      const double rn = sqrt(dot(n, r, r));
      res->rnorm = rn;
      if (!isfinite(rn)) {
        st = ORC_ERR_NAN;
        break;
      }
      if (rn <= rtol * bnorm) break;
      if (it >= maxit) {
        st = ORC_ERR_MAXIT;
        break;
      }
      for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
      for (int64_t i = 0; i < n; ++i) zt[i] = dinv[i] * rt[i];
      const double rho = dot(n, z, rt);
      if (rho == 0.0) {
        st = ORC_ERR_BREAKDOWN;
        break;
      }
      if (it == 0) {
        for (int64_t i = 0; i < n; ++i) p[i] = z[i];
        for (int64_t i = 0; i < n; ++i) pt[i] = zt[i];
      } else {
        const double beta = rho / rho_prev;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        for (int64_t i = 0; i < n; ++i) pt[i] = zt[i] + beta * pt[i];
      }
      orc_spmv(n, rp, ci, a, p, q);
      spmv_t(n, rp, ci, a, pt, qt);
      ++it;
      const double sigma = dot(n, pt, q);
      if (isnan(sigma)) {
        st = ORC_ERR_NAN;
        break;
      }
      if (sigma == 0.0) {
        st = ORC_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rho / sigma;
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
      for (int64_t i = 0; i < n; ++i) rt[i] = rt[i] - alpha * qt[i];
      rho_prev = rho;
    }
    res->iterations = (int32_t)it;
  }
  if (st == ORC_OK || st == ORC_ERR_MAXIT || st == ORC_ERR_BREAKDOWN || st == ORC_ERR_NAN)
    res->true_rel_residual = true_rel(n, rp, ci, a, b, x, bnorm, q);
  free(w);
  return res->status = st;
}

/*
 * TFQMR (Freund's transpose-free QMR) on the right-preconditioned system
 * A M^-1 u = b, x = M^-1 u, M = diag(A), so that its quasi-residual bound
 * refers to the true residual b - A x.  With B = A M^-1 and rt = r_0:
 *   w = y1 = r_0; v = B y1; d = 0; tau = ||r_0||; theta = eta = 0;
 *   rho = rt.r_0.  Each step: alpha = rho / (rt.v); y2 = y1 - alpha v;
 *   then two half steps with (y, By) = (y1, B y1) and (y2, B y2):
 *     w -= alpha By; d = y + (theta^2 eta / alpha) d; theta = ||w|| / tau;
 *     c = 1 / sqrt(1 + theta^2); tau = tau theta c; eta = c^2 alpha;
 *     x += eta M^-1 d;  stop when tau sqrt(m + 1) <= rtol ||b||
 *     (m = half steps taken, counting from 1);
 *   rho_new = rt.w; beta = rho_new / rho; y1 = w + beta y2;
 *   v = B y1 + beta (B y2 + beta v).
 * iterations counts the products with B; rnorm reports the bound at exit.
 * rt.v = 0 or rho = 0: BREAKDOWN.
 */
int orc_tfqmr(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
              const double *b, double *x, double rtol, int64_t maxit, int nonzero_guess,
              orc_result *res) {
  memset(res, 0, sizeof(*res));
  double *wk = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double) * 11);
  if (!wk) return res->status = ORC_ERR_ALLOC;
  double *dinv = wk, *r = wk + n, *rt = r + n, *w = rt + n, *y1 = w + n, *y2 = y1 + n,
         *v = y2 + n, *by1 = v + n, *by2 = by1 + n, *d = by2 + n, *t = d + n;
  double bnorm = 0.0;
  int st = jacobi(n, rp, ci, a, dinv);
  if (st == ORC_OK) st = start_residual(n, rp, ci, a, b, x, nonzero_guess, r, &bnorm, res);
  /* B y = A (M^-1 y) */
#define ORC_BMUL(yv, out)                                              \
  do {                                                                 \
    for (int64_t i_ = 0; i_ < n; ++i_) t[i_] = dinv[i_] * (yv)[i_];    \
    orc_spmv(n, rp, ci, a, t, (out));                                  \
  } while (0)
  if (st == ORC_OK && bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    res->rnorm0 = res->rnorm = 0.0;
  } else if (st == ORC_OK && res->rnorm0 <= rtol * bnorm) {
    /* already converged */
  } else if (st == ORC_OK) {
    for (int64_t i = 0; i < n; ++i) {
      rt[i] = r[i];
      w[i] = r[i];
      y1[i] = r[i];
      d[i] = 0.0;
    }
    ORC_BMUL(y1, by1);
    for (int64_t i = 0; i < n; ++i) v[i] = by1[i];
    int64_t it = 1, m = 0;
    double tau = res->rnorm0, theta = 0.0, eta = 0.0;
    double rho = dot(n, rt, r);
    for (;;) {
      if (!isfinite(tau) || !isfinite(rho)) {
        st = ORC_ERR_NAN;
        break;
      }
      const double sigma = dot(n, rt, v);
      if (sigma == 0.0 || rho == 0.0) {
        st = ORC_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rho / sigma;
      for (int64_t i = 0; i < n; ++i) y2[i] = y1[i] - alpha * v[i];
      ORC_BMUL(y2, by2);
      ++it;
      int done = 0;
      for (int half = 0; half < 2 && !done; ++half) {
        const double *yh = half == 0 ? y1 : y2;
        const double *byh = half == 0 ? by1 : by2;
        const double coef = theta * theta * eta / alpha;
        for (int64_t i = 0; i < n; ++i) w[i] = w[i] - alpha * byh[i];
        for (int64_t i = 0; i < n; ++i) d[i] = yh[i] + coef * d[i];
        theta = sqrt(dot(n, w, w)) / tau;
        const double c = 1.0 / sqrt(1.0 + theta * theta);
        tau = tau * theta * c;
        eta = c * c * alpha;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + eta * (dinv[i] * d[i]);
        ++m;
        res->rnorm = tau * sqrt((double)(m + 1));
        if (!isfinite(res->rnorm)) {
          st = ORC_ERR_NAN;
          done = 1;
        } else if (res->rnorm <= rtol * bnorm) {
          done = 1;
        }
      }
      if (done) break;
      if (it >= maxit) {
        st = ORC_ERR_MAXIT;
        break;
      }
      const double rho_new = dot(n, rt, w);
      const double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t i = 0; i < n; ++i) y1[i] = w[i] + beta * y2[i];
      ORC_BMUL(y1, by1);
      ++it;
      for (int64_t i = 0; i < n; ++i) v[i] = by1[i] + beta * (by2[i] + beta * v[i]);
    }
    res->iterations = (int32_t)it;
  }
#undef ORC_BMUL
  if (st == ORC_OK || st == ORC_ERR_MAXIT || st == ORC_ERR_BREAKDOWN || st == ORC_ERR_NAN)
    res->true_rel_residual = true_rel(n, rp, ci, a, b, x, bnorm, t);
  free(wk);
  return res->status = st;
}

/*
 * Pipelined PCG (Ghysels-Vanroose), M = diag(A).  Alongside x and r it keeps
 * u = M^-1 r, w = A u, p, s = A p, q = M^-1 s, z = A q by recurrences, so
 * that one iteration needs one reduction and one product:
 *   r = b - A x0; u = M^-1 r; w = A u;
 *   for i = 0, 1, ...:
 *     gamma = r.u; delta = w.u; rr = r.r   (the one reduction)
 *     stop if sqrt(rr) <= rtol ||b|| (iterations = i), or i >= maxit (MAXIT)
 *     m = M^-1 w; n = A m                  (the one product)
 *     beta = 0 and alpha = gamma / delta at i = 0, else
 *     beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
 *     z = n + beta z; q = m + beta q; s = w + beta s; p = u + beta p
 *     x += alpha p; r -= alpha s; u -= alpha q; w -= alpha z.
 * The recurrences let the recursive r drift from b - A x (more than CG's
 * do), so a recursive residual that meets the test is confirmed with the
 * true one, r = b - A x: if that misses the test too, the recurrences
 * restart from x (u = M^-1 r, w = A u, p = s = q = z = 0, the next
 * iteration with beta = 0); outer_iterations counts the restarts, and
 * iterations (the x updates) keeps counting across them.
 * A non-positive gamma or alpha denominator: BREAKDOWN.  rnorm reports the
 * last ||r|| (at a normal exit the confirmed true residual).  aux (7 n
 * doubles, or NULL) receives r, u, w, p, s, q, z at exit, for checking the
 * recurrences' invariants.
 */
int orc_pipecg(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
               const double *b, double *x, double rtol, int64_t maxit, int nonzero_guess,
               orc_result *res, double *aux) {
  memset(res, 0, sizeof(*res));
  double *wk = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double) * 10);
  if (!wk) return res->status = ORC_ERR_ALLOC;
  double *dinv = wk, *r = wk + n, *u = r + n, *w = u + n, *m = w + n, *nv = m + n,
         *p = nv + n, *s = p + n, *q = s + n, *z = q + n;
  double bnorm = 0.0;
  int st = jacobi(n, rp, ci, a, dinv);
  if (st == ORC_OK) st = start_residual(n, rp, ci, a, b, x, nonzero_guess, r, &bnorm, res);
  if (st == ORC_OK && bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    res->rnorm0 = res->rnorm = 0.0;
  } else if (st == ORC_OK) {
    for (int64_t i = 0; i < n; ++i) u[i] = dinv[i] * r[i];
    orc_spmv(n, rp, ci, a, u, w);
    for (int64_t i = 0; i < n; ++i) p[i] = s[i] = q[i] = z[i] = 0.0;
    double gamma_prev = 0.0, alpha_prev = 0.0;
    int64_t it = 0, restarts = 0;
    int fresh = 1; /* the next iteration starts the recurrences: beta = 0 */
    for (;;) {
      const double gamma = dot(n, r, u);
      const double delta = dot(n, w, u);
      const double rn = sqrt(dot(n, r, r));
      res->rnorm = rn;
      if (!isfinite(rn) || !isfinite(gamma) || !isfinite(delta)) {
        st = ORC_ERR_NAN;
        break;
      }
      if (rn <= rtol * bnorm) {
        /* confirm with the true residual (m as scratch) */
        orc_spmv(n, rp, ci, a, x, m);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - m[i];
        const double tn = sqrt(dot(n, r, r));
        res->rnorm = tn;
        if (!isfinite(tn)) {
          st = ORC_ERR_NAN;
          break;
        }
        if (tn <= rtol * bnorm) break;
        /* restart the recurrences from x */
        ++restarts;
        for (int64_t i = 0; i < n; ++i) u[i] = dinv[i] * r[i];
        orc_spmv(n, rp, ci, a, u, w);
        for (int64_t i = 0; i < n; ++i) p[i] = s[i] = q[i] = z[i] = 0.0;
        fresh = 1;
        continue;
      }
      if (it >= maxit) {
        st = ORC_ERR_MAXIT;
        break;
      }
      for (int64_t i = 0; i < n; ++i) m[i] = dinv[i] * w[i];
      orc_spmv(n, rp, ci, a, m, nv);
      double beta = 0.0, den = delta;
      if (!fresh) {
        beta = gamma / gamma_prev;
        den = delta - beta * gamma / alpha_prev;
      }
      if (!(gamma > 0.0) || !(den > 0.0)) {
        st = ORC_ERR_BREAKDOWN;
        break;
      }
      const double alpha = gamma / den;
      for (int64_t i = 0; i < n; ++i) z[i] = nv[i] + beta * z[i];
      for (int64_t i = 0; i < n; ++i) q[i] = m[i] + beta * q[i];
      for (int64_t i = 0; i < n; ++i) s[i] = w[i] + beta * s[i];
      for (int64_t i = 0; i < n; ++i) p[i] = u[i] + beta * p[i];
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * s[i];
      for (int64_t i = 0; i < n; ++i) u[i] = u[i] - alpha * q[i];
      for (int64_t i = 0; i < n; ++i) w[i] = w[i] - alpha * z[i];
      gamma_prev = gamma;
      alpha_prev = alpha;
      fresh = 0;
      ++it;
    }
    res->iterations = (int32_t)it;
    res->outer_iterations = (int32_t)restarts;
  }
  if (aux && n > 0) {
    const double *src[7] = {r, u, w, p, s, q, z};
    for (int k = 0; k < 7; ++k) memcpy(aux + (size_t)k * (size_t)n, src[k], sizeof(double) * (size_t)n);
  }
  if (st == ORC_OK || st == ORC_ERR_MAXIT || st == ORC_ERR_BREAKDOWN || st == ORC_ERR_NAN)
    res->true_rel_residual = true_rel(n, rp, ci, a, b, x, bnorm, m);
  free(wk);
  return res->status = st;
}

/*
 * Single-reduction Jacobi-PCG: Chronopoulos and Gear's reformulation of CG
 * (J. Comput. Appl. Math. 25, 1989), in its preconditioned form.  The same
 * iterates as PCG in exact arithmetic; the two inner products of an
 * iteration are taken together, right after the product w = A u:
 *   r = b - A x0, u = M^-1 r; then per iteration
 *     w = A u; gamma = r.u, delta = w.u, ||r||^2 (one reduction);
 *     stop if ||r|| <= rtol ||b||;
 *     beta = gamma / gamma_prev (0 on the first iteration);
 *     den = delta - beta gamma / alpha_prev (= p.Ap; delta on the first);
 *     alpha = gamma / den;
 *     p = u + beta p, s = w + beta s (s = A p by recurrence);
 *     x += alpha p, r -= alpha s, u = M^-1 r.
 * M = diag(A).  Stops when ||r||_2 <= rtol ||b||_2 (the recursively updated
 * r, tested before each update); iterations counts the x updates (= PCG's
 * count).  A missing or non-positive diagonal: NOT_SPD; gamma <= 0 or
 * den <= 0: BREAKDOWN; a non-finite norm or product: NAN.  aux (5 n doubles
 * or NULL) receives r, u, w, p, s at exit, for checking the invariants
 * u = M^-1 r, w = A u, s = A p, r = b - A x.
 */
int orc_pcg_sr(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
               const double *b, double *x, double rtol, int64_t maxit, int nonzero_guess,
               orc_result *res, double *aux) {
  memset(res, 0, sizeof(*res));
  double *wk = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double) * 6);
  if (!wk) return res->status = ORC_ERR_ALLOC;
  double *dinv = wk, *r = wk + n, *u = r + n, *w = u + n, *p = w + n, *s = p + n;
  double bnorm = 0.0;
  int st = jacobi(n, rp, ci, a, dinv);
  if (st == ORC_OK) st = start_residual(n, rp, ci, a, b, x, nonzero_guess, r, &bnorm, res);
  for (int64_t i = 0; i < n; ++i) u[i] = w[i] = p[i] = s[i] = 0.0;
  if (st == ORC_OK && bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    res->rnorm0 = res->rnorm = 0.0;
  } else if (st == ORC_OK) {
    for (int64_t i = 0; i < n; ++i) u[i] = dinv[i] * r[i];
    double gamma_prev = 0.0, alpha_prev = 0.0;
    int64_t it = 0;
    for (;;) {
      orc_spmv(n, rp, ci, a, u, w);
      const double gamma = dot(n, r, u);
      const double delta = dot(n, w, u);
      const double rn = sqrt(dot(n, r, r));
      res->rnorm = rn;
      if (!isfinite(rn) || !isfinite(gamma) || !isfinite(delta)) {
        st = ORC_ERR_NAN;
        break;
      }
      if (rn <= rtol * bnorm) break;
      if (it >= maxit) {
        st = ORC_ERR_MAXIT;
        break;
      }
      double beta = 0.0, den = delta;
      if (it > 0) {
        beta = gamma / gamma_prev;
        den = delta - beta * gamma / alpha_prev;
      }
      if (!(gamma > 0.0) || !(den > 0.0)) {
        st = ORC_ERR_BREAKDOWN;
        break;
      }
      const double alpha = gamma / den;
      for (int64_t i = 0; i < n; ++i) p[i] = u[i] + beta * p[i];
      for (int64_t i = 0; i < n; ++i) s[i] = w[i] + beta * s[i];
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
      for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * s[i];
      for (int64_t i = 0; i < n; ++i) u[i] = dinv[i] * r[i];
      gamma_prev = gamma;
      alpha_prev = alpha;
      ++it;
    }
    res->iterations = (int32_t)it;
  }
  if (aux && n > 0) {
    const double *src[5] = {r, u, w, p, s};
    for (int k = 0; k < 5; ++k) memcpy(aux + (size_t)k * (size_t)n, src[k], sizeof(double) * (size_t)n);
  }
  if (st == ORC_OK || st == ORC_ERR_MAXIT || st == ORC_ERR_BREAKDOWN || st == ORC_ERR_NAN)
    res->true_rel_residual = true_rel(n, rp, ci, a, b, x, bnorm, w);
  free(wk);
  return res->status = st;
}

/* Batched solves, each system alone: method 1 = BiCG, 2 = TFQMR, 3 =
 * pipelined CG, 4 = single-reduction CG. */
int orc_krylov_batched(int32_t nsys, const int64_t *row_off, const int32_t *rp,
                       const int32_t *ci, const double *a, const double *b, double *x,
                       double rtol, int64_t maxit, int method, orc_result *res) {
  int first = ORC_OK;
  for (int32_t s = 0; s < nsys; ++s) {
    int64_t r0 = row_off[s], r1 = row_off[s + 1], n = r1 - r0;
    int64_t base = rp[r0], nz = (int64_t)rp[r1] - base;
    int32_t *lrp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *lci = (int32_t *)malloc((size_t)(nz > 0 ? nz : 1) * sizeof(int32_t));
    if (!lrp || !lci) {
      free(lrp);
      free(lci);
      return ORC_ERR_ALLOC;
    }
    for (int64_t i = 0; i <= n; ++i) lrp[i] = (int32_t)(rp[r0 + i] - base);
    for (int64_t p = 0; p < nz; ++p) lci[p] = (int32_t)(ci[base + p] - r0);
    const int st =
        method == 1   ? orc_bicg(n, lrp, lci, a + base, b + r0, x + r0, rtol, maxit, 0, &res[s])
        : method == 2 ? orc_tfqmr(n, lrp, lci, a + base, b + r0, x + r0, rtol, maxit, 0, &res[s])
        : method == 3 ? orc_pipecg(n, lrp, lci, a + base, b + r0, x + r0, rtol, maxit, 0,
                                   &res[s], NULL)
                      : orc_pcg_sr(n, lrp, lci, a + base, b + r0, x + r0, rtol, maxit, 0,
                                   &res[s], NULL);
    if (st != ORC_OK && first == ORC_OK) first = st;
    free(lrp);
    free(lci);
  }
  return first;
}

/* ------------------------------------------------------------------------ */
/* O5: adjoint of x = A^{-1} b                                               */
/* ------------------------------------------------------------------------ */

/* 1 if the CSR matrix equals its transpose exactly (pattern and values). */
int orc_csr_is_symmetric(int64_t n, const int32_t *rp, const int32_t *ci,
                         const double *a) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      int found = 0;
      for (int64_t t = rp[j]; t < rp[j + 1]; ++t)
        if (ci[t] == i) {
          found = (a[t] == a[p]);
          break;
        }
      if (!found) return 0;
    }
  return 1;
}

/*
 * Given x = A^{-1} b and g = dL/dx: solve A^T lambda = g (A symmetric, so the
 * same PCG), then dL/db = lambda and dL/da_p = -lambda_{row p} x_{col p}.
 * dlda may be NULL.
 */
int orc_adjoint(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                const double *x, const double *g, double *lambda, double *dlda,
                double rtol, int64_t maxit, orc_result *res) {
  if (!orc_csr_is_symmetric(n, rp, ci, a)) {
    memset(res, 0, sizeof(*res));
    return res->status = ORC_ERR_ARG;
  }
  int st = orc_pcg(n, rp, ci, a, g, lambda, rtol, maxit, 0, res);
  if (dlda)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) dlda[p] = -lambda[i] * x[ci[p]];
  return st;
}

/* ------------------------------------------------------------------------ */
/* O6: batched                                                               */
/* ------------------------------------------------------------------------ */

/*
 * Block-diagonal CSR (global row/column numbering); system s owns rows
 * [row_off[s], row_off[s+1]) and only couples to its own columns.  Each system
 * is solved independently by orc_pcg (precision 0) or orc_pcg_refined
 * (precision 1), with its own stopping test ||r_s|| <= rtol ||b_s||.
 * res has nsys entries.  Returns the first non-OK status, else OK.
 */
int orc_pcg_batched(int32_t nsys, const int64_t *row_off, const int32_t *rp,
                    const int32_t *ci, const double *a, const double *b,
                    double *x, double rtol, int64_t maxit, int precision,
                    double inner_rtol, int64_t inner_maxit, int32_t max_outer,
                    orc_result *res) {
  int first = ORC_OK;
  for (int32_t s = 0; s < nsys; ++s) {
    int64_t r0 = row_off[s], r1 = row_off[s + 1], n = r1 - r0;
    int64_t base = rp[r0], nz = (int64_t)rp[r1] - base;
    int32_t *lrp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *lci = (int32_t *)malloc((size_t)(nz > 0 ? nz : 1) * sizeof(int32_t));
    if (!lrp || !lci) {
      free(lrp);
      free(lci);
      return ORC_ERR_ALLOC;
    }
    for (int64_t i = 0; i <= n; ++i) lrp[i] = (int32_t)(rp[r0 + i] - base);
    for (int64_t p = 0; p < nz; ++p) lci[p] = (int32_t)(ci[base + p] - r0);
    int st;
    if (precision == 0)
      st = orc_pcg(n, lrp, lci, a + base, b + r0, x + r0, rtol, maxit, 0, &res[s]);
    else
      st = orc_pcg_refined(n, lrp, lci, a + base, b + r0, x + r0, rtol, inner_rtol,
                           inner_maxit, max_outer, 0, &res[s], NULL);
    if (st != ORC_OK && first == ORC_OK) first = st;
    free(lrp);
    free(lci);
  }
  return first;
}
