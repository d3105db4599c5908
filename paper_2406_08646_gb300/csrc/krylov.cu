// Nonsymmetric batched Krylov solvers (Sec. 7: PETSc's batched solvers are
// TFQMR and BiCG with diagonal preconditioning), one CTA per system.
//
// Both methods run FP64 and keep every iteration of a system inside one CTA of
// one kernel launch, like the per-CTA PCG (cta.cuh): CTA barriers only, block
// reductions in a fixed tree whose totals reach every thread, and scalar
// recurrences that every thread evaluates identically from those totals, so
// all control flow is uniform across the CTA without extra broadcasts.
//
//   BiCG (Jacobi on both sequences, rt0 = r0): per iteration the p/pt update,
//   the products q = A p (fused with pt.q) and qt = A^T pt, and the x/r/rt
//   update fused with ||r||^2 and (D^-1 r).rt.  A^T is a second sliced-ELL
//   copy made from the transpose of the COO pattern by the library's own
//   symbolic stage (deterministic, bit-exact), kept as an internal handle.
//
//   TFQMR (Freund 1993, right-preconditioned: B = A D^-1): per step two
//   products with B over t = D^-1 y, each fused with the elementwise work
//   that follows it, three reductions.  The x update of each half step is
//   deferred into the next pass over the rows (it only needs that half
//   step's eta and d), and applied at exit when the loop ends on a half step.
//
// The same two methods also run on the grid-wide phase kernels (the CG
// driver's block tables, last-arriver reductions and graph WHILE loop): for
// one large system, and for the stacked "ensemble" of Sec. 7 that a standard
// solver would see.  BiCG: setup, WHILE { products and pt.q; updates with
// ||r||^2 and (D^-1 r).rt; directions }, closing residual.  TFQMR: setup,
// WHILE { B y1 with rt.v; half step 1; B y2 fused with half step 2; y1 and
// the x update }, the x update left pending by a half step that ended the
// solve, closing residual.
//
// The oracle counts, statuses and tests are followed exactly; only the
// summation order of the dot products differs (a fixed tree here).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cta.cuh"
#include "device_util.cuh"
#include "internal.cuh"
#include "phases.cuh"

namespace gbs {

struct KrylovArgs {
  int32_t ensemble;                        // 1: one CTA over the whole matrix
  int32_t nrows, nslices;                  // whole matrix (ensemble)
  const int32_t *order;                    // system of each CTA, largest first
  const int32_t *sys_row0, *sys_slice0;    // nsys + 1
  SellView sv;                             // sliced-ELL copy of A
  const double *sval;
  SellView tv;                             // sliced-ELL copy of A^T (same slices)
  const double *tval;
  int32_t stream_matrix;                   // evict-first loads of the copies
  const double *dinv;
  double *v[KRYLOV_NVEC];
  SysState *st;
  DevCtl *ctl;
  const CallArgs *call;
};

struct KSys {
  int s, r0, r1, s0, s1;
};

__device__ __forceinline__ KSys kry_system(const KrylovArgs &a) {
  KSys g;
  if (a.ensemble) {
    g.s = 0;
    g.r0 = 0;
    g.r1 = a.nrows;
    g.s0 = 0;
    g.s1 = a.nslices;
  } else {
    g.s = __ldg(a.order + blockIdx.x);
    g.r0 = __ldg(a.sys_row0 + g.s);
    g.r1 = __ldg(a.sys_row0 + g.s + 1);
    g.s0 = __ldg(a.sys_slice0 + g.s);
    g.s1 = __ldg(a.sys_slice0 + g.s + 1);
  }
  return g;
}

// Row products of the system with one of the two sliced copies; x may have
// been written by this CTA, so its gathers take the coherent path.
template <class F>
__device__ __forceinline__ void kry_rows(const KrylovArgs &a, const KSys &g, const SellView &S,
                                         const double *sval, const double *x, F &f) {
  if (a.stream_matrix) sell_rows<double, true, GATHER_CA>(S, sval, x, g.s0, g.s1, f);
  else sell_rows<double, false, GATHER_CA>(S, sval, x, g.s0, g.s1, f);
}

// The system's closing state (thread 0), x = 0 where b = 0, then
// ||b - A x||^2 into S.tt.
__device__ void kry_close(const KrylovArgs &a, const KSys &g, CtaShared &sh, int status,
                          bool timed_out, int iterations, double bb, double rnorm0,
                          double rnorm, bool zero_x) {
  SysState &S = a.st[g.s];
  double *x = a.call->x;
  if (zero_x)
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) x[r] = 0.0;
  __syncthreads();  // x complete
  if (threadIdx.x == 0) {
    memset(&S, 0, sizeof(SysState));
    S.bb = bb;
    S.rnorm0 = rnorm0;
    S.rnorm = rnorm;
    S.iterations = iterations;
    S.status = timed_out ? GBS_OK : status;
    S.active = timed_out ? 1 : 0;  // reported as the control word's error
    if (timed_out) a.ctl->err = GBS_ERR_TIMEOUT;
  }
  const double *b = a.call->b;
  double tt[1] = {0.0};
  auto f = [&](int r, double t) {
    const double d = b[r] - t;
    tt[0] = fma(d, d, tt[0]);
  };
  kry_rows(a, g, a.sv, a.sval, x, f);
  cta_sum0<double, 1>(tt, sh);
  if (threadIdx.x == 0) S.tt = tt[0];
}

// Start-up checks shared by both methods: a missing or non-positive diagonal
// (NOT_SPD, the Jacobi preconditioner's requirement), b not finite (NAN), or
// b = 0 (x = 0, OK).  Returns the status, or -1 to iterate.
__device__ __forceinline__ int kry_start_status(double missing, double bb) {
  if (missing > 0.0) return GBS_ERR_NOT_SPD;
  if (!isfinite(bb)) return GBS_ERR_NAN;
  if (bb == 0.0) return GBS_OK;
  return -1;
}

// The scalar recurrences run in thread 0 (FP64 scalar work in every warp
// would cost 32 times the FP64 issue slots, see cta.cuh); after each block
// sum thread 0 publishes the next pass's coefficients and whether to go on
// (sh.ipub[0] < 0), and every thread reads them after one barrier.

// ------------------------------------------------------------------ BiCG
__device__ void kry_bicg(const KrylovArgs &a, const KSys &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  const double *dinv = a.dinv;
  double *r = a.v[0], *rt = a.v[1], *p = a.v[2], *pt = a.v[3], *q = a.v[4], *qt = a.v[5];
  const bool t0 = threadIdx.x == 0;
  // r0 = b - A x0, rt0 = r0; sums r.r, b.b, (D^-1 r).rt, missing diagonals
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  auto start = [&](int i, double ax) {
    const double bv = b[i], rv = bv - ax, dv = dinv[i];
    r[i] = rv;
    rt[i] = rv;
    v[0] = fma(rv, rv, v[0]);
    v[1] = fma(bv, bv, v[1]);
    v[2] = fma(dv * rv, rv, v[2]);
    v[3] += (dv == 0.0) ? 1.0 : 0.0;
  };
  if (C.nonzero_guess) {
    kry_rows(a, g, a.sv, a.sval, x, start);
  } else {
    for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x) {
      x[i] = 0.0;
      start(i, 0.0);
    }
  }
  cta_sum0<double, 4>(v, sh);
  // thread 0's scalars
  double bb = 0.0, thr = 0.0, rn = 0.0, rnorm0 = 0.0, rho = 0.0, rho_prev = 0.0;
  int status = -1, it = 0;
  bool timed = false;
  // the tests before an iteration; publishes beta (ipub[1]: first iteration)
  auto top = [&]() {
    if (!isfinite(rn)) status = GBS_ERR_NAN;
    else if (rn <= thr) status = GBS_OK;
    else if (it >= C.maxit) status = GBS_ERR_MAXIT;
    else if (rho == 0.0) status = GBS_ERR_BREAKDOWN;
    else if (it > 0 && cta_timed_out(a.ctl, C.timeout_ns)) timed = true;
    else sh.pub[0] = it == 0 ? 0.0 : rho / rho_prev;
    sh.ipub[0] = (status < 0 && !timed) ? -1 : 0;
    sh.ipub[1] = it == 0;
  };
  if (t0) {
    bb = v[1];
    thr = C.rtol * sqrt(bb);
    rn = rnorm0 = sqrt(v[0]);
    rho = v[2];
    status = kry_start_status(v[3], bb);
    sh.ipub[2] = status == GBS_OK;  // b = 0: x = 0
    if (status == GBS_OK) rn = rnorm0 = 0.0;
    if (status < 0) top();
    else sh.ipub[0] = 0;
  }
  cta_publish();
  const bool zero_x = sh.ipub[2] != 0;
  while (sh.ipub[0] < 0) {
    // p = z + beta p, pt = zt + beta pt (z = D^-1 r, zt = D^-1 rt)
    const double beta = sh.pub[0];
    const bool first = sh.ipub[1] != 0;
    for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x) {
      const double dv = dinv[i], z = dv * r[i], zt = dv * rt[i];
      p[i] = first ? z : fma(beta, p[i], z);
      pt[i] = first ? zt : fma(beta, pt[i], zt);
    }
    __syncthreads();
    // q = A p with pt.q, qt = A^T pt
    double sg[1] = {0.0};
    auto fq = [&](int i, double y) {
      q[i] = y;
      sg[0] = fma(pt[i], y, sg[0]);
    };
    kry_rows(a, g, a.sv, a.sval, p, fq);
    auto fqt = [&](int i, double y) { qt[i] = y; };
    kry_rows(a, g, a.tv, a.tval, pt, fqt);
    cta_sum0<double, 1>(sg, sh);
    if (t0) {
      ++it;
      if (isnan(sg[0])) status = GBS_ERR_NAN;
      else if (sg[0] == 0.0) status = GBS_ERR_BREAKDOWN;
      else sh.pub[1] = rho / sg[0];
      sh.ipub[0] = status;
    }
    cta_publish();
    if (sh.ipub[0] >= 0) break;
    const double alpha = sh.pub[1];
    // x += alpha p, r -= alpha q, rt -= alpha qt; ||r||^2, (D^-1 r).rt
    double u[2] = {0.0, 0.0};
    for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x) {
      x[i] = fma(alpha, p[i], x[i]);
      const double rv = fma(-alpha, q[i], r[i]);
      const double rtv = fma(-alpha, qt[i], rt[i]);
      r[i] = rv;
      rt[i] = rtv;
      u[0] = fma(rv, rv, u[0]);
      u[1] = fma(dinv[i] * rv, rtv, u[1]);
    }
    cta_sum0<double, 2>(u, sh);
    if (t0) {
      rn = sqrt(u[0]);
      rho_prev = rho;
      rho = u[1];
      top();
    }
    cta_publish();
  }
  kry_close(a, g, sh, status, timed, it, bb, rnorm0, rn, zero_x);
}

// ------------------------------------------------------------------ TFQMR
__device__ void kry_tfqmr(const KrylovArgs &a, const KSys &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  const double *dinv = a.dinv;
  double *w = a.v[0], *y1 = a.v[1], *y2 = a.v[2], *rt = a.v[3], *vv = a.v[4], *by1 = a.v[5],
         *by2 = a.v[6], *d = a.v[7], *t = a.v[8];
  const bool t0 = threadIdx.x == 0;
  // r0 = b - A x0 into w, y1 and rt; d = 0; t = D^-1 y1; sums r.r, b.b,
  // missing diagonals
  double v[3] = {0.0, 0.0, 0.0};
  auto start = [&](int i, double ax) {
    const double bv = b[i], rv = bv - ax, dv = dinv[i];
    w[i] = rv;
    y1[i] = rv;
    rt[i] = rv;
    d[i] = 0.0;
    t[i] = dv * rv;
    v[0] = fma(rv, rv, v[0]);
    v[1] = fma(bv, bv, v[1]);
    v[2] += (dv == 0.0) ? 1.0 : 0.0;
  };
  if (C.nonzero_guess) {
    kry_rows(a, g, a.sv, a.sval, x, start);
  } else {
    for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x) {
      x[i] = 0.0;
      start(i, 0.0);
    }
  }
  cta_sum0<double, 3>(v, sh);
  // thread 0's scalars
  double bb = 0.0, thr = 0.0, rnorm0 = 0.0, rn = 0.0;
  double rho = 0.0, tau = 0.0, theta = 0.0, eta = 0.0, alpha = 0.0;
  int status = -1, it = 0, m = 0;
  bool timed = false;
  if (t0) {
    bb = v[1];
    thr = C.rtol * sqrt(bb);
    rn = rnorm0 = sqrt(v[0]);
    status = kry_start_status(v[2], bb);
    sh.ipub[2] = status == GBS_OK;  // b = 0: x = 0
    if (status == GBS_OK) rn = rnorm0 = 0.0;
    else if (status < 0 && rnorm0 <= thr) status = GBS_OK;  // x0 already meets the test
    rho = v[0];  // rt.r0 = ||r0||^2
    tau = rnorm0;
    sh.ipub[0] = status;
  }
  cta_publish();
  const bool zero_x = sh.ipub[2] != 0;
  // one half step's scalars from ||w||^2 and its tests (thread 0); returns
  // whether the solve ends here
  auto half = [&](double ww) {
    theta = sqrt(ww) / tau;
    const double c = 1.0 / sqrt(1.0 + theta * theta);
    tau = tau * theta * c;
    eta = c * c * alpha;
    ++m;
    rn = tau * sqrt((double)(m + 1));
    if (!isfinite(rn)) status = GBS_ERR_NAN;
    else if (rn <= thr) status = GBS_OK;
    return status >= 0;
  };
  // the tests at the top of a step from sigma = rt.v; publishes alpha and the
  // first half step's d coefficient
  auto top = [&](double sigma) {
    if (!isfinite(tau) || !isfinite(rho)) status = GBS_ERR_NAN;
    else if (sigma == 0.0 || rho == 0.0) status = GBS_ERR_BREAKDOWN;
    else {
      alpha = rho / sigma;
      ++it;  // the product B y2 of this step
      sh.pub[0] = alpha;
      sh.pub[1] = theta * theta * eta / alpha;
    }
    sh.ipub[0] = status;
  };
  bool pend = false;  // a half step's x update (x += eta D^-1 d) not applied yet
  if (sh.ipub[0] < 0) {
    // v = B y1 (= A t), rt.v
    double sg[1] = {0.0};
    auto f0 = [&](int i, double y) {
      by1[i] = y;
      vv[i] = y;
      sg[0] = fma(rt[i], y, sg[0]);
    };
    kry_rows(a, g, a.sv, a.sval, t, f0);
    cta_sum0<double, 1>(sg, sh);
    if (t0) {
      it = 1;
      top(sg[0]);
    }
    cta_publish();
    while (sh.ipub[0] < 0) {
      const double al = sh.pub[0], coef1 = sh.pub[1];
      // half step 1 with (y1, B y1); y2 = y1 - alpha v, t = D^-1 y2
      double s1[1] = {0.0};
      for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x) {
        const double y1i = y1[i];
        const double y2i = y1i - al * vv[i];
        y2[i] = y2i;
        t[i] = dinv[i] * y2i;
        const double wn = w[i] - al * by1[i];
        w[i] = wn;
        d[i] = y1i + coef1 * d[i];
        s1[0] = fma(wn, wn, s1[0]);
      }
      cta_sum0<double, 1>(s1, sh);
      if (t0) {
        const bool done = half(s1[0]);
        sh.pub[2] = eta;
        sh.pub[3] = theta * theta * eta / alpha;
        sh.ipub[0] = done ? 0 : -1;
      }
      cta_publish();
      pend = true;
      if (sh.ipub[0] >= 0) break;
      // B y2 (= A t) fused with half step 1's x update and half step 2
      const double e1 = sh.pub[2], coef2 = sh.pub[3];
      double s2[2] = {0.0, 0.0};
      auto f1 = [&](int i, double y) {
        by2[i] = y;
        const double di = d[i];
        x[i] = fma(e1, dinv[i] * di, x[i]);
        d[i] = y2[i] + coef2 * di;
        const double wn = w[i] - al * y;
        w[i] = wn;
        s2[0] = fma(wn, wn, s2[0]);
        s2[1] = fma(rt[i], wn, s2[1]);
      };
      kry_rows(a, g, a.sv, a.sval, t, f1);
      cta_sum0<double, 2>(s2, sh);
      if (t0) {
        bool stop = half(s2[0]);
        if (!stop && it >= C.maxit) {
          status = GBS_ERR_MAXIT;
          stop = true;
        }
        if (!stop && cta_timed_out(a.ctl, C.timeout_ns)) {
          timed = true;
          stop = true;
        }
        sh.pub[2] = eta;
        if (!stop) {
          sh.pub[3] = s2[1] / rho;  // beta
          rho = s2[1];
        }
        sh.ipub[0] = stop ? 0 : -1;
      }
      cta_publish();
      if (sh.ipub[0] >= 0) break;
      // y1 = w + beta y2, t = D^-1 y1, half step 2's x update
      const double e2 = sh.pub[2], beta = sh.pub[3];
      for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x) {
        const double dv = dinv[i];
        const double y = w[i] + beta * y2[i];
        y1[i] = y;
        t[i] = dv * y;
        x[i] = fma(e2, dv * d[i], x[i]);
      }
      pend = false;
      __syncthreads();
      // B y1 (= A t), v = B y1 + beta (B y2 + beta v), rt.v
      double s3[1] = {0.0};
      auto f2 = [&](int i, double y) {
        by1[i] = y;
        const double vn = y + beta * (by2[i] + beta * vv[i]);
        vv[i] = vn;
        s3[0] = fma(rt[i], vn, s3[0]);
      };
      kry_rows(a, g, a.sv, a.sval, t, f2);
      cta_sum0<double, 1>(s3, sh);
      if (t0) {
        ++it;  // B y1
        top(s3[0]);
      }
      cta_publish();
    }
  }
  if (pend) {  // the last half step's x update (eta published with it)
    const double e = sh.pub[2];
    for (int i = g.r0 + threadIdx.x; i < g.r1; i += blockDim.x)
      x[i] = fma(e, dinv[i] * d[i], x[i]);
  }
  kry_close(a, g, sh, status, timed, it, bb, rnorm0, rn, zero_x);
}

// MINB CTAs per SM: 1 keeps every value in registers (64 per thread); 2 (32
// registers, a few hundred bytes of spills) keeps two systems in flight per
// SM, which a batch of at least two systems per SM repays (about 1.4x the
// solves per second on 1024 convection-diffusion systems).
template <int METHOD, int MINB>
__global__ void __launch_bounds__(CTA_TPB, MINB) k_cta_krylov(KrylovArgs a) {
  __shared__ CtaShared sh;
  const KSys g = kry_system(a);
  if (METHOD == GBS_KSP_BICG) kry_bicg(a, g, sh);
  else kry_tfqmr(a, g, sh);
}

// ------------------------------------------------------------------ phases
//
// Grid-wide versions: every kernel walks a block table, so one system spans
// the whole GPU; per-system scalars live in SysState and are finished by the
// last CTA to reduce (phases.cuh).  Row products use the sliced copies (the
// block tables carry slice offsets whatever the plan's kernel).

struct NsView {
  double alpha, beta, eta, coef;
  int first;
};
__device__ __forceinline__ NsView ns_view(const PcgArgs &a, int s) {
  const SysState *S = a.st + s;
  return NsView{ld_state(&S->alpha), ld_state(&S->beta), ld_state(&S->eta),
                ld_state(&S->coef), ld_state(&S->first)};
}

// Row products of block b with A^T's sliced copy.
template <class F>
__device__ __forceinline__ void rows_t(const PcgArgs &a, int b, const double *x, F &f) {
  const int s0 = __ldg(a.ta.slice0 + b), s1 = blk_slice_end(a.ta, b);
  if (a.stream_matrix)
    sell_rows<double, true, GATHER_NC>(a.tv, a.tval, x, s0, s1, f);
  else sell_rows<double, false, GATHER_NC>(a.tv, a.tval, x, s0, s1, f);
}

__device__ __forceinline__ void ns_activate(const PcgArgs &a, SysState &S, int status) {
  if (status >= 0) {
    S.status = status;
    S.active = 0;
  } else {
    S.status = GBS_OK;
    S.active = 1;
    atomicAdd(&a.ctl->n_active, 1);
  }
}

// BiCG's tests before an iteration: NAN, converged, limit, rho = 0.
__device__ __forceinline__ int bicg_top(const CallArgs &C, const SysState &S) {
  if (!isfinite(S.rnorm)) return GBS_ERR_NAN;
  if (S.rnorm <= S.thr) return GBS_OK;
  if (S.iterations >= C.maxit) return GBS_ERR_MAXIT;
  if (S.rho == 0.0) return GBS_ERR_BREAKDOWN;
  return -1;
}

// r = b - A x0, rt = r, p = pt = D^-1 r; r.r, b.b, (D^-1 r).rt, missing
// diagonals; fin: start-up and pre-iteration tests.  Table A.
__device__ __forceinline__ void bicg_setup(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  double *r = a.kv[0], *rt = a.kv[1], *p = a.kv[2], *pt = a.kv[3];
  auto want = [&](int) -> int { return 1; };
  auto row = [&](int i, double ax, double(&acc)[4]) {
    const double bv = b[i], rv = bv - ax, dv = a.dinv[i], z = dv * rv;
    r[i] = rv;
    rt[i] = rv;
    p[i] = z;
    pt[i] = z;
    acc[0] = fma(rv, rv, acc[0]);
    acc[1] = fma(bv, bv, acc[1]);
    acc[2] = fma(z, rv, acc[2]);
    acc[3] += (dv == 0.0) ? 1.0 : 0.0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[4]) {
    if (C.nonzero_guess) {
      auto f = [&](int i, double ax) { row(i, ax, acc); };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, x, f);
    } else {
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        x[i] = 0.0;
        row(i, 0.0, acc);
      }
    }
  };
  auto fin = [&](int s, double(&tot)[4]) {
    SysState &S = a.st[s];
    memset(&S, 0, sizeof(SysState));
    S.bb = tot[1];
    set_thr(S, C.rtol * sqrt(S.bb));
    S.rr = tot[0];
    S.rho = tot[2];
    S.rnorm0 = S.rnorm = sqrt(tot[0]);
    int st = kry_start_status(tot[3], tot[1]);
    if (st == GBS_OK) {
      S.zero_x = 1;
      S.rnorm0 = S.rnorm = 0.0;
    } else if (st < 0) {
      st = bicg_top(C, S);
    }
    ns_activate(a, S, st);
  };
  walk<4>(a, a.ta, 0, red, want, work, fin);
}

// q = A p with pt.q, qt = A^T pt; fin: alpha.  Table A.
__device__ __forceinline__ void bicg_products(const PcgArgs &a, double *red) {
  const double *p = a.kv[2], *pt = a.kv[3];
  double *q = a.kv[4], *qt = a.kv[5];
  auto want = [&](int s) -> int { return sys_active(a, s) ? 1 : 0; };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[1]) {
    double sg = acc[0];
    auto fq = [&](int i, double y) {
      q[i] = y;
      sg = fma(__ldg(pt + i), y, sg);
    };
    row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, p, fq);
    auto fqt = [&](int i, double y) { qt[i] = y; };
    rows_t(a, blk, pt, fqt);
    acc[0] = sg;
  };
  auto fin = [&](int s, double(&tot)[1]) {
    SysState &S = a.st[s];
    S.iterations += 1;
    if (isnan(tot[0])) deactivate(a, S, GBS_ERR_NAN);
    else if (tot[0] == 0.0) deactivate(a, S, GBS_ERR_BREAKDOWN);
    else S.alpha = S.rho / tot[0];
  };
  walk<1>(a, a.ta, 0, red, want, work, fin);
}

// x += alpha p, r -= alpha q, rt -= alpha qt; ||r||^2, (D^-1 r).rt; fin:
// the tests of the next iteration, beta.  Table E.
__device__ __forceinline__ void bicg_update(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  double *x = C.x;
  double *r = a.kv[0], *rt = a.kv[1];
  const double *p = a.kv[2], *q = a.kv[4], *qt = a.kv[5];
  NsView v{};
  auto want = [&](int s) -> int {
    v = ns_view(a, s);  // issued with the active flag: one round trip
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int, int r0, int r1, double(&acc)[2]) {
    const double al = v.alpha;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      x[i] = fma(al, p[i], x[i]);
      const double rv = fma(-al, q[i], r[i]);
      const double rtv = fma(-al, qt[i], rt[i]);
      r[i] = rv;
      rt[i] = rtv;
      acc[0] = fma(rv, rv, acc[0]);
      acc[1] = fma(a.dinv[i] * rv, rtv, acc[1]);
    }
  };
  auto fin = [&](int s, double(&tot)[2]) {
    SysState &S = a.st[s];
    const double beta = tot[1] / S.rho;
    S.rr = tot[0];
    S.rnorm = sqrt(tot[0]);
    S.rho = tot[1];
    const int st = bicg_top(C, S);
    if (st >= 0) deactivate(a, S, st);
    else S.beta = beta;
  };
  walk<2>(a, a.te, a.part_e, red, want, work, fin);
}

// p = D^-1 r + beta p, pt = D^-1 rt + beta pt.  Table E.
__device__ __forceinline__ void bicg_direction(const PcgArgs &a, double *red) {
  const double *r = a.kv[0], *rt = a.kv[1];
  double *p = a.kv[2], *pt = a.kv[3];
  NsView v{};
  auto want = [&](int s) -> int {
    v = ns_view(a, s);  // issued with the active flag: one round trip
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int, int r0, int r1, double(&)[1]) {
    const double be = v.beta;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double dv = a.dinv[i];
      p[i] = fma(be, p[i], dv * r[i]);
      pt[i] = fma(be, pt[i], dv * rt[i]);
    }
  };
  auto fin = [&](int, double(&)[1]) {};
  walk<0>(a, a.te, a.part_e, red, want, work, fin);
}

// One TFQMR half step's scalars from ||w||^2: theta, c, tau, eta, m; returns
// the bound tau sqrt(m + 1).
__device__ __forceinline__ double tfq_half(SysState &S, double ww) {
  S.theta = sqrt(ww) / S.tau;
  const double c = 1.0 / sqrt(1.0 + S.theta * S.theta);
  S.tau = S.tau * S.theta * c;
  S.eta = c * c * S.alpha;
  S.m += 1;
  return S.tau * sqrt((double)(S.m + 1));
}

// r0 = b - A x0 into w, y1, rt; d = 0; t = D^-1 r0; r.r, b.b, missing
// diagonals; fin: start-up tests.  Table A.
__device__ __forceinline__ void tfq_setup(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  double *w = a.kv[0], *y1 = a.kv[1], *rt = a.kv[3], *d = a.kv[7], *t = a.kv[8];
  auto want = [&](int) -> int { return 1; };
  auto row = [&](int i, double ax, double(&acc)[3]) {
    const double bv = b[i], rv = bv - ax, dv = a.dinv[i];
    w[i] = rv;
    y1[i] = rv;
    rt[i] = rv;
    d[i] = 0.0;
    t[i] = dv * rv;
    acc[0] = fma(rv, rv, acc[0]);
    acc[1] = fma(bv, bv, acc[1]);
    acc[2] += (dv == 0.0) ? 1.0 : 0.0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[3]) {
    if (C.nonzero_guess) {
      auto f = [&](int i, double ax) { row(i, ax, acc); };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, x, f);
    } else {
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        x[i] = 0.0;
        row(i, 0.0, acc);
      }
    }
  };
  auto fin = [&](int s, double(&tot)[3]) {
    SysState &S = a.st[s];
    memset(&S, 0, sizeof(SysState));
    S.bb = tot[1];
    set_thr(S, C.rtol * sqrt(S.bb));
    S.rr = tot[0];
    S.rnorm0 = S.rnorm = sqrt(tot[0]);
    int st = kry_start_status(tot[2], tot[1]);
    if (st == GBS_OK) {
      S.zero_x = 1;
      S.rnorm0 = S.rnorm = 0.0;
    } else if (st < 0 && S.rnorm0 <= S.thr) {
      st = GBS_OK;  // x0 already meets the test
    }
    S.rho = tot[0];  // rt.r0 = ||r0||^2
    S.tau = S.rnorm0;
    S.first = 1;
    ns_activate(a, S, st);
  };
  walk<3>(a, a.ta, 0, red, want, work, fin);
}

// B y1 (= A t), v = B y1 (+ beta (B y2 + beta v) after the first step), rt.v;
// fin: the tests at the top of a step, alpha.  Table A.
__device__ __forceinline__ void tfq_v(const PcgArgs &a, double *red) {
  const double *rt = a.kv[3], *by2 = a.kv[6], *t = a.kv[8];
  double *vv = a.kv[4], *by1 = a.kv[5];
  NsView v{};
  auto want = [&](int s) -> int {
    v = ns_view(a, s);  // issued with the active flag: one round trip
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[1]) {
    const double be = v.beta;
    const bool first = v.first != 0;
    double sg = acc[0];
    auto f = [&](int i, double y) {
      by1[i] = y;
      const double vn = first ? y : y + be * (by2[i] + be * vv[i]);
      vv[i] = vn;
      sg = fma(rt[i], vn, sg);
    };
    row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, t, f);
    acc[0] = sg;
  };
  auto fin = [&](int s, double(&tot)[1]) {
    SysState &S = a.st[s];
    S.iterations += 1;
    S.first = 0;
    S.pend = 0;  // the last step's x update has been applied
    if (!isfinite(S.tau) || !isfinite(S.rho)) deactivate(a, S, GBS_ERR_NAN);
    else if (tot[0] == 0.0 || S.rho == 0.0) deactivate(a, S, GBS_ERR_BREAKDOWN);
    else {
      S.alpha = S.rho / tot[0];
      S.coef = S.theta * S.theta * S.eta / S.alpha;
    }
  };
  walk<1>(a, a.ta, 0, red, want, work, fin);
}

// Half step 1: y2 = y1 - alpha v, t = D^-1 y2, w -= alpha B y1,
// d = y1 + coef d; ||w||^2; fin: its scalars and tests.  Table E.
__device__ __forceinline__ void tfq_half1(const PcgArgs &a, double *red) {
  const double *y1 = a.kv[1], *vv = a.kv[4], *by1 = a.kv[5];
  double *w = a.kv[0], *y2 = a.kv[2], *d = a.kv[7], *t = a.kv[8];
  NsView v{};
  auto want = [&](int s) -> int {
    v = ns_view(a, s);  // issued with the active flag: one round trip
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int, int r0, int r1, double(&acc)[1]) {
    const double al = v.alpha, cf = v.coef;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double y1i = y1[i];
      const double y2i = y1i - al * vv[i];
      y2[i] = y2i;
      t[i] = a.dinv[i] * y2i;
      const double wn = w[i] - al * by1[i];
      w[i] = wn;
      d[i] = y1i + cf * d[i];
      acc[0] = fma(wn, wn, acc[0]);
    }
  };
  auto fin = [&](int s, double(&tot)[1]) {
    SysState &S = a.st[s];
    S.iterations += 1;  // the product B y2 of this step
    const double rn = tfq_half(S, tot[0]);
    S.rnorm = rn;
    S.pend = 1;
    if (!isfinite(rn)) deactivate(a, S, GBS_ERR_NAN);
    else if (rn <= S.thr) deactivate(a, S, GBS_OK);
    else S.coef = S.theta * S.theta * S.eta / S.alpha;
  };
  walk<1>(a, a.te, a.part_e, red, want, work, fin);
}

// B y2 (= A t) fused with half step 1's x update and half step 2:
// x += eta D^-1 d, d = y2 + coef d, w -= alpha B y2; ||w||^2, rt.w; fin:
// its scalars, tests and beta.  Table A.
__device__ __forceinline__ void tfq_half2(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  double *x = C.x;
  const double *y2 = a.kv[2], *rt = a.kv[3], *t = a.kv[8];
  double *w = a.kv[0], *by2 = a.kv[6], *d = a.kv[7];
  NsView v{};
  auto want = [&](int s) -> int {
    v = ns_view(a, s);  // issued with the active flag: one round trip
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[2]) {
    const double al = v.alpha, e1 = v.eta, cf = v.coef;
    double a0 = acc[0], a1 = acc[1];
    auto f = [&](int i, double y) {
      by2[i] = y;
      const double di = d[i];
      x[i] = fma(e1, a.dinv[i] * di, x[i]);
      d[i] = y2[i] + cf * di;
      const double wn = w[i] - al * y;
      w[i] = wn;
      a0 = fma(wn, wn, a0);
      a1 = fma(rt[i], wn, a1);
    };
    row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, t, f);
    acc[0] = a0;
    acc[1] = a1;
  };
  auto fin = [&](int s, double(&tot)[2]) {
    SysState &S = a.st[s];
    const double rn = tfq_half(S, tot[0]);
    S.rnorm = rn;
    if (!isfinite(rn)) deactivate(a, S, GBS_ERR_NAN);
    else if (rn <= S.thr) deactivate(a, S, GBS_OK);
    else if (S.iterations >= C.maxit) deactivate(a, S, GBS_ERR_MAXIT);
    else {
      S.beta = tot[1] / S.rho;
      S.rho = tot[1];
    }
  };
  walk<2>(a, a.ta, 0, red, want, work, fin);
}

// y1 = w + beta y2, t = D^-1 y1, half step 2's x update.  Table E.
__device__ __forceinline__ void tfq_next(const PcgArgs &a, double *red) {
  double *x = a.call->x;
  const double *w = a.kv[0], *y2 = a.kv[2], *d = a.kv[7];
  double *y1 = a.kv[1], *t = a.kv[8];
  NsView v{};
  auto want = [&](int s) -> int {
    v = ns_view(a, s);  // issued with the active flag: one round trip
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int, int r0, int r1, double(&)[1]) {
    const double be = v.beta, e2 = v.eta;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double dv = a.dinv[i];
      const double y = w[i] + be * y2[i];
      y1[i] = y;
      t[i] = dv * y;
      x[i] = fma(e2, dv * d[i], x[i]);
    }
  };
  auto fin = [&](int, double(&)[1]) {};
  walk<0>(a, a.te, a.part_e, red, want, work, fin);
}

// The x update of a half step that ended its system's solve.  Table E.
__device__ __forceinline__ void tfq_pending_x(const PcgArgs &a, double *red) {
  double *x = a.call->x;
  const double *d = a.kv[7];
  double eta = 0.0;
  auto want = [&](int s) -> int {
    const SysState *S = a.st + s;
    if (ld_state(&S->active) || !ld_state(&S->pend)) return 0;
    eta = ld_state(&S->eta);
    return 1;
  };
  auto work = [&](int, int, int r0, int r1, double(&)[1]) {
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
      x[i] = fma(eta, a.dinv[i] * d[i], x[i]);
  };
  auto fin = [&](int, double(&)[1]) {};
  walk<0>(a, a.te, a.part_e, red, want, work, fin);
}

#define NS_ROWS __launch_bounds__(PHASE_TPB, SELL_MIN_CTAS)
#define NS_UPD __launch_bounds__(PHASE_TPB)

__device__ __forceinline__ void ns_start_clock(const PcgArgs &a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->t_start = (int64_t)global_ns();
}

__global__ void NS_ROWS k_bicg_setup(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  ns_start_clock(a);
  bicg_setup(a, red);
}
__global__ void NS_ROWS k_bicg_products(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (!trip_live(a)) return;
  bicg_products(a, red);
}
__global__ void NS_UPD k_bicg_update(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (!trip_live(a)) return;
  bicg_update(a, red);
}
__global__ void NS_UPD k_bicg_direction(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  const bool live = trip_live(a);
  loop_control(a, live);  // after the update's tests: n_active is final
  if (!live) return;
  bicg_direction(a, red);
}
__global__ void NS_ROWS k_tfq_setup(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  ns_start_clock(a);
  tfq_setup(a, red);
}
__global__ void NS_ROWS k_tfq_v(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (!trip_live(a)) return;
  tfq_v(a, red);
}
__global__ void NS_UPD k_tfq_half1(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (!trip_live(a)) return;
  tfq_half1(a, red);
}
__global__ void NS_ROWS k_tfq_half2(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (!trip_live(a)) return;
  tfq_half2(a, red);
}
__global__ void NS_UPD k_tfq_next(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  const bool live = trip_live(a);
  loop_control(a, live);  // after half step 2's tests: n_active is final
  if (!live) return;
  tfq_next(a, red);
}
__global__ void NS_UPD k_tfq_pending_x(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  tfq_pending_x(a, red);
}
__global__ void NS_ROWS k_ns_final(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  phase_final<0>(a, red);
}

static LoopPlan bicg_plan() {
  LoopPlan P;
  memset(&P, 0, sizeof(P));
  P.npre = 1;
  P.pre[0] = k_bicg_setup;
  P.nbody = 3;
  P.body[0] = k_bicg_products;
  P.body[1] = k_bicg_update;
  P.body[2] = k_bicg_direction;
  P.body_e[1] = P.body_e[2] = true;
  P.npost = 1;
  P.post[0] = k_ns_final;
  return P;
}

// Body order: the step's first product, half step 1, the product fused with
// half step 2, then y1 (whose kernel sets the loop condition after half step
// 2's tests).  A system retired by a later step's top tests leaves one empty
// trip at most.
static LoopPlan tfqmr_plan() {
  LoopPlan P;
  memset(&P, 0, sizeof(P));
  P.npre = 1;
  P.pre[0] = k_tfq_setup;
  P.nbody = 4;
  P.body[0] = k_tfq_v;
  P.body[1] = k_tfq_half1;
  P.body[2] = k_tfq_half2;
  P.body[3] = k_tfq_next;
  P.body_e[1] = P.body_e[3] = true;
  P.npost = 2;
  P.post[0] = k_tfq_pending_x;
  P.post_e[0] = true;
  P.post[1] = k_ns_final;
  return P;
}

// ------------------------------------------------------------------ pipelined CG
//
// Pipelined Jacobi-PCG (one reduction per iteration; Ghysels-Vanroose, the
// oracle's recurrences): u = M^-1 r, w = A u, p, s = A p, q = M^-1 s, z = A q
// updated alongside x and r.  The loop body is ONE kernel on table A: the
// product n = A m (m = M^-1 w, gathered from the buffer of this iteration's
// parity), fused per row with all eight updates, the next m = M^-1 w (into
// the other buffer: other CTAs still gather this iteration's m) and the
// partial gamma = r.u, delta = w.u, ||r||^2; the last arriver's fin runs the
// tests and computes the next alpha and beta.  CG's three kernels and two
// reductions per iteration become one and one.
//
// A recursive residual that meets the test is confirmed with the true one
// (the oracle's reading): the same kernel, in mode PIPE_VERIFY for that
// system, computes r = b - A x and u = M^-1 r; if ||r|| misses the test too,
// mode PIPE_RESTART computes w = A u and the next m, zeroes p, s, q, z and
// restarts the recurrences (beta = 0), counted in outer_iterations.
enum { PIPE_ITER = 0, PIPE_VERIFY = 1, PIPE_RESTART = 2 };

// The tests at the top of an iteration and the next alpha, beta from
// (gamma, delta, r.r); returns the status (GBS_OK: the recursive residual
// meets the test, to be confirmed), or -1 to go on.  S.first: the
// recurrences (re)start here, beta = 0.
__device__ __forceinline__ int pipe_top(const CallArgs &C, SysState &S, double gamma,
                                        double delta, double rr, bool may_converge) {
  const double rn = sqrt(rr);
  S.rr = rr;
  S.rnorm = rn;
  if (!isfinite(rn) || !isfinite(gamma) || !isfinite(delta)) return GBS_ERR_NAN;
  if (may_converge && rn <= S.thr) return GBS_OK;
  if (S.iterations >= C.maxit) return GBS_ERR_MAXIT;
  double beta = 0.0, den = delta;
  if (!S.first) {
    beta = gamma / S.rho;  // S.rho: the previous gamma
    den = delta - beta * gamma / S.alpha;
  }
  if (!(gamma > 0.0) || !(den > 0.0)) return GBS_ERR_BREAKDOWN;
  S.beta = beta;
  S.alpha = gamma / den;
  S.rho = gamma;
  S.first = 0;
  return -1;
}

// The single-reduction CG's step at the top of an iteration, run by all
// lanes of one warp: pipe_top's tests and recurrences, with the tests on
// the integer pipe (finite64, positive64, meets_thr), the square root of
// ||r||^2 taken only when the system stops (rn_stale otherwise: the closing
// kernel takes it), and beta = gamma / rho and gamma / alpha_prev divided in
// one instruction sequence on two lanes -- the last CTA's scalar step waits
// on each FP64 instruction.  den = delta - beta (gamma / alpha_prev) is the
// oracle's delta - (beta gamma) / alpha_prev with the product and quotient
// taken in the other order (equal in exact arithmetic).  Lane 0 writes the
// state; the status is the same on every lane.
__device__ __forceinline__ int sr_top(const CallArgs &C, SysState &S, double gamma, double delta,
                                      double rr, int lane) {
  int st = -1;
  if (!finite64(rr) || !finite64(gamma) || !finite64(delta)) st = GBS_ERR_NAN;
  else if (meets_thr(rr, S)) st = GBS_OK;
  else if (S.iterations >= C.maxit) st = GBS_ERR_MAXIT;
  double beta = 0.0, den = delta;
  if (st < 0 && !S.first) {
    const double d = gamma / (lane == 1 ? S.alpha : S.rho);  // lane 0: beta, lane 1: gamma / alpha
    beta = __shfl_sync(FULL_MASK, d, 0);
    den = delta - beta * __shfl_sync(FULL_MASK, d, 1);
  }
  if (st < 0 && (!positive64(gamma) || !positive64(den))) st = GBS_ERR_BREAKDOWN;
  if (st >= 0) {
    if (lane == 0) {
      S.rr = rr;
      S.rnorm = sqrt(rr);
      S.rn_stale = 0;
    }
    return st;
  }
  const double alpha = gamma / den;
  if (lane == 0) {
    S.rr = rr;
    S.rn_stale = 1;
    S.beta = beta;
    S.alpha = alpha;
    S.rho = gamma;
    S.first = 0;
  }
  return -1;
}

// After pipe_top: a recursive convergence goes to the confirmation, any
// other status ends the system.
__device__ __forceinline__ void pipe_after_top(const PcgArgs &a, SysState &S, int st) {
  if (st == GBS_OK) S.mode = PIPE_VERIFY;
  else if (st >= 0) deactivate(a, S, st);
}

// r = b - A x0, u = M^-1 r; r.r, b.b, missing diagonals; fin: start-up
// tests.  Table A.
__device__ __forceinline__ void pipe_setup(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  double *r = a.kv[0], *u = a.kv[1];
  auto want = [&](int) -> int { return 1; };
  auto row = [&](int i, double ax, double(&acc)[3]) {
    const double bv = b[i], rv = bv - ax, dv = a.dinv[i];
    r[i] = rv;
    u[i] = dv * rv;
    acc[0] = fma(rv, rv, acc[0]);
    acc[1] = fma(bv, bv, acc[1]);
    acc[2] += (dv == 0.0) ? 1.0 : 0.0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[3]) {
    if (C.nonzero_guess) {
      auto f = [&](int i, double ax) { row(i, ax, acc); };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, x, f);
    } else {
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        x[i] = 0.0;
        row(i, 0.0, acc);
      }
    }
  };
  auto fin = [&](int s, double(&tot)[3]) {
    SysState &S = a.st[s];
    memset(&S, 0, sizeof(SysState));
    S.bb = tot[1];
    set_thr(S, C.rtol * sqrt(S.bb));
    S.rr = tot[0];
    S.rnorm0 = S.rnorm = sqrt(tot[0]);
    S.first = 1;
    S.mode = PIPE_ITER;
    const int st = kry_start_status(tot[2], tot[1]);
    if (st == GBS_OK) {
      S.zero_x = 1;
      S.rnorm0 = S.rnorm = 0.0;
    }
    ns_activate(a, S, st);
  };
  walk<3>(a, a.ta, 0, red, want, work, fin);
}

// w = A u with m = M^-1 w (buffer 0), gamma, delta, r.r; p = s = q = z = 0;
// fin: the first iteration's tests, alpha.  Table A.
__device__ __forceinline__ void pipe_start(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *r = a.kv[0], *u = a.kv[1];
  double *w = a.kv[2], *p = a.kv[3], *sv = a.kv[4], *q = a.kv[5], *z = a.kv[6], *m = a.kv[7];
  auto want = [&](int s) -> int { return sys_active(a, s) ? 1 : 0; };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[3]) {
    double a0 = acc[0], a1 = acc[1], a2 = acc[2];
    auto f = [&](int i, double y) {
      const double ri = r[i], ui = u[i];
      w[i] = y;
      m[i] = a.dinv[i] * y;
      p[i] = 0.0;
      sv[i] = 0.0;
      q[i] = 0.0;
      z[i] = 0.0;
      a0 = fma(ri, ui, a0);
      a1 = fma(y, ui, a1);
      a2 = fma(ri, ri, a2);
    };
    row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, u, f);
    acc[0] = a0;
    acc[1] = a1;
    acc[2] = a2;
  };
  auto fin = [&](int s, double(&tot)[3]) {
    SysState &S = a.st[s];
    pipe_after_top(a, S, pipe_top(C, S, tot[0], tot[1], tot[2], true));
  };
  walk<3>(a, a.ta, 0, red, want, work, fin);
}

// One trip: an iteration, or for a system in PIPE_VERIFY / PIPE_RESTART the
// confirmation or the restart.  Table A.
__device__ __forceinline__ void pipe_iterate(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  double *r = a.kv[0], *u = a.kv[1], *w = a.kv[2], *p = a.kv[3], *sv = a.kv[4],
         *q = a.kv[5], *z = a.kv[6];
  double alpha = 0.0, beta = 0.0;
  int par = 0, mode = PIPE_ITER;
  auto want = [&](int s) -> int {
    const SysState *S = a.st + s;  // all loads issued together: one round trip
    alpha = ld_state(&S->alpha);
    beta = ld_state(&S->beta);
    par = ld_state(&S->iterations) & 1;
    mode = ld_state(&S->mode);
    return sys_active(a, s) ? 1 : 0;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[3]) {
    double a0 = acc[0], a1 = acc[1], a2 = acc[2];
    if (mode == PIPE_ITER) {
      const double *m_in = a.kv[7 + par];
      double *m_out = a.kv[8 - par];
      auto f = [&](int i, double nv) {
        const double dv = a.dinv[i];
        const double wi = w[i], ui = u[i];
        const double zi = nv + beta * z[i];
        const double qi = dv * wi + beta * q[i];  // m = M^-1 w at this row
        const double si = wi + beta * sv[i];
        const double pi = ui + beta * p[i];
        z[i] = zi;
        q[i] = qi;
        sv[i] = si;
        p[i] = pi;
        x[i] = x[i] + alpha * pi;
        const double rn = r[i] - alpha * si;
        const double un = ui - alpha * qi;
        const double wn = wi - alpha * zi;
        r[i] = rn;
        u[i] = un;
        w[i] = wn;
        m_out[i] = dv * wn;
        a0 = fma(rn, un, a0);
        a1 = fma(wn, un, a1);
        a2 = fma(rn, rn, a2);
      };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, m_in, f);
    } else if (mode == PIPE_VERIFY) {  // r = b - A x, u = M^-1 r, ||r||^2
      auto f = [&](int i, double ax) {
        const double rv = b[i] - ax;
        r[i] = rv;
        u[i] = a.dinv[i] * rv;
        a0 = fma(rv, rv, a0);
      };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, x, f);
    } else {  // PIPE_RESTART: w = A u, the next m, p = s = q = z = 0
      double *m_next = a.kv[7 + par];
      auto f = [&](int i, double y) {
        const double ri = r[i], ui = u[i];
        w[i] = y;
        m_next[i] = a.dinv[i] * y;
        p[i] = 0.0;
        sv[i] = 0.0;
        q[i] = 0.0;
        z[i] = 0.0;
        a0 = fma(ri, ui, a0);
        a1 = fma(y, ui, a1);
        a2 = fma(ri, ri, a2);
      };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, u, f);
    }
    acc[0] = a0;
    acc[1] = a1;
    acc[2] = a2;
  };
  auto fin = [&](int s, double(&tot)[3]) {
    SysState &S = a.st[s];
    const int md = S.mode;
    if (md == PIPE_ITER) {
      S.iterations += 1;
      pipe_after_top(a, S, pipe_top(C, S, tot[0], tot[1], tot[2], true));
    } else if (md == PIPE_VERIFY) {
      const double tn = sqrt(tot[0]);
      S.rnorm = tn;
      if (!isfinite(tn)) deactivate(a, S, GBS_ERR_NAN);
      else if (tn <= S.thr) deactivate(a, S, GBS_OK);
      else {
        S.outer += 1;  // a restart
        S.mode = PIPE_RESTART;
      }
    } else {  // the restarted recurrences' first tests (the true residual just missed)
      S.first = 1;
      const int st = pipe_top(C, S, tot[0], tot[1], tot[2], false);
      if (st >= 0) deactivate(a, S, st);
      else S.mode = PIPE_ITER;
    }
  };
  walk<3>(a, a.ta, 0, red, want, work, fin);
}

__global__ void NS_ROWS k_pipe_setup(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  ns_start_clock(a);
  pipe_setup(a, red);
}
__global__ void NS_ROWS k_pipe_start(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  pipe_start(a, red);
}
__global__ void __launch_bounds__(PHASE_TPB, 2) k_pipe_iterate(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  const bool live = trip_live(a);
  loop_control(a, live);  // after the previous iteration's tests
  if (!live) return;
  pipe_iterate(a, red);
}

// setup, w = A u, WHILE { iterate }, final residual.
static LoopPlan pipecg_plan() {
  LoopPlan P;
  memset(&P, 0, sizeof(P));
  P.npre = 2;
  P.pre[0] = k_pipe_setup;
  P.pre[1] = k_pipe_start;
  P.nbody = 1;
  P.body[0] = k_pipe_iterate;
  P.npost = 1;
  P.post[0] = k_ns_final;
  return P;
}
// ------------------------------------------------------------------ single-reduction CG
//
// Jacobi-PCG in Chronopoulos and Gear's single-reduction form (the oracle's
// orc_pcg_sr): PCG's iterates in exact arithmetic, with both inner products
// of an iteration taken together after the product, so that an iteration is
// one reduction and TWO kernels instead of the textbook form's two and three:
//   SpMV kernel (table A): w = A u fused with the partial delta = w.u; its
//     last arriver adds up delta and the update kernel's partials of
//     gamma = r.u and ||r||^2 (below), runs the tests and computes
//     beta = gamma / gamma_prev and alpha = gamma / (delta - beta gamma /
//     alpha_prev) (pipe_top, shared with the pipelined CG);
//   update kernel (table E): p = u + beta p, s = w + beta s, x += alpha p,
//     r -= alpha s, u = M^-1 r, fused with the partial sums of the new
//     r.u and r.r; each CTA writes its partials to its reduction slot and
//     goes on -- no arrival count, no last CTA waiting: the next SpMV
//     kernel's fin sums the slots.  Its last CTA sets the loop condition.
// So the SpMV kernel does exactly the textbook CG's product work, and the
// update kernel has no reduction tail.  The first trip takes r.u and ||r||^2
// of the start residual from the setup (S.gam, S.rr).  Work vectors: r, u,
// w, p, s = kv[0..4].  Traffic 12 nnz + 120 n bytes and nnz + 8 n FP64
// operations per iteration.

// r = b - A x0, u = M^-1 r; partials r.r, b.b, missing diagonals, r.u;
// fin: start-up tests (those of the pipelined CG), S.gam = r.u.  Table A.
__device__ __forceinline__ void sr_setup(const PcgArgs &a, double *red) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  double *r = a.kv[0], *u = a.kv[1];
  auto want = [&](int) -> int { return 1; };
  auto row = [&](int i, double ax, double(&acc)[4]) {
    const double bv = b[i], rv = bv - ax, dv = a.dinv[i], uv = dv * rv;
    r[i] = rv;
    u[i] = uv;
    acc[0] = fma(rv, rv, acc[0]);
    acc[1] = fma(bv, bv, acc[1]);
    acc[2] += (dv == 0.0) ? 1.0 : 0.0;
    acc[3] = fma(rv, uv, acc[3]);
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[4]) {
    if (C.nonzero_guess) {
      auto f = [&](int i, double ax) { row(i, ax, acc); };
      row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, x, f);
    } else {
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        x[i] = 0.0;
        row(i, 0.0, acc);
      }
    }
  };
  auto fin = [&](int s, double(&tot)[4]) {
    SysState &S = a.st[s];
    memset(&S, 0, sizeof(SysState));
    S.bb = tot[1];
    set_thr(S, C.rtol * sqrt(S.bb));
    S.rr = tot[0];
    S.gam = tot[3];
    S.rnorm0 = S.rnorm = sqrt(tot[0]);
    S.first = 1;
    const int st = kry_start_status(tot[2], tot[1]);
    if (st == GBS_OK) {
      S.zero_x = 1;
      S.rnorm0 = S.rnorm = 0.0;
    }
    ns_activate(a, S, st);
  };
  walk<4>(a, a.ta, 0, red, want, work, fin);
}

// w = A u with delta = w.u; fin (the last arriver): the tests, alpha, beta.
// gamma and ||r||^2 are the update kernel's slot partials (on the first trip
// the setup's).  Ensemble solves sum them in the product kernel's wide
// finish, with its own slots; per-system solves, whose finish is warp 0's,
// sum them while the product runs -- by warp 1 of the CTA that holds the
// system's first block, before that CTA's own arrival, so the sums are in
// S.gam / S.rr when the last arriver reads them.  Table A.
// (Not inlined, like sr_fin below: the product kernel runs at 32 registers,
// and these rarely run paths would otherwise make the compiler spill around
// the row loop.)
__device__ __noinline__ void sr_presum(const PcgArgs &a, int s) {
  SysState &S = a.st[s];
  if (ldcg(&S.first)) return;
  double gr[2];
  const int ns = min(sys_nblk(a, a.te, s), a.grid_e);
  slot_sums<2>(a.part, a.part_e + sys_slot0(a, a.te, s), ns, gr);
  if ((threadIdx.x & 31) == 0) {
    S.gam = gr[0];
    S.rr = gr[1];
    __threadfence();  // before this CTA's arrival (block_reduce barrier, fence, count)
  }
}

__device__ __noinline__ void sr_fin(const PcgArgs &a, int s, double delta, double gam,
                                    double rr, int lane) {
  SysState &S = a.st[s];
  // on the first trip, and for per-system solves, r.u and ||r||^2 are in the
  // state (the setup's, or sr_presum's sums); ensemble solves get the update
  // kernel's sums from the wide finish
  if (!a.ensemble || S.first) {
    gam = ldcg(&S.gam);
    rr = ldcg(&S.rr);
  }
  const int st = sr_top(*a.call, S, gam, delta, rr, lane);
  if (lane == 0) {
    if (st >= 0) deactivate(a, S, st);
    else S.iterations += 1;  // the update kernel applies this iteration
  }
}

template <bool ENS>
__device__ __forceinline__ void sr_spmv(const PcgArgs &a, double *red) {
  const double *u = a.kv[1];
  double *w = a.kv[2];
  auto want = [&](int s) -> int {
    if (!sys_active(a, s)) return 0;
    // per-system solves: warp 1 of the CTA whose first block of s is the
    // system's first block (ensemble solves sum them in the wide finish)
    if constexpr (!ENS) {
      if (blockIdx.x == sys_b0(a, a.ta, s) % gridDim.x && (threadIdx.x >> 5) == 1)
        sr_presum(a, s);
    }
    return 1;
  };
  auto work = [&](int, int blk, int r0, int r1, double(&acc)[1]) {
    double dl = acc[0];
    auto f = [&](int i, double y) {
      w[i] = y;
      dl = fma(y, __ldg(u + i), dl);
    };
    row_products<double, 0>(a, blk, r0, r1, a.val, a.sval, u, f);
    acc[0] = dl;
  };
  auto fin = [&](int s, double(&tot)[3], int lane) { sr_fin(a, s, tot[0], tot[1], tot[2], lane); };
  walk<1, true, 2>(a, a.ta, 0, red, want, work, fin);
}

// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^-1 r
// (beta = 0: p = u, s = w, whatever p and s held), with the partial r.u and
// r.r of the new r, u written to the CTA's slot (no arrival).  Table E.
__device__ __forceinline__ void sr_update(const PcgArgs &a, double *red) {
  double *x = a.call->x;
  double *r = a.kv[0], *u = a.kv[1], *p = a.kv[3], *sv = a.kv[4];
  const double *w = a.kv[2];
  double alpha = 0.0, beta = 0.0;
  auto want = [&](int s) -> int {
    const SysState *S = a.st + s;  // issued with the active flag: one round trip
    alpha = ld_state(&S->alpha);
    beta = ld_state(&S->beta);
    return sys_active(a, s) ? 1 : 0;
  };
  auto fin = [&](int, double(&)[2]) {};
  auto work = [&](int, int, int r0, int r1, double(&acc)[2]) {
    const double al = alpha, be = beta;
    double g = acc[0], q = acc[1];
    if (be == 0.0) {  // the first iteration
      for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double ui = u[i], wi = w[i];
        p[i] = ui;
        sv[i] = wi;
        x[i] = fma(al, ui, x[i]);
        const double rn = fma(-al, wi, r[i]);
        const double un = a.dinv[i] * rn;
        r[i] = rn;
        u[i] = un;
        g = fma(rn, un, g);
        q = fma(rn, rn, q);
      }
    } else {
      auto load = [&](int i) {
        return Vals<double, 7>{{u[i], w[i], p[i], sv[i], x[i], r[i], a.dinv[i]}};
      };
      auto apply = [&](int i, const Vals<double, 7> &v) {
        const double pi = fma(be, v.v[2], v.v[0]);
        const double si = fma(be, v.v[3], v.v[1]);
        p[i] = pi;
        sv[i] = si;
        x[i] = fma(al, pi, v.v[4]);
        const double rn = fma(-al, si, v.v[5]);
        const double un = v.v[6] * rn;
        r[i] = rn;
        u[i] = un;
        g = fma(rn, un, g);
        q = fma(rn, rn, q);
      };
      rows2(r0, r1, load, apply);
    }
    acc[0] = g;
    acc[1] = q;
  };
  walk<2, false>(a, a.te, a.part_e, red, want, work, fin);
}

// ENS: an ensemble solve (a.ensemble; no per-system pre-sums in the kernel)
// MB = 2: the build for plans capped at one or two CTAs per SM (64 registers;
// C2 product phase 55.1 -> 54.7 us per iteration).
template <bool ENS, int MB = SELL_MIN_CTAS>
__global__ void __launch_bounds__(PHASE_TPB, MB) k_sr_spmv(PcgArgs a) {
  __shared__ double red[RED_SCRATCH1];
  if (!trip_live(a)) return;
  stamp_phase(a, 1);
  sr_spmv<ENS>(a, red);
}
__global__ void __launch_bounds__(PHASE_TPB) k_sr_update(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  const bool live = trip_live(a);
  loop_control(a, live);  // after this trip's tests (the SpMV kernel's fin)
  if (!live) return;
  stamp_phase(a, 2);
  sr_update(a, red);
}

// The start-up and the closing residual, with the phase clock of
// ksp_get_phase_ns started and closed as for CG (setup, SpMV phase, update
// phase, closing residual).
__global__ void NS_ROWS k_sr_setup(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t t = (int64_t)global_ns();
    a.ctl->t_start = t;
    a.ctl->stamp = t;
    a.ctl->last_phase = 0;
  }
  sr_setup(a, red);
}
__global__ void NS_ROWS k_sr_final(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  stamp_phase(a, 4);
  phase_final<0>(a, red);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->phase_ns[4] += (int64_t)global_ns() - a.ctl->stamp;
}

// setup, WHILE { SpMV + reduction, update }, final residual.
static LoopPlan cgsr_plan(bool ensemble, bool wide) {
  LoopPlan P;
  memset(&P, 0, sizeof(P));
  P.npre = 1;
  P.pre[0] = k_sr_setup;
  P.nbody = 2;
  if (wide) P.body[0] = ensemble ? k_sr_spmv<true, 2> : k_sr_spmv<false, 2>;
  else P.body[0] = ensemble ? k_sr_spmv<true> : k_sr_spmv<false>;
  P.body[1] = k_sr_update;
  P.body_e[1] = true;
  P.npost = 1;
  P.post[0] = k_sr_final;
  return P;
}

// ------------------------------------------------------------------ single-kernel form
//
// The single-reduction loop as ONE kernel per iteration (ensemble solves on
// the sliced copy).  Between an iteration's vector update and its product
// w = A u no global synchronisation is needed: the product of a row reads u
// at the row's columns only, all within col_span rows of it.  So CTA c of
// table A (blocks c, c + G, ...):
//   1. updates its rows: p = u + beta p, s = w + beta s, x += alpha p,
//      r -= alpha s, u = M^-1 r, with the partial r.u and r.r;
//   2. publishes the iteration number in its flag (a barrier, a fence, a
//      release store);
//   3. waits until CTAs c - halo_lo .. c - halo_lo + halo_n - 1 (mod G) --
//      those holding every row within col_span of its rows, a window
//      build_plan derives from the block table -- have published it;
//   4. runs its row products w = A u with the partial w.u;
//   5. reduces the three partials; the last arriver runs the tests and the
//      next alpha and beta (pipe_top, as the two-kernel form's product
//      kernel does).
// The kernel boundary orders step 4 of one iteration before step 1 of the
// next (which overwrites u), so the flags are the only waits.  All CTAs of
// the grid are resident at once (cooperative launch: the grid is at most the
// kernel's occupancy times the SMs) and every CTA reaches step 2 without
// waiting on another, so every wait ends; each is still bounded (HALO_WAIT_NS
// of polling), after which the CTA records GBS_ERR_TIMEOUT in the control
// words and goes on, and the fin ends the solve with that status.
// Coherence: step 1 reads u through L2 (no L1 copy of an old value is made);
// the gathers of step 4 may use L1: a block's rows start at a multiple of 32,
// so each 128-byte line of u lies in one CTA's rows, and every line a CTA of
// this SM brings into L1 after its wait belongs to a CTA that has finished
// its update (L1 keeps nothing across launches).
// Same iterates as the two-kernel form; r.u and r.r are summed over table
// A's blocks instead of table E's, so they may differ from it in the last
// bits.  Per iteration: one launch, one reduction, the two-kernel form's
// FP64 work, and the vectors of the update read while the product's matrix
// stream has not yet passed over them.
constexpr uint64_t HALO_WAIT_NS = 1000000000ull;  // 1 s
constexpr uint32_t HALO_MAX_POLLS = 1u << 22;     // and a poll count, whatever the clock

// Step 3, by warp 0: lane l polls the flags of window entries l, l + 32, ...
// With one block per CTA the window does not wrap around the grid (CTA c's
// block is block c), with more it does (CTA c also holds c + G, ...).
__device__ __forceinline__ void halo_wait(const PcgArgs &a, int32_t epoch) {
  const int G = (int)gridDim.x;
  const bool wrap = a.ta.nblocks > G;
  const uint64_t t0 = global_ns();
  bool late = false;
  for (int j = (int)(threadIdx.x & 31); j < a.halo_n; j += 32) {
    int c = (int)blockIdx.x - a.halo_lo + j;  // halo_lo < G and j < G
    if (!wrap && (c < 0 || c >= G)) continue;
    c = c < 0 ? c + G : (c >= G ? c - G : c);
    const int32_t *f = a.halo_flags + c;
    for (uint32_t polls = 0; !late && ld_acquire(f) < epoch;)
      if (++polls >= HALO_MAX_POLLS || global_ns() - t0 > HALO_WAIT_NS) late = true;
  }
  if (late) atomicCAS(&a.ctl->err, 0, GBS_ERR_TIMEOUT);
  __threadfence();
  __syncwarp();
}

__global__ void NS_ROWS k_sr_fused(PcgArgs a) {
  // per-warp partials: r.u and r.r of the update, w.u of the products (the
  // sums need little shared memory, which leaves L1 its room for u)
  __shared__ double wred[3][PHASE_TPB / 32];
  const bool live = trip_live(a);
  loop_control(a, live);  // after the previous iteration's tests (its fin)
  if (!live) return;
  stamp_phase(a, 2);
  SysState *S = a.st;  // ensemble: one system
  const int act = ld_state(&S->active);  // issued together: one round trip
  const double al = ld_state(&S->alpha), be = ld_state(&S->beta);
  const int32_t epoch = ld_state(&S->iterations);
  if (!act) return;
  const int G = (int)gridDim.x, nb = a.ta.nblocks;
  double *x = a.call->x;
  double *r = a.kv[0], *u = a.kv[1], *w = a.kv[2], *p = a.kv[3], *sv = a.kv[4];
  double acc[2] = {0.0, 0.0};  // r.u, r.r
  // 1. the update of the CTA's rows
  for (int b = blockIdx.x; b < nb; b += G) {
    const int r0 = __ldg(a.ta.row0 + b), r1 = blk_row_end(a.ta, b);
    for (int i = r0 + (int)threadIdx.x; i < r1; i += (int)blockDim.x) {
      const double ui = __ldcg(u + i), wi = w[i], pv = p[i], sw = sv[i], xi = x[i], ri = r[i];
      const double di = a.dinv[i];
      const double pi = be == 0.0 ? ui : fma(be, pv, ui);  // beta = 0: p = u, s = w
      const double si = be == 0.0 ? wi : fma(be, sw, wi);
      p[i] = pi;
      sv[i] = si;
      x[i] = fma(al, pi, xi);
      const double rn = fma(-al, si, ri);
      const double un = di * rn;
      r[i] = rn;
      u[i] = un;
      acc[0] = fma(rn, un, acc[0]);
      acc[1] = fma(rn, rn, acc[1]);
    }
  }
  // the update's partials wait in shared memory, one pair per warp, while the
  // row products run
  warp_sums<double, 2>(acc);
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  if (lane == 0) {
    wred[0][warp] = acc[0];
    wred[1][warp] = acc[1];
  }
  // 2. publish, 3. wait for the window
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(a.halo_flags + blockIdx.x, epoch);
  }
  if (threadIdx.x < 32) halo_wait(a, epoch);
  __syncthreads();
  stamp_phase(a, 1);
  // 4. the row products and w.u
  int last = blockIdx.x;
  double acc2 = 0.0;
  for (int b = blockIdx.x; b < nb; b += G) {
    const int s0 = __ldg(a.ta.slice0 + b), s1 = blk_slice_end(a.ta, b);
    double dl = acc2;
    auto f = [&](int i, double y) {
      w[i] = y;
      dl = fma(y, __ldca(u + i), dl);
    };
    if (a.stream_matrix)
      sell_rows<double, true, GATHER_CA>(a.sv, a.sval, u, s0, s1, f);
    else
      sell_rows<double, false, GATHER_CA>(a.sv, a.sval, u, s0, s1, f);
    acc2 = dl;
    last = b;
  }
  // 5. one reduction; the last arriver runs the tests and the next scalars
  auto fin = [&](int s, double(&tot)[3], int lane) {
    SysState &T = a.st[s];
    int st = sr_top(*a.call, T, tot[0], tot[2], tot[1], lane);
    const int err = ldcg(&a.ctl->err);  // a bounded wait that ran out
    if (lane != 0) return;
    if (err) {
      st = err;
      T.rnorm = sqrt(T.rr);
      T.rn_stale = 0;
    }
    if (st >= 0) deactivate(a, T, st);
    else T.iterations += 1;
  };
  acc2 = warp_sum(acc2);
  if (lane == 0) wred[2][warp] = acc2;
  __syncthreads();
  if (warp != 0) return;
  double tot[3];
  const bool have = lane < (int)(blockDim.x >> 5);
#pragma unroll
  for (int k = 0; k < 3; ++k) tot[k] = have ? wred[k][lane] : 0.0;
  warp_sums<double, 3>(tot);
  flush<3, true, true>(a, a.ta, 0, 0, last, tot, nullptr, false, fin);
}

// setup, first product (alpha for the first update), WHILE { one kernel },
// final residual.
static LoopPlan cgsr_fused_plan() {
  LoopPlan P;
  memset(&P, 0, sizeof(P));
  P.npre = 2;
  P.pre[0] = k_sr_setup;
  P.pre[1] = k_sr_spmv<true>;
  P.nbody = 1;
  P.body[0] = k_sr_fused;
  P.body_coop = true;
  P.npost = 1;
  P.post[0] = k_sr_final;
  return P;
}

// The single-kernel form applies: an ensemble solve on the sliced copy whose
// table A grid fits on the device at once.
static bool fused_fits(gbs_mat A, bool per_system) {
  if (per_system || A->lanes != GBS_SPMV_SELL || A->halo_n <= 0) return false;
  int occ = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sr_fused, PHASE_TPB, 0) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return A->ta.grid <= occ * nsm;
}

// ------------------------------------------------------------------ transpose

// Transposed COO indices, local to each system: nonzero p of row r (system s,
// first row o_s) becomes (col_p - o_s, r - o_s).  Its COO index is p, so the
// transpose's numeric stage reads A's CSR values directly.
__global__ void k_transpose_coo(int64_t nrows, int32_t nsys, const int64_t *__restrict__ row_off,
                                const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col, int32_t *__restrict__ ti,
                                int32_t *__restrict__ tj) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nsys;  // row_off[lo] <= r < row_off[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (row_off[mid] <= r) lo = mid;
      else hi = mid;
    }
    const int64_t o = row_off[lo];
    for (int32_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      ti[p] = col[p] - (int32_t)o;
      tj[p] = (int32_t)(r - o);
    }
  }
}

// nnz offsets of the systems: row_ptr at each system's first row.
__global__ void k_system_nnz_off(int32_t nsys, const int64_t *__restrict__ row_off,
                                 const int32_t *__restrict__ row_ptr, int64_t *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s <= nsys) out[s] = row_ptr[row_off[s]];
}

namespace {
struct DevBuf {  // device scratch returned to the pool on every exit path
  void *p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() { dev_free(p, s); }
};
unsigned grid_rows(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 16));
}
}  // namespace

static int build_transpose(gbs_mat A, cudaStream_t s) {
  const int32_t ns = A->nsys;
  DevBuf off, ti, tj, cnt;
  off.s = ti.s = tj.s = cnt.s = s;
  const size_t m = (size_t)std::max<int64_t>(A->nnz, 1);
  GBS_TRY(dev_alloc_bytes(&off.p, sizeof(int64_t) * (ns + 1), s));
  GBS_TRY(dev_alloc_bytes(&cnt.p, sizeof(int64_t) * (ns + 1), s));
  GBS_TRY(dev_alloc_bytes(&ti.p, sizeof(int32_t) * m, s));
  GBS_TRY(dev_alloc_bytes(&tj.p, sizeof(int32_t) * m, s));
  GBS_TRY_CUDA(cudaMemcpyAsync(off.p, A->row_off_h.data(), sizeof(int64_t) * (ns + 1),
                               cudaMemcpyHostToDevice, s));
  std::vector<int64_t> coo_off(ns + 1, 0);
  if (A->nrows > 0) {
    k_transpose_coo<<<grid_rows(A->nrows), 256, 0, s>>>(A->nrows, ns, (const int64_t *)off.p,
                                                        A->row_ptr, A->col, (int32_t *)ti.p,
                                                        (int32_t *)tj.p);
    GBS_LAUNCHED(1);
  }
  k_system_nnz_off<<<(ns + 256) / 256, 256, 0, s>>>(ns, (const int64_t *)off.p, A->row_ptr,
                                                    (int64_t *)cnt.p);
  GBS_LAUNCHED(1);
  GBS_TRY_CUDA(cudaMemcpyAsync(coo_off.data(), cnt.p, sizeof(int64_t) * (ns + 1),
                               cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaStreamSynchronize(s));
  gbs_mat T = new (std::nothrow) gbs_mat_s();
  if (!T) return GBS_ERR_ALLOC;
  T->device = A->device;
  T->nrows = A->ncols;
  T->ncols = A->nrows;
  T->ncoo = A->nnz;
  T->nsys = ns;
  T->batched = A->batched;
  T->row_off_h = A->row_off_h;
  T->sell_patterns = A->sell_patterns;
  int st = symbolic(T, (const int32_t *)ti.p, (const int32_t *)tj.p,
                    A->batched ? coo_off.data() : nullptr, s);
  if (st == GBS_OK) st = sell_build(T, s);
  if (st == GBS_OK && cudaStreamSynchronize(s) != cudaSuccess) st = GBS_ERR_CUDA;
  if (st == GBS_OK && (T->nnz != A->nnz || T->nslices != A->nslices)) {
    set_error("transpose: %lld nonzeros in %lld slices, expected %lld in %lld",
              (long long)T->nnz, (long long)T->nslices, (long long)A->nnz,
              (long long)A->nslices);
    st = GBS_ERR_CUDA;
  }
  if (st != GBS_OK) {
    free_handle(T);
    return st;
  }
  A->At = T;
  A->at_version = -1;
  return GBS_OK;
}

// Sliced copy of A, work vectors, per-system ranges and (BiCG) the transpose
// with A's current values.
static int ensure_krylov(gbs_mat A, bool transpose, cudaStream_t s) {
  GBS_TRY(sell_build(A, s));
  bool grew = false;
  if (!A->kv) {
    GBS_TRY(dev_alloc(&A->kv, KRYLOV_NVEC * (size_t)std::max<int64_t>(A->nrows, 1), s));
    grew = true;
  }
  if (!A->sys_row0) {
    std::vector<int32_t> r0(A->nsys + 1), s0(A->nsys + 1);
    for (int32_t q = 0; q <= A->nsys; ++q) {
      r0[q] = (int32_t)A->row_off_h[q];
      s0[q] = A->sell_slice0_h[q];
    }
    int32_t *d = nullptr;
    GBS_TRY(dev_alloc(&d, 2 * ((size_t)A->nsys + 1), s));
    A->sys_row0 = d;
    A->sys_slice0 = d + A->nsys + 1;
    GBS_TRY_CUDA(cudaMemcpyAsync(A->sys_row0, r0.data(), sizeof(int32_t) * (A->nsys + 1),
                                 cudaMemcpyHostToDevice, s));
    GBS_TRY_CUDA(cudaMemcpyAsync(A->sys_slice0, s0.data(), sizeof(int32_t) * (A->nsys + 1),
                                 cudaMemcpyHostToDevice, s));
    grew = true;
  }
  if (grew) GBS_TRY_CUDA(cudaStreamSynchronize(s));
  if (transpose) {
    if (!A->At) GBS_TRY(build_transpose(A, s));
    if (A->at_version != A->values_version) {
      GBS_TRY(launch_set_values(A->At, A->val, GBS_INSERT, s));
      A->at_version = A->values_version;
    }
  }
  return GBS_OK;
}

int solve_krylov(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
                 cudaStream_t s) {
  const bool bicg = o.method == GBS_KSP_BICG, pipe = o.method == GBS_KSP_PIPECG,
             sr = o.method == GBS_KSP_CGSR;
  GBS_TRY(ensure_solver_workspace(A, false, s));
  GBS_TRY(ensure_krylov(A, bicg, s));
  A->last_count = per_system ? A->nsys : 1;
  A->last_ensemble = !per_system;
  A->trips_counted = true;
  // automatic: one 1024-thread CTA per SM already beats the phase kernels;
  // pipelined and single-reduction CG exist for the phase kernels only
  const int32_t sv = solver_for(A, per_system);
  const bool on_ctas = !pipe && !sr && (sv == GBS_SOLVER_CTA ||
                                        ((sv == GBS_SOLVER_AUTO || sv == GBS_SOLVER_SPLIT) &&
                                         cta_size_rule(A, per_system, 1)));
  if (!on_ctas) {
    A->last_solver = GBS_SOLVER_PHASES;
    if (A->ta.nblocks == 0) {  // empty matrix: nothing to iterate
      GBS_TRY_CUDA(cudaMemsetAsync(A->st, 0, sizeof(SysState) * A->nsys, s));
      GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
      return GBS_OK;
    }
    PcgArgs pa = make_args(A, per_system, false);
    pa.stream_matrix = stream_matrix(A, bicg ? 24 : 12);
    if (pipe) return run_loop(A, pipecg_plan(), GBS_GRAPH_PIPECG, pa, b, x, o, per_system, s);
    if (sr && A->cg_form == GBS_CG_SINGLE_KERNEL && fused_fits(A, per_system))
      return run_loop(A, cgsr_fused_plan(), GBS_GRAPH_CGSR1, pa, b, x, o, per_system, s);
    if (sr) return run_loop(A, cgsr_plan(!per_system, wide_rows(A)), GBS_GRAPH_CGSR, pa, b, x, o, per_system, s);
    return run_loop(A, bicg ? bicg_plan() : tfqmr_plan(),
                    bicg ? GBS_GRAPH_BICG : GBS_GRAPH_TFQMR, pa, b, x, o, per_system, s);
  }
  A->last_solver = GBS_SOLVER_CTA;
  GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
  GBS_TRY(put_call(A->call, call_args(b, x, o), s, A->ctl));
  KrylovArgs a;
  memset(&a, 0, sizeof(a));
  a.ensemble = per_system ? 0 : 1;
  a.nrows = (int32_t)A->nrows;
  a.nslices = (int32_t)A->nslices;
  a.order = A->cta_order;
  a.sys_row0 = A->sys_row0;
  a.sys_slice0 = A->sys_slice0;
  a.sv = sell_view(A);
  a.sval = A->sell_val;
  if (bicg) {
    a.tv = sell_view(A->At);
    a.tval = A->At->sell_val;
  }
  a.stream_matrix = stream_matrix(A, bicg ? 24 : 12);
  a.dinv = A->dinv;
  for (int k = 0; k < KRYLOV_NVEC; ++k) a.v[k] = A->kv + (size_t)k * (size_t)A->nrows;
  a.st = A->st;
  a.ctl = A->ctl;
  a.call = A->call;
  const unsigned grid = per_system ? (unsigned)A->nsys : 1u;
  const bool two = per_system && A->nsys >= 2 * sm_count(A);
  if (bicg) {
    if (two) k_cta_krylov<GBS_KSP_BICG, 2><<<grid, CTA_TPB, 0, s>>>(a);
    else k_cta_krylov<GBS_KSP_BICG, 1><<<grid, CTA_TPB, 0, s>>>(a);
  } else {
    if (two) k_cta_krylov<GBS_KSP_TFQMR, 2><<<grid, CTA_TPB, 0, s>>>(a);
    else k_cta_krylov<GBS_KSP_TFQMR, 1><<<grid, CTA_TPB, 0, s>>>(a);
  }
  GBS_LAUNCHED(1);
  return GBS_OK;
}

}  // namespace gbs
