// Jacobi-PCG with one CTA per system (Sec. 6.1 CG with device-resident scalars
// and no host round trip; Sec. 7 batched systems; Sec. 2 A7 FP32 inner solve
// under FP64 refinement).
//
// The CTA owns every row of its system, so every iteration runs inside one
// kernel launch with CTA barriers only: no kernel boundary, no grid-wide
// reduction and no inter-CTA wait.  This is the latency path: a small system
// iterates in a few microseconds, and a batch of systems runs as independent
// CTAs (largest first) that fill the GPU together.  The arithmetic is the
// phase kernels' (phases.cuh): sliced-ELL row products with one FMA per
// nonzero, the same updates, deterministic block reductions in a fixed order,
// and the same per-system state (SysState) and statuses.
//
// Loads of vectors the CTA itself writes use the coherent L1 path (ld_x<false>
// and plain loads): __syncthreads orders a CTA's global writes for its own
// threads, the read-only path does not.
#pragma once

#include "phases.cuh"

namespace gbs {

constexpr int CTA_TPB = 1024;  // threads of a system's CTA

struct CtaShared {
  double red[2 * 4 * 32];  // two halves of block_allreduce scratch
  int flag[2];             // [1]: the wall-clock limit was reached
};

// Block sums for the per-CTA solvers: every thread receives the totals (one
// barrier each), so every thread runs the scalar recurrences and the tests
// itself, identically, and control flow stays uniform without broadcasts.
struct CtaRed {
  CtaShared &sh;
  int half;
};

template <typename T, int NV>
__device__ __forceinline__ void cta_sum(T (&v)[NV], CtaRed &R) {
  block_allreduce<T, NV>(v, reinterpret_cast<T *>(R.sh.red), R.half);
  R.half ^= 1;
}

// Rows [r0, r1) and slices [s0, s1) of the system this CTA solves.
struct SysRange {
  int s, r0, r1, s0, s1;
};

__device__ __forceinline__ SysRange cta_system(const PcgArgs &a) {
  SysRange g;
  if (a.ensemble) {
    g.s = 0;
    g.r0 = 0;
    g.r1 = __ldg(a.ta.row0 + a.ta.nblocks);
    g.s0 = 0;
    g.s1 = __ldg(a.ta.slice0 + a.ta.nblocks);
  } else {
    g.s = a.order ? __ldg(a.order + blockIdx.x) : (int)blockIdx.x;
    const int b0 = __ldg(a.ta.sys_blk0 + g.s), b1 = __ldg(a.ta.sys_blk0 + g.s + 1);
    g.r0 = __ldg(a.ta.row0 + b0);
    g.r1 = __ldg(a.ta.row0 + b1);
    g.s0 = __ldg(a.ta.slice0 + b0);
    g.s1 = __ldg(a.ta.slice0 + b1);
  }
  return g;
}

// Sliced-ELL row products of the system's slices, coherent x gathers.
template <typename T, class F>
__device__ __forceinline__ void cta_rows(const PcgArgs &a, const SysRange &g, const T *sval,
                                         const T *x, F &f) {
  if (a.stream_matrix) sell_rows<T, true, false>(a.sptr, a.srow0, a.scol, sval, x, g.s0, g.s1, f);
  else sell_rows<T, false, false>(a.sptr, a.srow0, a.scol, sval, x, g.s0, g.s1, f);
}

// Wall-clock limit (from the solve's start, DevCtl::t_start): thread 0 reads
// the clock, one barrier shares the answer (the flag is rewritten only after
// later barriers).  Callers skip it when no limit is set.
__device__ __forceinline__ bool cta_timed_out(const DevCtl *ctl, int64_t lim, CtaShared &sh) {
  if (threadIdx.x == 0) sh.flag[1] = (int64_t)global_ns() - ldcg(&ctl->t_start) > lim;
  __syncthreads();
  return sh.flag[1] != 0;
}

// The system's closing state, written by thread 0: status (a system stopped
// by the time limit stays active and is reported through DevCtl::err),
// iterations, norms.
__device__ __forceinline__ void cta_store_state(const PcgArgs &a, SysState &S, int status,
                                                bool timed_out, int iterations, int outer,
                                                double bb, double rnorm0, double rnorm,
                                                bool zero_x) {
  if (threadIdx.x != 0) return;
  memset(&S, 0, sizeof(SysState));
  S.bb = bb;
  S.rnorm0 = rnorm0;
  S.rnorm = rnorm;
  S.iterations = iterations;
  S.outer = outer;
  S.zero_x = zero_x ? 1 : 0;
  S.status = timed_out ? GBS_OK : status;
  S.active = timed_out ? 1 : 0;
  if (timed_out) a.ctl->err = GBS_ERR_TIMEOUT;
}

// ||b - A x||^2 into S.tt (x set to 0 first where b = 0).
__device__ __forceinline__ void cta_true_residual(const PcgArgs &a, const SysRange &g,
                                                  SysState &S, bool zero_x, CtaRed &R) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  if (zero_x)
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) x[r] = 0.0;
  __syncthreads();  // x complete
  double tt[1] = {0.0};
  auto f = [&](int r, double t) {
    const double d = b[r] - t;
    tt[0] = fma(d, d, tt[0]);
  };
  cta_rows<double>(a, g, a.sval, x, f);
  cta_sum<double, 1>(tt, R);
  if (threadIdx.x == 0) S.tt = tt[0];
}

// FP64 PCG: the phases A, B, C of phases.cuh in one CTA, same tests.
static __device__ void cta_pcg_fp64(const PcgArgs &a, const SysRange &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  SysState &S = a.st[g.s];
  CtaRed R{sh, 0};
  // setup: r = b - A x0, z = D^-1 r, p = z
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // r.z, r.r, b.b, missing diagonals
  auto row = [&](int r, double t) {
    const double bv = b[r], rv = bv - t, dv = a.dinv[r], z = dv * rv;
    a.r[r] = rv;
    a.p[r] = z;
    v[0] = fma(rv, z, v[0]);
    v[1] = fma(rv, rv, v[1]);
    v[2] = fma(bv, bv, v[2]);
    v[3] += (dv == 0.0) ? 1.0 : 0.0;
  };
  if (C.nonzero_guess) {
    cta_rows<double>(a, g, a.sval, x, row);
  } else {
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
      x[r] = 0.0;
      row(r, 0.0);
    }
  }
  cta_sum<double, 4>(v, R);
  double rho = v[0];
  const double bb = v[2], thr = C.rtol * sqrt(bb);
  double rn = sqrt(v[1]), rnorm0 = rn;
  bool zero = false;
  int status = -1;
  if (v[3] > 0.0) status = GBS_ERR_NOT_SPD;
  else if (!isfinite(bb)) status = GBS_ERR_NAN;
  else if (bb == 0.0) {
    status = GBS_OK;
    zero = true;
    rn = rnorm0 = 0.0;
  } else if (!isfinite(v[1]) || !isfinite(rho)) status = GBS_ERR_NAN;
  else if (rn <= thr) status = GBS_OK;
  else if (C.maxit <= 0) status = GBS_ERR_MAXIT;
  int it = 0;
  bool timed = false;
  while (status < 0) {
    // A: q = A p, p.q
    double pq[1] = {0.0};
    auto fa = [&](int r, double qv) {
      a.q[r] = qv;
      pq[0] = fma(a.p[r], qv, pq[0]);
    };
    cta_rows<double>(a, g, a.sval, a.p, fa);
    cta_sum<double, 1>(pq, R);
    ++it;
    if (isnan(pq[0])) {
      status = GBS_ERR_NAN;
      break;
    }
    if (!(pq[0] > 0.0)) {
      status = GBS_ERR_BREAKDOWN;
      break;
    }
    const double al = rho / pq[0];
    // B: x += alpha p, r -= alpha q, z = D^-1 r (over q), r.z, r.r
    double w[2] = {0.0, 0.0};
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
      const double rv = fma(-al, a.q[r], a.r[r]);
      const double z = a.dinv[r] * rv;
      x[r] = fma(al, a.p[r], x[r]);
      a.r[r] = rv;
      a.q[r] = z;
      w[0] = fma(rv, z, w[0]);
      w[1] = fma(rv, rv, w[1]);
    }
    cta_sum<double, 2>(w, R);
    rn = sqrt(w[1]);
    if (!isfinite(rn) || !isfinite(w[0])) {
      status = GBS_ERR_NAN;
      break;
    }
    if (rn <= thr) {
      status = GBS_OK;
      break;
    }
    if (it >= C.maxit) {
      status = GBS_ERR_MAXIT;
      break;
    }
    if (C.timeout_ns > 0 && cta_timed_out(a.ctl, C.timeout_ns, sh)) {
      timed = true;
      break;
    }
    const double be = w[0] / rho;
    rho = w[0];
    // C: p = z + beta p (each thread its own rows: the rows B wrote)
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) a.p[r] = fma(be, a.p[r], a.q[r]);
    __syncthreads();  // p complete before the next product gathers it
  }
  cta_store_state(a, S, status, timed, it, 0, bb, rnorm0, rn, zero);
  cta_true_residual(a, g, S, zero, R);
}

// FP32 inner PCG under FP64 refinement, the oracle's order of steps.
static __device__ void cta_pcg_refined(const PcgArgs &a, const SysRange &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  SysState &S = a.st[g.s];
  CtaRed R{sh, 0};
  double v[2] = {0.0, 0.0};  // b.b, missing diagonals
  if (!C.nonzero_guess)
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) x[r] = 0.0;
  for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
    v[0] = fma(b[r], b[r], v[0]);
    v[1] += (a.dinv[r] == 0.0) ? 1.0 : 0.0;
  }
  cta_sum<double, 2>(v, R);  // (also orders the x writes before the first product)
  const double bb = v[0], bnorm = sqrt(bb);
  bool zero = false;
  int status = -1;
  if (v[1] > 0.0) status = GBS_ERR_NOT_SPD;
  else if (!isfinite(bb)) status = GBS_ERR_NAN;
  else if (bb == 0.0) {
    status = GBS_OK;
    zero = true;
  }
  double rnorm0 = 0.0, rn = 0.0, prev_rn = INFINITY;
  int outer = 0, stall = 0, iters = 0;
  bool timed = false;
  while (status < 0) {
    // outer FP64 residual r = b - A x
    double rr[1] = {0.0};
    auto fo = [&](int r, double t) {
      const double rv = b[r] - t;
      a.r[r] = rv;
      rr[0] = fma(rv, rv, rr[0]);
    };
    cta_rows<double>(a, g, a.sval, x, fo);
    cta_sum<double, 1>(rr, R);
    rn = sqrt(rr[0]);
    if (outer == 0) rnorm0 = rn;
    if (!isfinite(rn)) {
      status = GBS_ERR_NAN;
      break;
    }
    if (rn <= C.rtol * bnorm) {
      status = GBS_OK;
      break;
    }
    if (outer >= C.max_outer) {
      status = GBS_ERR_MAXIT;
      break;
    }
    if (outer > 0) {
      stall = (rn > 0.5 * prev_rn) ? stall + 1 : 0;
      if (stall >= 2) {
        status = GBS_ERR_STAGNATION;
        break;
      }
    }
    if (C.timeout_ns > 0 && cta_timed_out(a.ctl, C.timeout_ns, sh)) {
      timed = true;
      break;
    }
    prev_rn = rn;
    // inner FP32 PCG on RN(r / s) from d = 0
    const double s = rn;
    float w[2] = {0.0f, 0.0f};
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
      const float rv = __double2float_rn(a.r[r] / s);
      const float z = a.dinv32[r] * rv;
      a.r32[r] = rv;
      a.d32[r] = 0.0f;
      a.q32[r] = z;
      a.p32[r] = z;
      w[0] = fmaf(rv, z, w[0]);
      w[1] = fmaf(rv, rv, w[1]);
    }
    cta_sum<float, 2>(w, R);
    float rho = w[0], rr32 = w[1];
    const double tgt = fmax(C.inner_rtol, 0.5 * C.rtol * bnorm / s);
    const double thr = tgt * (double)sqrtf(rr32);
    int it = 0;
    while ((double)sqrtf(rr32) > thr && it < C.inner_maxit) {
      float pq[1] = {0.0f};
      auto fa = [&](int r, float qv) {
        a.q32[r] = qv;
        pq[0] = fmaf(a.p32[r], qv, pq[0]);
      };
      cta_rows<float>(a, g, a.sval32, a.p32, fa);
      cta_sum<float, 1>(pq, R);
      if (!(pq[0] > 0.0f)) break;
      ++it;
      const float al = rho / pq[0];
      float u[2] = {0.0f, 0.0f};
      for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
        const float rv = fmaf(-al, a.q32[r], a.r32[r]);
        const float z = a.dinv32[r] * rv;
        a.d32[r] = fmaf(al, a.p32[r], a.d32[r]);
        a.r32[r] = rv;
        a.q32[r] = z;
        u[0] = fmaf(rv, z, u[0]);
        u[1] = fmaf(rv, rv, u[1]);
      }
      cta_sum<float, 2>(u, R);
      const float be = u[0] / rho;
      rho = u[0];
      rr32 = u[1];
      for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x)
        a.p32[r] = fmaf(be, a.p32[r], a.q32[r]);
      __syncthreads();
    }
    iters += it;
    if (it == 0) {
      status = GBS_ERR_BREAKDOWN;
      break;
    }
    ++outer;
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x)
      x[r] = fma(s, (double)a.d32[r], x[r]);
    __syncthreads();  // x complete before the next outer residual gathers it
  }
  cta_store_state(a, S, status, timed, iters, outer, bb, rnorm0, rn, zero);
  cta_true_residual(a, g, S, zero, R);
}

template <bool REFINED>
__global__ void __launch_bounds__(CTA_TPB, 2) k_cta_pcg(PcgArgs a) {
  __shared__ CtaShared sh;
  const SysRange g = cta_system(a);
  if (REFINED) cta_pcg_refined(a, g, sh);
  else cta_pcg_fp64(a, g, sh);
}

}  // namespace gbs
