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
  double red[4 * 32];
  double sc[4];   // scalars broadcast by thread 0
  int flag[2];    // [0]: keep iterating, [1]: spare
};

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

// Block sum of NV values in a fixed tree; every thread gets the totals.
template <typename T, int NV>
__device__ __forceinline__ void cta_sum(T (&v)[NV], CtaShared &sh) {
  block_reduce<T, NV>(v, reinterpret_cast<T *>(sh.red));
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) reinterpret_cast<T *>(sh.sc)[k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = reinterpret_cast<T *>(sh.sc)[k];
  __syncthreads();
}

// Wall-clock limit (from the solve's start, DevCtl::t_start), checked by
// thread 0 once per iteration.
__device__ __forceinline__ bool cta_timed_out(const PcgArgs &a) {
  const int64_t lim = a.call->timeout_ns;
  return lim > 0 && (int64_t)global_ns() - ldcg(&a.ctl->t_start) > lim;
}

__device__ __forceinline__ void cta_finish(const PcgArgs &a, SysState &S, int status) {
  S.status = status;
  S.active = 0;
}

// ||b - A x||^2 into S.tt (x = 0 exactly where b = 0).
__device__ __forceinline__ void cta_true_residual(const PcgArgs &a, const SysRange &g,
                                                  SysState &S, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  if (ldcg(&S.zero_x)) {
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) x[r] = 0.0;
    __syncthreads();
  }
  double tt[1] = {0.0};
  auto f = [&](int r, double t) {
    const double d = b[r] - t;
    tt[0] = fma(d, d, tt[0]);
  };
  cta_rows<double>(a, g, a.sval, x, f);
  cta_sum<double, 1>(tt, sh);
  if (threadIdx.x == 0) S.tt = tt[0];
}

// FP64 PCG: the phases A, B, C of phases.cuh in one CTA, same tests.
static __device__ void cta_pcg_fp64(const PcgArgs &a, const SysRange &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  SysState &S = a.st[g.s];
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
  cta_sum<double, 4>(v, sh);
  double rho = v[0];
  const double bb = v[2];
  if (threadIdx.x == 0) {
    memset(&S, 0, sizeof(SysState));
    S.bb = bb;
    S.rho = rho;
    S.rr = v[1];
    S.rnorm0 = S.rnorm = sqrt(v[1]);
    int status = -1;
    if (v[3] > 0.0) status = GBS_ERR_NOT_SPD;
    else if (!isfinite(bb)) status = GBS_ERR_NAN;
    else if (bb == 0.0) {
      status = GBS_OK;
      S.zero_x = 1;
      S.rnorm0 = S.rnorm = 0.0;
    } else if (!isfinite(v[1]) || !isfinite(rho)) status = GBS_ERR_NAN;
    else if (sqrt(v[1]) <= C.rtol * sqrt(bb)) status = GBS_OK;
    else if (C.maxit <= 0) status = GBS_ERR_MAXIT;
    S.status = status >= 0 ? status : GBS_OK;
    S.active = status >= 0 ? 0 : 1;
    sh.flag[0] = S.active;
  }
  __syncthreads();
  while (sh.flag[0]) {
    // A: q = A p, p.q
    double pq[1] = {0.0};
    auto fa = [&](int r, double qv) {
      a.q[r] = qv;
      pq[0] = fma(a.p[r], qv, pq[0]);
    };
    cta_rows<double>(a, g, a.sval, a.p, fa);
    cta_sum<double, 1>(pq, sh);
    if (threadIdx.x == 0) {
      S.iterations += 1;
      if (isnan(pq[0])) cta_finish(a, S, GBS_ERR_NAN);
      else if (!(pq[0] > 0.0)) cta_finish(a, S, GBS_ERR_BREAKDOWN);
      else S.alpha = S.rho / pq[0];
      sh.flag[0] = S.active;
      sh.sc[3] = S.alpha;
    }
    __syncthreads();
    if (!sh.flag[0]) break;
    const double al = sh.sc[3];
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
    cta_sum<double, 2>(w, sh);
    if (threadIdx.x == 0) {
      const double rn = sqrt(w[1]);
      S.rr = w[1];
      S.rnorm = rn;
      if (!isfinite(rn) || !isfinite(w[0])) cta_finish(a, S, GBS_ERR_NAN);
      else if (rn <= C.rtol * sqrt(S.bb)) cta_finish(a, S, GBS_OK);
      else if (S.iterations >= C.maxit) cta_finish(a, S, GBS_ERR_MAXIT);
      else {
        S.beta = w[0] / S.rho;
        S.rho = w[0];
      }
      int go = S.active;
      if (go && cta_timed_out(a)) {  // the system stays active: reported as TIMEOUT
        a.ctl->err = GBS_ERR_TIMEOUT;
        go = 0;
      }
      sh.flag[0] = go;
      sh.sc[3] = S.beta;
    }
    __syncthreads();
    if (!sh.flag[0]) break;
    const double be = sh.sc[3];
    // C: p = z + beta p
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) a.p[r] = fma(be, a.p[r], a.q[r]);
    __syncthreads();
  }
  __syncthreads();
  cta_true_residual(a, g, S, sh);
}

// FP32 inner PCG under FP64 refinement, the oracle's order of steps.
static __device__ void cta_pcg_refined(const PcgArgs &a, const SysRange &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  SysState &S = a.st[g.s];
  double v[3] = {0.0, 0.0, 0.0};  // b.b, missing diagonals, (unused)
  if (!C.nonzero_guess)
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) x[r] = 0.0;
  for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
    v[0] = fma(b[r], b[r], v[0]);
    v[1] += (a.dinv[r] == 0.0) ? 1.0 : 0.0;
  }
  cta_sum<double, 3>(v, sh);
  const double bb = v[0];
  if (threadIdx.x == 0) {
    memset(&S, 0, sizeof(SysState));
    S.bb = bb;
    S.prev_rn = INFINITY;
    int status = -1;
    if (v[1] > 0.0) status = GBS_ERR_NOT_SPD;
    else if (!isfinite(bb)) status = GBS_ERR_NAN;
    else if (bb == 0.0) {
      status = GBS_OK;
      S.zero_x = 1;
    }
    S.status = status >= 0 ? status : GBS_OK;
    S.active = status >= 0 ? 0 : 1;
    sh.flag[0] = S.active;
  }
  __syncthreads();
  const double bnorm = sqrt(bb);
  while (sh.flag[0]) {
    // outer FP64 residual r = b - A x
    double rr[1] = {0.0};
    auto fo = [&](int r, double t) {
      const double rv = b[r] - t;
      a.r[r] = rv;
      rr[0] = fma(rv, rv, rr[0]);
    };
    cta_rows<double>(a, g, a.sval, x, fo);
    cta_sum<double, 1>(rr, sh);
    const double rn = sqrt(rr[0]);
    if (threadIdx.x == 0) {
      if (S.outer == 0) S.rnorm0 = rn;
      S.rnorm = rn;
      int go = 1;
      if (!isfinite(rn)) cta_finish(a, S, GBS_ERR_NAN);
      else if (rn <= C.rtol * bnorm) cta_finish(a, S, GBS_OK);
      else if (S.outer >= C.max_outer) cta_finish(a, S, GBS_ERR_MAXIT);
      else if (S.outer > 0) {
        S.stall = (rn > 0.5 * S.prev_rn) ? S.stall + 1 : 0;
        if (S.stall >= 2) cta_finish(a, S, GBS_ERR_STAGNATION);
      }
      if (S.active && cta_timed_out(a)) {
        a.ctl->err = GBS_ERR_TIMEOUT;
        go = 0;
      }
      if (S.active && go) {
        S.prev_rn = rn;
        S.scale = rn;
      }
      sh.flag[0] = S.active && go;
    }
    __syncthreads();
    if (!sh.flag[0]) break;
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
    cta_sum<float, 2>(w, sh);
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
      cta_sum<float, 1>(pq, sh);
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
      cta_sum<float, 2>(u, sh);
      const float be = u[0] / rho;
      rho = u[0];
      rr32 = u[1];
      for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x)
        a.p32[r] = fmaf(be, a.p32[r], a.q32[r]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      S.iterations += it;
      if (it == 0) cta_finish(a, S, GBS_ERR_BREAKDOWN);
      else S.outer += 1;
      sh.flag[0] = S.active;
    }
    __syncthreads();
    if (!sh.flag[0]) break;
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x)
      x[r] = fma(s, (double)a.d32[r], x[r]);
    __syncthreads();
  }
  __syncthreads();
  cta_true_residual(a, g, S, sh);
}

template <bool REFINED>
__global__ void __launch_bounds__(CTA_TPB, 2) k_cta_pcg(PcgArgs a) {
  __shared__ CtaShared sh;
  const SysRange g = cta_system(a);
  if (REFINED) cta_pcg_refined(a, g, sh);
  else cta_pcg_fp64(a, g, sh);
}

}  // namespace gbs
