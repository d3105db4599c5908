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

// Thread 0 owns a system's scalars (FP64 scalar arithmetic is slow on this
// part: an FP64 warp instruction occupies a sub-partition's FP64 pipe for 64
// clocks, so the recurrences run in one thread, not redundantly in 32
// warps).  A block sum hands its totals to warp 0 (cta_sum0, two barriers);
// thread 0 updates the scalars and publishes what the next pass needs in
// `pub` / `ipub`; one more barrier (cta_publish) and every thread reads
// them.
struct CtaShared {
  double red[4 * CTA_TPB];            // cta_sum0: every thread's values
  double lanes[BLOCK_SUMS_EXTRA];     // cta_sum0: lane partials
  double pub[4];                      // scalars published by thread 0
  int ipub[4];                        // [0]: < 0 keep going; [1], [2], [3]: flags
};

// Block sums of NV values, valid in warp 0 (thread 0): device_util.cuh's
// block_sums, spread over the four sub-partitions' FP64 pipes.
template <typename T, int NV>
__device__ __forceinline__ void cta_sum0(T (&v)[NV], CtaShared &sh) {
  static_assert(CTA_TPB % 128 == 0 && CTA_TPB >= 256, "block_sums needs 128 k threads");
  block_sums<T, NV>(v, reinterpret_cast<T *>(sh.red), reinterpret_cast<T *>(sh.lanes));
}

// A thread's rows r0 + t, r0 + t + T, ... (t = threadIdx.x, T = blockDim.x),
// U at a time and in that order: load(r, k) for the U rows first, then
// use(r, k) for each -- so U rows' loads are in flight together (the rows a
// thread writes are never the ones its other rows read, which the compiler
// cannot see through the unrestricted pointers), and every sum a thread
// carries still adds its rows in the same order.
template <int U, class L, class F>
__device__ __forceinline__ void cta_rows_by(int r0, int r1, L &load, F &use) {
  for (int r = r0 + (int)threadIdx.x; r < r1; r += U * (int)blockDim.x) {
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (r + k * (int)blockDim.x < r1) load(r + k * (int)blockDim.x, k);
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (r + k * (int)blockDim.x < r1) use(r + k * (int)blockDim.x, k);
  }
}

// The barrier after thread 0 filled sh.pub / sh.ipub.
__device__ __forceinline__ void cta_publish() { __syncthreads(); }

// Rows [r0, r1) and slices [s0, s1) of the k-th system of the solver's
// order (the whole matrix for an ensemble solve).
struct SysRange {
  int s, r0, r1, s0, s1;
};

__device__ __forceinline__ SysRange cta_system(const PcgArgs &a, int k) {
  SysRange g;
  if (a.ensemble) {
    g.s = 0;
    g.r0 = 0;
    g.r1 = __ldg(a.ta.row0 + a.ta.nblocks);
    g.s0 = 0;
    g.s1 = __ldg(a.ta.slice0 + a.ta.nblocks);
  } else {
    g.s = a.order ? __ldg(a.order + k) : k;
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
  if (a.stream_matrix)
    sell_rows<T, true, GATHER_CA>(a.sv, sval, x, g.s0, g.s1, f);
  else
    sell_rows<T, false, GATHER_CA>(a.sv, sval, x, g.s0, g.s1, f);
}

// Wall-clock limit (from the solve's start, DevCtl::t_start), for thread 0.
__device__ __forceinline__ bool cta_timed_out(const DevCtl *ctl, int64_t lim) {
  return lim > 0 && (int64_t)global_ns() - ldcg(&ctl->t_start) > lim;
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
                                                  SysState &S, bool zero_x, CtaShared &sh) {
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
  cta_sum0<double, 1>(tt, sh);
  if (threadIdx.x == 0) S.tt = tt[0];
}

// FP64 PCG: the phases A, B, C of phases.cuh in one CTA, same tests.
template <int U>
static __device__ __forceinline__ void cta_pcg_fp64(const PcgArgs &a, const SysRange &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  SysState &S = a.st[g.s];
  const bool t0 = threadIdx.x == 0;
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
  cta_sum0<double, 4>(v, sh);
  // thread 0's scalars
  double rho = 0.0, bb = 0.0, thr = 0.0, rn = 0.0, rnorm0 = 0.0;
  int it = 0, status = -1;
  bool zero = false, timed = false;
  if (t0) {
    rho = v[0];
    bb = v[2];
    thr = C.rtol * sqrt(bb);
    rn = rnorm0 = sqrt(v[1]);
    if (v[3] > 0.0) status = GBS_ERR_NOT_SPD;
    else if (!isfinite(bb)) status = GBS_ERR_NAN;
    else if (bb == 0.0) {
      status = GBS_OK;
      zero = true;
      rn = rnorm0 = 0.0;
    } else if (!isfinite(v[1]) || !isfinite(rho)) status = GBS_ERR_NAN;
    else if (rn <= thr) status = GBS_OK;
    else if (C.maxit <= 0) status = GBS_ERR_MAXIT;
    sh.ipub[0] = status;
    sh.ipub[1] = zero;
  }
  cta_publish();
  int go = sh.ipub[0] < 0;
  const bool zero_x = sh.ipub[1] != 0;
  while (go) {
    // A: q = A p, p.q -> alpha
    double pq[1] = {0.0};
    auto fa = [&](int r, double qv) {
      a.q[r] = qv;
      pq[0] = fma(a.p[r], qv, pq[0]);
    };
    cta_rows<double>(a, g, a.sval, a.p, fa);
    cta_sum0<double, 1>(pq, sh);
    if (t0) {
      ++it;
      if (isnan(pq[0])) status = GBS_ERR_NAN;
      else if (!(pq[0] > 0.0)) status = GBS_ERR_BREAKDOWN;
      else sh.pub[0] = rho / pq[0];
      sh.ipub[0] = status;
    }
    cta_publish();
    if (sh.ipub[0] >= 0) break;
    const double al = sh.pub[0];
    // B: x += alpha p, r -= alpha q, z = D^-1 r (over q), r.z, r.r -> tests, beta
    double w[2] = {0.0, 0.0};
    {
      double qv[U], rv0[U], dv[U], pv[U], xv[U];
      auto ld = [&](int r, int k) {
        qv[k] = a.q[r];
        rv0[k] = a.r[r];
        dv[k] = a.dinv[r];
        pv[k] = a.p[r];
        xv[k] = x[r];
      };
      auto use = [&](int r, int k) {
        const double rv = fma(-al, qv[k], rv0[k]);
        const double z = dv[k] * rv;
        x[r] = fma(al, pv[k], xv[k]);
        a.r[r] = rv;
        a.q[r] = z;
        w[0] = fma(rv, z, w[0]);
        w[1] = fma(rv, rv, w[1]);
      };
      cta_rows_by<U>(g.r0, g.r1, ld, use);
    }
    cta_sum0<double, 2>(w, sh);
    if (t0) {
      rn = sqrt(w[1]);
      if (!isfinite(rn) || !isfinite(w[0])) status = GBS_ERR_NAN;
      else if (rn <= thr) status = GBS_OK;
      else if (it >= C.maxit) status = GBS_ERR_MAXIT;
      else if (cta_timed_out(a.ctl, C.timeout_ns)) timed = true;
      else {
        sh.pub[0] = w[0] / rho;
        rho = w[0];
      }
      sh.ipub[0] = (status < 0 && !timed) ? -1 : 0;
    }
    cta_publish();
    if (sh.ipub[0] >= 0) break;
    const double be = sh.pub[0];
    // C: p = z + beta p (each thread its own rows: the rows B wrote)
    {
      double pv[U], zv[U];
      auto ld = [&](int r, int k) {
        pv[k] = a.p[r];
        zv[k] = a.q[r];
      };
      auto use = [&](int r, int k) { a.p[r] = fma(be, pv[k], zv[k]); };
      cta_rows_by<U>(g.r0, g.r1, ld, use);
    }
    __syncthreads();  // p complete before the next product gathers it
  }
  cta_store_state(a, S, status, timed, it, 0, bb, rnorm0, rn, zero);
  cta_true_residual(a, g, S, zero_x, sh);
}

// FP32 inner PCG under FP64 refinement, the oracle's order of steps.
template <int U>
static __device__ __forceinline__ void cta_pcg_refined(const PcgArgs &a, const SysRange &g, CtaShared &sh) {
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  SysState &S = a.st[g.s];
  const bool t0 = threadIdx.x == 0;
  double v[2] = {0.0, 0.0};  // b.b, missing diagonals
  if (!C.nonzero_guess)
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) x[r] = 0.0;
  for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x) {
    v[0] = fma(b[r], b[r], v[0]);
    v[1] += (a.dinv[r] == 0.0) ? 1.0 : 0.0;
  }
  cta_sum0<double, 2>(v, sh);  // (its barrier also orders the x writes before the first product)
  // thread 0's scalars
  double bb = 0.0, bnorm = 0.0, rnorm0 = 0.0, rn = 0.0, prev_rn = INFINITY;
  int status = -1, outer = 0, stall = 0, iters = 0;
  bool zero = false, timed = false;
  if (t0) {
    bb = v[0];
    bnorm = sqrt(bb);
    if (v[1] > 0.0) status = GBS_ERR_NOT_SPD;
    else if (!isfinite(bb)) status = GBS_ERR_NAN;
    else if (bb == 0.0) {
      status = GBS_OK;
      zero = true;
    }
    sh.ipub[0] = status;
    sh.ipub[1] = zero;
  }
  cta_publish();
  int go = sh.ipub[0] < 0;
  const bool zero_x = sh.ipub[1] != 0;
  while (go) {
    // outer FP64 residual r = b - A x -> the refinement tests, s = ||r||
    double rr[1] = {0.0};
    auto fo = [&](int r, double t) {
      const double rv = b[r] - t;
      a.r[r] = rv;
      rr[0] = fma(rv, rv, rr[0]);
    };
    cta_rows<double>(a, g, a.sval, x, fo);
    cta_sum0<double, 1>(rr, sh);
    if (t0) {
      rn = sqrt(rr[0]);
      if (outer == 0) rnorm0 = rn;
      if (!isfinite(rn)) status = GBS_ERR_NAN;
      else if (rn <= C.rtol * bnorm) status = GBS_OK;
      else if (outer >= C.max_outer) status = GBS_ERR_MAXIT;
      else if (outer > 0 && (stall = (rn > 0.5 * prev_rn) ? stall + 1 : 0) >= 2)
        status = GBS_ERR_STAGNATION;
      else if (cta_timed_out(a.ctl, C.timeout_ns)) timed = true;
      else {
        prev_rn = rn;
        sh.pub[0] = rn;
      }
      sh.ipub[0] = (status < 0 && !timed) ? -1 : 0;
    }
    cta_publish();
    if (sh.ipub[0] >= 0) break;
    const double s = sh.pub[0];
    // inner FP32 PCG on RN(r / s) from d = 0
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
    cta_sum0<float, 2>(w, sh);
    float rho = 0.0f;
    double thr = 0.0;
    int it = 0;
    if (t0) {
      rho = w[0];
      const double tgt = fmax(C.inner_rtol, 0.5 * C.rtol * bnorm / s);
      thr = tgt * (double)sqrtf(w[1]);
      sh.ipub[1] = (double)sqrtf(w[1]) > thr && 0 < C.inner_maxit;
    }
    cta_publish();
    int inner = sh.ipub[1];
    while (inner) {
      float pq[1] = {0.0f};
      auto fa = [&](int r, float qv) {
        a.q32[r] = qv;
        pq[0] = fmaf(a.p32[r], qv, pq[0]);
      };
      cta_rows<float>(a, g, a.sval32, a.p32, fa);
      cta_sum0<float, 1>(pq, sh);
      if (t0) {
        const bool ok = pq[0] > 0.0f;
        if (ok) {
          ++it;
          reinterpret_cast<float *>(sh.pub)[2] = rho / pq[0];
        }
        sh.ipub[1] = ok;
      }
      cta_publish();
      if (!sh.ipub[1]) break;
      const float al = reinterpret_cast<const float *>(sh.pub)[2];
      float u[2] = {0.0f, 0.0f};
      {
        float qv[U], rv0[U], dv[U], pv[U], d0[U];
        auto ld = [&](int r, int k) {
          qv[k] = a.q32[r];
          rv0[k] = a.r32[r];
          dv[k] = a.dinv32[r];
          pv[k] = a.p32[r];
          d0[k] = a.d32[r];
        };
        auto use = [&](int r, int k) {
          const float rv = fmaf(-al, qv[k], rv0[k]);
          const float z = dv[k] * rv;
          a.d32[r] = fmaf(al, pv[k], d0[k]);
          a.r32[r] = rv;
          a.q32[r] = z;
          u[0] = fmaf(rv, z, u[0]);
          u[1] = fmaf(rv, rv, u[1]);
        };
        cta_rows_by<U>(g.r0, g.r1, ld, use);
      }
      cta_sum0<float, 2>(u, sh);
      if (t0) {
        reinterpret_cast<float *>(sh.pub)[3] = u[0] / rho;
        rho = u[0];
        sh.ipub[1] = (double)sqrtf(u[1]) > thr && it < C.inner_maxit;
      }
      cta_publish();
      const float be = reinterpret_cast<const float *>(sh.pub)[3];
      inner = sh.ipub[1];
      {
        float pv[U], zv[U];
        auto ld = [&](int r, int k) {
          pv[k] = a.p32[r];
          zv[k] = a.q32[r];
        };
        auto use = [&](int r, int k) { a.p32[r] = fmaf(be, pv[k], zv[k]); };
        cta_rows_by<U>(g.r0, g.r1, ld, use);
      }
      __syncthreads();
    }
    if (t0) {
      iters += it;
      if (it == 0) status = GBS_ERR_BREAKDOWN;
      else ++outer;
      sh.ipub[0] = status;
    }
    cta_publish();
    if (sh.ipub[0] >= 0) break;
    for (int r = g.r0 + threadIdx.x; r < g.r1; r += blockDim.x)
      x[r] = fma(s, (double)a.d32[r], x[r]);
    __syncthreads();  // x complete before the next outer residual gathers it
  }
  cta_store_state(a, S, status, timed, iters, outer, bb, rnorm0, rn, zero);
  cta_true_residual(a, g, S, zero_x, sh);
}

// A persistent grid: CTA c solves system order[c], then takes the next
// unsolved one (order[grid], order[grid + 1], ... by an atomic counter) until
// none is left -- largest first, so the largest systems start at once and
// the rest fill the SMs as they free up (greedy list scheduling).
// CPS: CTAs per SM the grid runs.  The register budget follows (32 per
// thread for two, 64 for one), and with it the rows a thread keeps in flight
// in the element-wise loops (cta_rows_by): one for two CTAs per SM; for one,
// two FP64 rows or four FP32 rows.  Measured on a batch of 512 systems of
// 1k-200k rows: one CTA per SM, FP64 CG 2.14 s with one row in flight, 1.96
// with two, 2.03 with four, 2.31 with eight; the refined solve 1.75, 1.43,
// 1.39, 1.55 s; two CTAs per SM with two rows spill and slow down.
template <bool REFINED, int CPS>
__global__ void __launch_bounds__(CTA_TPB, CPS) k_cta_pcg(PcgArgs a) {
  constexpr int U = CPS == 1 ? (REFINED ? 4 : 2) : 1;
  __shared__ CtaShared sh;
  __shared__ int next;
  for (int k = blockIdx.x; k < a.cta_n;) {
    const SysRange g = cta_system(a, k);
    if (REFINED) cta_pcg_refined<U>(a, g, sh);
    else cta_pcg_fp64<U>(a, g, sh);
    __syncthreads();  // every thread is done with sh and with the system
    if (threadIdx.x == 0) next = (int)gridDim.x + atomicAdd(&a.ctl->queue, 1);
    __syncthreads();
    k = next;
  }
}

}  // namespace gbs
