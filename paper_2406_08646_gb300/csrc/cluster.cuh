// Jacobi-PCG with one thread-block cluster per system (Sec. 6.1 CG with
// device-resident scalars; Sec. 7 batched systems).
//
// The per-CTA solver (cta.cuh) keeps a system on one SM, which caps it at one
// SM's FP64 rate; the phase kernels spread a system over the whole GPU but
// pay a fixed cost per iteration for kernel boundaries and grid-wide
// reductions.  This engine takes the middle road: a cluster of up to 16 CTAs
// (one per SM) per system, the system's slices split evenly over them, every
// iteration inside one launch, and the reductions through distributed shared
// memory: each CTA sums its rows (block sum to warp 0), publishes the sum in
// its shared memory, one cluster barrier, and thread 0 of every CTA adds the
// cluster's sums in rank order -- so all CTAs hold the same totals and take
// the same decisions without another exchange.  Vectors one CTA writes and
// others gather (p, and x for the closing residual) are read through L2
// (GATHER_CG) after a cluster barrier, whose release / acquire semantics
// order the writes before the reads.
//
// Every decision is uniform over the cluster: it depends only on the summed
// totals (the wall-clock limit too: rank 0's verdict enters a sum), so every
// CTA executes the same sequence of cluster barriers.
#pragma once

#include <cooperative_groups.h>

#include "cta.cuh"

namespace gbs {

namespace cgrp = cooperative_groups;

constexpr int CLUSTER_MAX = 16;  // CTAs per cluster (16 needs the non-portable opt-in)

struct ClusterShared {
  double red[4 * CTA_TPB];         // block sums: every thread's values
  double lanes[BLOCK_SUMS_EXTRA];  // block sums: lane partials
  double part[2][4];               // this CTA's sums, two halves used in turn
  double pub[4];            // scalars published by thread 0
  int ipub[4];              // [0]: < 0 keep going; [1]: x = 0 (b = 0)
};

// Block sums of the CTA, then the cluster's sums in rank order: the totals
// are valid in thread 0 of every CTA, the same in all of them.  A half of
// `part` is rewritten two calls later, after the intervening call's cluster
// barrier, which no CTA passes before every CTA has read it.  Every call is
// followed by a CTA barrier (cta_publish) before the next one rewrites `red`.
template <int NV>
__device__ __forceinline__ void cluster_sum0(double (&v)[NV], ClusterShared &sh, int &half,
                                             const cgrp::cluster_group &cl) {
  block_sums<double, NV>(v, sh.red, sh.lanes);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh.part[half][k] = v[k];
  }
  cl.sync();
  if (threadIdx.x == 0) {
    const int nr = (int)cl.num_blocks();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int r = 0; r < nr; ++r) t += *cl.map_shared_rank(&sh.part[half][k], r);
      v[k] = t;
    }
  }
  half ^= 1;
}

// Rows [r0, r1) and slices [s0, s1) of this CTA's share of its system.
struct ClusterPart {
  int s0, s1, r0, r1;
};

__device__ __forceinline__ SysRange cluster_system(const PcgArgs &a, int cid) {
  SysRange g;
  if (a.ensemble) {
    g.s = 0;
    g.r0 = 0;
    g.r1 = __ldg(a.ta.row0 + a.ta.nblocks);
    g.s0 = 0;
    g.s1 = __ldg(a.ta.slice0 + a.ta.nblocks);
  } else {
    g.s = a.order ? __ldg(a.order + cid) : cid;
    const int b0 = __ldg(a.ta.sys_blk0 + g.s), b1 = __ldg(a.ta.sys_blk0 + g.s + 1);
    g.r0 = __ldg(a.ta.row0 + b0);
    g.r1 = __ldg(a.ta.row0 + b1);
    g.s0 = __ldg(a.ta.slice0 + b0);
    g.s1 = __ldg(a.ta.slice0 + b1);
  }
  return g;
}

__device__ __forceinline__ ClusterPart cluster_part(const PcgArgs &a, const SysRange &g,
                                                    int rank, int nrank) {
  const int64_t ns = g.s1 - g.s0;
  ClusterPart c;
  c.s0 = g.s0 + (int)(ns * rank / nrank);
  c.s1 = g.s0 + (int)(ns * (rank + 1) / nrank);
  c.r0 = __ldg(a.srow0 + c.s0);  // slice offsets end with nrows: valid for s <= nslices
  c.r1 = __ldg(a.srow0 + c.s1);
  return c;
}

template <int GATHER, class F>
__device__ __forceinline__ void cluster_rows(const PcgArgs &a, const ClusterPart &c,
                                             const double *x, F &f) {
  if (a.stream_matrix)
    sell_rows<double, true, GATHER>(a.sptr, a.srow0, a.scol, a.soff, a.sval, x, c.s0, c.s1,
                                    f);
  else sell_rows<double, false, GATHER>(a.sptr, a.srow0, a.scol, a.soff, a.sval, x, c.s0, c.s1, f);
}

// FP64 PCG of phases.cuh / cta.cuh, the system spread over a cluster.
__global__ void __launch_bounds__(CTA_TPB, 1) k_cluster_pcg(PcgArgs a) {
  __shared__ ClusterShared sh;
  const cgrp::cluster_group cl = cgrp::this_cluster();
  const int rank = (int)cl.block_rank(), nrank = (int)cl.num_blocks();
  const SysRange g = cluster_system(a, (int)(blockIdx.x / nrank));
  const ClusterPart c = cluster_part(a, g, rank, nrank);
  const CallArgs &C = *a.call;
  const double *b = C.b;
  double *x = C.x;
  const bool t0 = threadIdx.x == 0;
  int half = 0;
  // setup: r = b - A x0, z = D^-1 r, p = z over this CTA's rows
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
    cluster_rows<GATHER_CA>(a, c, x, row);  // x is written by no CTA before this
  } else {
    for (int r = c.r0 + threadIdx.x; r < c.r1; r += blockDim.x) {
      x[r] = 0.0;
      row(r, 0.0);
    }
  }
  cluster_sum0<4>(v, sh, half, cl);  // (its cluster barrier also publishes p)
  // thread 0's scalars (the same in every CTA of the cluster)
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
  const bool zero_x = sh.ipub[1] != 0;
  int go = sh.ipub[0] < 0;
  while (go) {
    // A: q = A p (p gathered through L2), p.q -> alpha
    double pq[1] = {0.0};
    auto fa = [&](int r, double qv) {
      a.q[r] = qv;
      pq[0] = fma(a.p[r], qv, pq[0]);
    };
    cluster_rows<GATHER_CG>(a, c, a.p, fa);
    cluster_sum0<1>(pq, sh, half, cl);
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
    // B: x += alpha p, r -= alpha q, z = D^-1 r (over q), r.z, r.r, and
    // rank 0's wall-clock verdict
    double w[3] = {0.0, 0.0, 0.0};
    if (t0 && rank == 0 && cta_timed_out(a.ctl, C.timeout_ns)) w[2] = 1.0;
    for (int r = c.r0 + threadIdx.x; r < c.r1; r += blockDim.x) {
      const double rv = fma(-al, a.q[r], a.r[r]);
      const double z = a.dinv[r] * rv;
      x[r] = fma(al, a.p[r], x[r]);
      a.r[r] = rv;
      a.q[r] = z;
      w[0] = fma(rv, z, w[0]);
      w[1] = fma(rv, rv, w[1]);
    }
    cluster_sum0<3>(w, sh, half, cl);
    if (t0) {
      rn = sqrt(w[1]);
      if (!isfinite(rn) || !isfinite(w[0])) status = GBS_ERR_NAN;
      else if (rn <= thr) status = GBS_OK;
      else if (it >= C.maxit) status = GBS_ERR_MAXIT;
      else if (w[2] > 0.0) timed = true;
      else {
        sh.pub[0] = w[0] / rho;
        rho = w[0];
      }
      sh.ipub[0] = (status < 0 && !timed) ? -1 : 0;
    }
    cta_publish();
    if (sh.ipub[0] >= 0) break;
    const double be = sh.pub[0];
    // C: p = z + beta p over this CTA's rows, then a cluster barrier: the
    // next product gathers p from every CTA
    for (int r = c.r0 + threadIdx.x; r < c.r1; r += blockDim.x) a.p[r] = fma(be, a.p[r], a.q[r]);
    cl.sync();
  }
  // closing residual ||b - A x||^2 (x = 0 where b = 0), gathered through L2
  if (zero_x)
    for (int r = c.r0 + threadIdx.x; r < c.r1; r += blockDim.x) x[r] = 0.0;
  cl.sync();
  double tt[1] = {0.0};
  auto ft = [&](int r, double t) {
    const double d = b[r] - t;
    tt[0] = fma(d, d, tt[0]);
  };
  cluster_rows<GATHER_CG>(a, c, x, ft);
  cluster_sum0<1>(tt, sh, half, cl);
  if (rank == 0) {
    SysState &S = a.st[g.s];
    cta_store_state(a, S, status, timed, it, 0, bb, rnorm0, rn, zero);
    if (t0) S.tt = tt[0];
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace gbs
