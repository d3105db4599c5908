// Persistent fused Jacobi-PCG (Sec. 6.1 CG with device-resident scalars and
// no host round trip; Sec. 7 diagonal preconditioning and batched systems;
// Sec. 2 A7 FP32 inner solve under FP64 refinement).
//
// One cooperative launch runs the whole solve.  Every warp is an independent
// worker with its own bulk-copy pipeline (pipe.cuh); global warp w takes
// blocks w, w+W, w+2W, ... of the phase's block table (SpMV blocks for
// products, larger update blocks for the vector updates; blocks never straddle
// two systems).  Per iteration:
//   A: q = A p (one FMA per nonzero) fused with the partial p.q     | barrier
//   B: x += alpha p, r -= alpha q, z = D^-1 r (stored over q),
//      partial r.z and r.r                                          | barrier
//   C: p = z + beta p                                               | barrier
// FP64 work per row and iteration is nnz_row + 7 FMA/MUL, the least the
// algorithm allows, because GB300's FP64 issue rate is about the same as the
// rate at which HBM delivers nonzeros.
//
// Reductions are deterministic: each warp reduces its rows of a system with a
// fixed shuffle tree and writes one slot per (system, worker); the warp whose
// slot arrives last (atomic arrival counter per system) sums the system's
// slots in slot order and updates that system's scalars (alpha, beta, norms,
// status).  Every warp reads them after the next grid barrier, so all take
// the same decisions and iteration counts are reproducible run to run.
// Converged systems are frozen (their blocks are skipped); the launch ends
// when no system is active.  A final phase recomputes ||b - A x|| per system.
//
// Refined mode (per-system state machine, M_* modes): an FP32 PCG on FP32
// copies of A and D^-1 with FP32 vectors and FP32 reductions solves
// A d = r / ||r||; between inner solves the same A/B/C slots run the FP64
// outer step: x += s d (slot C), r = b - A x and ||r|| (slot A), and the inner
// restart r32 = RN(r / s), d = 0 (slot B).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "device_util.cuh"
#include "internal.cuh"
#include "pipe.cuh"

namespace gbs {

enum { M_INNER = 0, M_XUPD = 1, M_START = 2 };
constexpr int SLOT_STRIDE = 4;  // doubles per reduction slot
constexpr int PCG_MAX_TPB = 512;

struct PcgArgs {
  int32_t nsys, ensemble;
  BlockTable ta, te;  // SpMV blocks, update blocks
  int32_t cap, Ra, Re, ns;
  int64_t stage_bytes;
  int64_t part_e;  // first reduction slot of table te
  const int32_t *row_ptr, *col;
  const double *val;
  const float *val32;
  const double *dinv;
  const float *dinv32;
  const double *b;
  double *x;
  double *r, *p, *q;
  float *r32, *p32, *q32, *d32;
  double *part;
  unsigned *sys_cnt;
  SysState *st;
  DevCtl *ctl;
  double rtol, inner_rtol;
  int32_t maxit, inner_maxit, max_outer, nonzero_guess;
  int64_t timeout_ns;
  int32_t barrier_extra;
  int64_t max_global;  // cap on loop trips: every trip advances each active system
};

__device__ __forceinline__ int sys_of(const PcgArgs &a, const BlockTable &t, int b) {
  return a.ensemble ? 0 : __ldg(t.sys + b);
}
__device__ __forceinline__ int sys_b0(const PcgArgs &a, const BlockTable &t, int s) {
  return a.ensemble ? 0 : __ldg(t.sys_blk0 + s);
}
__device__ __forceinline__ int sys_nblk(const PcgArgs &a, const BlockTable &t, int s) {
  return a.ensemble ? t.nblocks : __ldg(t.sys_blk0 + s + 1) - __ldg(t.sys_blk0 + s);
}
__device__ __forceinline__ int64_t sys_slot0(const PcgArgs &a, const BlockTable &t, int s) {
  return a.ensemble ? 0 : (int64_t)__ldg(t.sys_slot0 + s);
}

__device__ __forceinline__ void deactivate(const PcgArgs &a, SysState &S, int status) {
  S.status = status;
  S.active = 0;
  atomicSub(&a.ctl->n_active, 1);
}

template <typename T, int NV>
__device__ __forceinline__ void warp_sum(T (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(FULL_MASK, v[k], off);
}

// Reduce the warp's NV partials over its run on system s (last block b of
// table t) into the system's slot; the last arriving worker sums all slots in
// slot order and calls fin(s, totals) on lane 0.  f32: FP32 accumulation.
template <int NV, class Fin>
__device__ __forceinline__ void wflush(const PcgArgs &a, const BlockTable &t, int64_t part_off,
                                       int s, int b, int W, double (&acc)[NV], bool f32,
                                       Fin &fin) {
  const int lane = threadIdx.x & 31;
  if (f32) {
    float v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = (float)acc[k];
    warp_sum<float, NV>(v);
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = (double)v[k];
  } else {
    warp_sum<double, NV>(acc);
  }
  const int b0 = sys_b0(a, t, s), nb = sys_nblk(a, t, s);
  const int ns = min(nb, W);
  const int slot = (b - b0) % W;
  const int64_t base = part_off + sys_slot0(a, t, s);
  int last = 0;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) a.part[(base + slot) * SLOT_STRIDE + k] = acc[k];
    __threadfence();
    const unsigned prev = atomicAdd(a.sys_cnt + s, 1u);
    last = (prev == (unsigned)(ns - 1)) ? 1 : 0;
  }
  last = __shfl_sync(FULL_MASK, last, 0);
  if (last) {
    __threadfence();
    if (f32) {
      float tot[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) tot[k] = 0.f;
      for (int i = lane; i < ns; i += 32)
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] += (float)ldcg(a.part + (base + i) * SLOT_STRIDE + k);
      warp_sum<float, NV>(tot);
      if (lane == 0) {
        double d[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) d[k] = (double)tot[k];
        a.sys_cnt[s] = 0u;
        fin(s, d);
        __threadfence();
      }
    } else {
      double tot[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) tot[k] = 0.0;
      for (int i = lane; i < ns; i += 32)
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] += ldcg(a.part + (base + i) * SLOT_STRIDE + k);
      warp_sum<double, NV>(tot);
      if (lane == 0) {
        a.sys_cnt[s] = 0u;
        fin(s, tot);
        __threadfence();
      }
    }
  }
  __syncwarp();
}

// One warp's pass over its wanted blocks of table t, through its pipeline
// (PIPE) or with plain loads.  work(s, d, stage, acc) processes block d of
// system s; partials are flushed when the system changes and at the end.
template <int NV, bool PIPE, class Want, class Issue, class Work, class Fin, class Load>
__device__ __forceinline__ void wwalk(const PcgArgs &a, const BlockTable &t, int64_t part_off,
                                      WarpPipe &P, int worker, int W, bool f32, Want &want,
                                      Issue &issue, Work &work, Fin &fin, Load &load_sys) {
  int cur_s = -1, cur_b = -1;
  double acc[NV > 0 ? NV : 1];
  auto on_block = [&](int b, const BlkDesc &d, unsigned char *stg) {
    const int s = sys_of(a, t, b);
    if (s != cur_s) {
      if constexpr (NV > 0) {
        if (cur_s >= 0) wflush<NV>(a, t, part_off, cur_s, cur_b, W, acc, f32, fin);
      }
      cur_s = s;
      load_sys(s);
#pragma unroll
      for (int k = 0; k < (NV > 0 ? NV : 1); ++k) acc[k] = 0.0;
    }
    cur_b = b;
    work(s, d, stg, acc);
  };
  if constexpr (PIPE) {
    warp_stream(P, t, worker, W, want, issue, on_block);
  } else {
    for (int b = worker; b < t.nblocks; b += W)
      if (want(b)) on_block(b, load_desc(t, b), P.stage(0));
  }
  if constexpr (NV > 0) {
    if (cur_s >= 0) wflush<NV>(a, t, part_off, cur_s, cur_b, W, acc, f32, fin);
  }
}

// Per-system "does this phase process system s", one-entry cache (the state
// it reads is not modified during the phase while this warp still has blocks
// of s to visit).
struct WantCache {
  int s = -1;
  bool v = false;
};

template <bool REFINED>
__global__ void __launch_bounds__(PCG_MAX_TPB) k_pcg(PcgArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int W = gridDim.x * nw, worker = blockIdx.x * nw + warp;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)nw * a.ns * a.stage_bytes);
  WarpPipe P{smem_raw + (size_t)warp * a.ns * a.stage_bytes, bars + warp * a.ns, a.ns, a.cap,
             a.Ra, a.Re, a.stage_bytes, 0u, &a.ctl->err, a.timeout_ns, policy_evict_first(),
             policy_evict_last()};
  if (lane == 0) P.init_barriers();
  __syncthreads();
  GridBarrier gb{&a.ctl->bar, &a.ctl->err, 0ull, a.timeout_ns, (unsigned)a.barrier_extra};
  // CTA 0 keeps the time spent in each phase (between grid barriers)
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  uint64_t t_mark = timer ? global_ns() : 0;
  int64_t t_acc[5] = {0, 0, 0, 0, 0};
  auto lap = [&](int k) {
    if (timer) {
      const uint64_t t = global_ns();
      t_acc[k] += (int64_t)(t - t_mark);
      t_mark = t;
    }
  };
  const NzRange z0(0, 0, 0);  // dummies for plain (unstaged) row products
  const SliceRange<int32_t> rq0(0, 0);
  const int64_t pa = 0, pe = a.part_e;  // slot regions of the two tables

  // warp-uniform copies of the current system's scalars (set by load_sys())
  double c_alpha = 0, c_beta = 0, c_scale = 0;
  int c_mode = M_INNER, c_first = 0, c_zero = 0;
  auto load_sys = [&](int s) {
    const SysState *S = a.st + s;
    c_alpha = ldcg(&S->alpha);
    c_beta = ldcg(&S->beta);
    c_scale = ldcg(&S->scale);
    c_mode = ldcg(&S->mode);
    c_first = ldcg(&S->first);
    c_zero = ldcg(&S->zero_x);
  };
  auto active_mode = [&](WantCache &wc, const BlockTable &t, int b, int mode) -> bool {
    const int s = sys_of(a, t, b);
    if (s != wc.s) {
      const SysState *S = a.st + s;
      wc.s = s;
      wc.v = ldcg(&S->active) != 0 && (mode < 0 || ldcg(&S->mode) == mode);
    }
    return wc.v;
  };
  auto no_issue = [&](const BlkDesc &, unsigned char *, uint64_t *) {};
  auto plain_row = [&](const double *xv, int r) -> double {
    return row_product<double, false>(P, nullptr, z0, rq0, a.row_ptr, a.col, a.val, xv, r);
  };

  // ---------------------------------------------------------------- setup
  {
    auto want = [&](int) -> bool { return true; };
    auto work = [&](int s, const BlkDesc &d, unsigned char *, double(&acc)[4]) {
      for (int r = d.r0 + lane; r < d.r1; r += 32) {
        const double bv = a.b[r];
        const double rv = a.nonzero_guess ? bv - plain_row(a.x, r) : bv;
        if (!a.nonzero_guess) a.x[r] = 0.0;
        const double dv = a.dinv[r];
        if (REFINED) {
          a.r[r] = rv;
          acc[0] = fma(rv, rv, acc[0]);
        } else {
          const double z = dv * rv;
          a.r[r] = rv;
          a.p[r] = z;
          acc[0] = fma(rv, z, acc[0]);
          acc[1] = fma(rv, rv, acc[1]);
        }
        acc[2] = fma(bv, bv, acc[2]);
        acc[3] += (dv == 0.0) ? 1.0 : 0.0;
      }
    };
    auto fin = [&](int s, double(&tot)[4]) {
      SysState &S = a.st[s];
      const double bb = tot[2], nbad = tot[3];
      const double rr = REFINED ? tot[0] : tot[1];
      const double rho = REFINED ? 0.0 : tot[0];
      memset(&S, 0, sizeof(SysState));
      S.bb = bb;
      S.rho = rho;
      S.rr = rr;
      S.rnorm0 = S.rnorm = sqrt(rr);
      int status = -1;
      if (nbad > 0.0) status = GBS_ERR_NOT_SPD;
      else if (!isfinite(bb)) status = GBS_ERR_NAN;
      else if (bb == 0.0) {
        status = GBS_OK;
        S.zero_x = 1;
        S.rnorm0 = S.rnorm = 0.0;
      } else if (!isfinite(rr) || !isfinite(rho)) status = GBS_ERR_NAN;
      else if (sqrt(rr) <= a.rtol * sqrt(bb)) status = GBS_OK;
      else if (REFINED ? (a.max_outer <= 0) : (a.maxit <= 0)) status = GBS_ERR_MAXIT;
      if (status >= 0) {
        S.status = status;
        S.active = 0;
      } else {
        S.status = GBS_OK;
        S.active = 1;
        if (REFINED) {
          S.prev_rn = S.rnorm;
          S.scale = S.rnorm;
          S.mode = M_START;
        }
        atomicAdd(&a.ctl->n_active, 1);
      }
    };
    wwalk<4, false>(a, a.ta, pa, P, worker, W, false, want, no_issue, work, fin, load_sys);
  }

  // ---------------------------------------------------------------- iterations
  // Each trip runs one A/B/C round for every active system; the trip cap is a
  // safety net (systems left active when it trips are reported as MAXIT).
  for (int64_t trip = 0;; ++trip) {
    const bool ok_top = gb.sync();
    lap(trip == 0 ? 0 : 3);
    if (!ok_top) break;
    if (ld_relaxed_s32(&a.ctl->n_active) == 0) break;
    if (trip >= a.max_global) break;

    // ---- slot A: q = A p and p.q (FP64, or FP32 inner); refined outer
    //      residual r = b - A x and ||r||^2 in FP64 (plain pass)
    {
      auto fin = [&](int s, double(&tot)[1]) {
        SysState &S = a.st[s];
        if (!REFINED) {
          const double sigma = tot[0];
          S.iterations += 1;
          if (isnan(sigma)) deactivate(a, S, GBS_ERR_NAN);
          else if (!(sigma > 0.0)) deactivate(a, S, GBS_ERR_BREAKDOWN);
          else S.alpha = S.rho / sigma;
        } else if (S.mode == M_INNER) {
          const float sigma = (float)tot[0];
          S.first = 0;
          if (!(sigma > 0.0f)) {
            if (S.inner_it == 0) deactivate(a, S, GBS_ERR_BREAKDOWN);
            else {
              S.mode = M_XUPD;
              S.outer += 1;
            }
          } else {
            S.alpha = (double)((float)S.rho / sigma);
            S.inner_it += 1;
            S.iterations += 1;
          }
        } else {  // outer residual
          const double rn = sqrt(tot[0]);
          S.rnorm = rn;
          if (!isfinite(rn)) deactivate(a, S, GBS_ERR_NAN);
          else if (rn <= a.rtol * sqrt(S.bb)) deactivate(a, S, GBS_OK);
          else if (S.outer >= a.max_outer) deactivate(a, S, GBS_ERR_MAXIT);
          else {
            S.stall = (rn > 0.5 * S.prev_rn) ? S.stall + 1 : 0;
            if (S.stall >= 2) deactivate(a, S, GBS_ERR_STAGNATION);
            else {
              S.prev_rn = rn;
              S.scale = rn;
              S.mode = M_START;
            }
          }
        }
      };
      if (!REFINED) {
        WantCache wc;
        auto want = [&](int b) -> bool { return active_mode(wc, a.ta, b, -1); };
        auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
          const SliceRange<double> q(d.r0, d.r1);
          if (arrive_for(bar, csr_bytes<double>(d, P.cap) + q.bytes())) {
            csr_copy<double>(P, st, d, a.row_ptr, a.col, a.val, bar);
            slice_copy<double>(P.SA(st), a.p, q, bar, P.pol_vec);
          }
        };
        auto work = [&](int s, const BlkDesc &d, unsigned char *st, double(&acc)[1]) {
          const SliceRange<double> q(d.r0, d.r1);
          auto f = [&](int r, double qv) {
            a.q[r] = qv;
            acc[0] = fma(slice_get<double>(P.SA(st), a.p, q, r), qv, acc[0]);
          };
          block_rows<double>(P, st, d, a.row_ptr, a.col, a.val, a.p, f);
        };
        wwalk<1, true>(a, a.ta, pa, P, worker, W, false, want, issue, work, fin, load_sys);
      } else {
        {  // inner FP32 SpMV, pipelined
          WantCache wc;
          auto want = [&](int b) -> bool { return active_mode(wc, a.ta, b, M_INNER); };
          auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
            const SliceRange<float> q(d.r0, d.r1);
            if (arrive_for(bar, csr_bytes<float>(d, P.cap) + q.bytes())) {
              csr_copy<float>(P, st, d, a.row_ptr, a.col, a.val32, bar);
              slice_copy<float>(P.SA(st), a.p32, q, bar, P.pol_vec);
            }
          };
          auto work = [&](int s, const BlkDesc &d, unsigned char *st, double(&acc)[1]) {
            const SliceRange<float> q(d.r0, d.r1);
            auto f = [&](int r, float qv) {
              a.q32[r] = qv;
              acc[0] = (double)fmaf(slice_get<float>(P.SA(st), a.p32, q, r), qv, (float)acc[0]);
            };
            block_rows<float>(P, st, d, a.row_ptr, a.col, a.val32, a.p32, f);
          };
          wwalk<1, true>(a, a.ta, pa, P, worker, W, true, want, issue, work, fin, load_sys);
        }
        {  // FP64 outer residual, plain
          WantCache wc;
          auto want = [&](int b) -> bool { return active_mode(wc, a.ta, b, M_XUPD); };
          auto work = [&](int s, const BlkDesc &d, unsigned char *, double(&acc)[1]) {
            for (int r = d.r0 + lane; r < d.r1; r += 32) {
              const double rv = a.b[r] - plain_row(a.x, r);
              a.r[r] = rv;
              acc[0] = fma(rv, rv, acc[0]);
            }
          };
          wwalk<1, false>(a, a.ta, pa, P, worker, W, false, want, no_issue, work, fin, load_sys);
        }
      }
    }
    const bool ok_a = gb.sync();
    lap(1);
    if (!ok_a) break;

    // ---- slot B: x += alpha p, r -= alpha q, z = D^-1 r (kept in q for slot
    //      C), r.z and r.r; or the refined inner restart
    {
      auto fin = [&](int s, double(&tot)[2]) {
        SysState &S = a.st[s];
        if (!REFINED) {
          const double rho_new = tot[0], rr = tot[1];
          const double rn = sqrt(rr);
          S.rr = rr;
          S.rnorm = rn;
          if (!isfinite(rn) || !isfinite(rho_new)) deactivate(a, S, GBS_ERR_NAN);
          else if (rn <= a.rtol * sqrt(S.bb)) deactivate(a, S, GBS_OK);
          else if (S.iterations >= a.maxit) deactivate(a, S, GBS_ERR_MAXIT);
          else {
            S.beta = rho_new / S.rho;
            S.rho = rho_new;
          }
        } else if (S.mode == M_START) {
          const float rho = (float)tot[0], rr = (float)tot[1];
          const float r0 = sqrtf(rr);
          S.rho = rho;
          S.rr = rr;
          S.r0in = r0;
          S.inner_it = 0;
          if (!((double)r0 > a.inner_rtol * (double)r0) || a.inner_maxit <= 0)
            deactivate(a, S, GBS_ERR_BREAKDOWN);
          else {
            S.mode = M_INNER;
            S.first = 1;
          }
        } else {  // M_INNER
          const float rho_new = (float)tot[0], rr = (float)tot[1];
          const float beta = rho_new / (float)S.rho;
          S.rho = rho_new;
          S.rr = rr;
          if (!((double)sqrtf(rr) > a.inner_rtol * S.r0in) || S.inner_it >= a.inner_maxit) {
            S.mode = M_XUPD;
            S.outer += 1;
          } else {
            S.beta = beta;
          }
        }
      };
      if (!REFINED) {
        WantCache wc;
        auto want = [&](int b) -> bool { return active_mode(wc, a.te, b, -1); };
        auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
          const SliceRange<double> q(d.r0, d.r1);
          if (arrive_for(bar, 5u * q.bytes())) {
            slice_copy<double>(P.SE(st, 0), a.p, q, bar, P.pol_vec);
            slice_copy<double>(P.SE(st, 1), a.q, q, bar, P.pol_vec);
            slice_copy<double>(P.SE(st, 2), a.x, q, bar, P.pol_vec);
            slice_copy<double>(P.SE(st, 3), a.r, q, bar, P.pol_vec);
            slice_copy<double>(P.SE(st, 4), a.dinv, q, bar, P.pol_vec);
          }
        };
        auto work = [&](int s, const BlkDesc &d, unsigned char *st, double(&acc)[2]) {
          const SliceRange<double> q(d.r0, d.r1);
          for (int r = d.r0 + lane; r < d.r1; r += 32) {
            const double pv = slice_get<double>(P.SE(st, 0), a.p, q, r);
            const double qv = slice_get<double>(P.SE(st, 1), a.q, q, r);
            const double xv = fma(c_alpha, pv, slice_get<double>(P.SE(st, 2), a.x, q, r));
            const double rv = fma(-c_alpha, qv, slice_get<double>(P.SE(st, 3), a.r, q, r));
            const double z = slice_get<double>(P.SE(st, 4), a.dinv, q, r) * rv;
            a.x[r] = xv;
            a.r[r] = rv;
            a.q[r] = z;
            acc[0] = fma(rv, z, acc[0]);
            acc[1] = fma(rv, rv, acc[1]);
          }
        };
        wwalk<2, true>(a, a.te, pe, P, worker, W, false, want, issue, work, fin, load_sys);
      } else {
        {  // inner FP32 update, pipelined
          WantCache wc;
          auto want = [&](int b) -> bool { return active_mode(wc, a.te, b, M_INNER); };
          auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
            const SliceRange<float> q(d.r0, d.r1);
            if (arrive_for(bar, 5u * q.bytes())) {
              slice_copy<float>(P.SE(st, 0), a.p32, q, bar, P.pol_vec);
              slice_copy<float>(P.SE(st, 1), a.q32, q, bar, P.pol_vec);
              slice_copy<float>(P.SE(st, 2), a.d32, q, bar, P.pol_vec);
              slice_copy<float>(P.SE(st, 3), a.r32, q, bar, P.pol_vec);
              slice_copy<float>(P.SE(st, 4), a.dinv32, q, bar, P.pol_vec);
            }
          };
          auto work = [&](int s, const BlkDesc &d, unsigned char *st, double(&acc)[2]) {
            const SliceRange<float> q(d.r0, d.r1);
            const float al = (float)c_alpha;
            float a0 = (float)acc[0], a1 = (float)acc[1];
            for (int r = d.r0 + lane; r < d.r1; r += 32) {
              const float pv = slice_get<float>(P.SE(st, 0), a.p32, q, r);
              const float qv = slice_get<float>(P.SE(st, 1), a.q32, q, r);
              const float dv = fmaf(al, pv, slice_get<float>(P.SE(st, 2), a.d32, q, r));
              const float rv = fmaf(-al, qv, slice_get<float>(P.SE(st, 3), a.r32, q, r));
              const float z = slice_get<float>(P.SE(st, 4), a.dinv32, q, r) * rv;
              a.d32[r] = dv;
              a.r32[r] = rv;
              a.q32[r] = z;
              a0 = fmaf(rv, z, a0);
              a1 = fmaf(rv, rv, a1);
            }
            acc[0] = (double)a0;
            acc[1] = (double)a1;
          };
          wwalk<2, true>(a, a.te, pe, P, worker, W, true, want, issue, work, fin, load_sys);
        }
        {  // inner restart on the scaled FP64 residual, plain
          WantCache wc;
          auto want = [&](int b) -> bool { return active_mode(wc, a.te, b, M_START); };
          auto work = [&](int s, const BlkDesc &d, unsigned char *, double(&acc)[2]) {
            float a0 = (float)acc[0], a1 = (float)acc[1];
            for (int r = d.r0 + lane; r < d.r1; r += 32) {
              const float rv = __double2float_rn(a.r[r] / c_scale);
              const float z = a.dinv32[r] * rv;
              a.r32[r] = rv;
              a.d32[r] = 0.0f;
              a.q32[r] = z;
              a0 = fmaf(rv, z, a0);
              a1 = fmaf(rv, rv, a1);
            }
            acc[0] = (double)a0;
            acc[1] = (double)a1;
          };
          wwalk<2, false>(a, a.te, pe, P, worker, W, true, want, no_issue, work, fin, load_sys);
        }
      }
    }
    const bool ok_b = gb.sync();
    lap(2);
    if (!ok_b) break;
    if (ld_relaxed_s32(&a.ctl->n_active) == 0) break;

    // ---- slot C (no reduction): p = z + beta p with z from slot B; refined
    //      x += s d
    {
      auto fin = [&](int, double(&)[1]) {};
      if (!REFINED) {
        WantCache wc;
        auto want = [&](int b) -> bool { return active_mode(wc, a.te, b, -1); };
        auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
          const SliceRange<double> q(d.r0, d.r1);
          if (arrive_for(bar, 2u * q.bytes())) {
            slice_copy<double>(P.SE(st, 0), a.p, q, bar, P.pol_vec);
            slice_copy<double>(P.SE(st, 1), a.q, q, bar, P.pol_vec);
          }
        };
        auto work = [&](int s, const BlkDesc &d, unsigned char *st, double(&)[1]) {
          const SliceRange<double> q(d.r0, d.r1);
          for (int r = d.r0 + lane; r < d.r1; r += 32) {
            const double pv = slice_get<double>(P.SE(st, 0), a.p, q, r);
            const double z = slice_get<double>(P.SE(st, 1), a.q, q, r);
            a.p[r] = fma(c_beta, pv, z);
          }
        };
        wwalk<0, true>(a, a.te, pe, P, worker, W, false, want, issue, work, fin, load_sys);
      } else {
        {
          WantCache wc;
          auto want = [&](int b) -> bool { return active_mode(wc, a.te, b, M_INNER); };
          auto issue = [&](const BlkDesc &d, unsigned char *st, uint64_t *bar) {
            const SliceRange<float> q(d.r0, d.r1);
            if (arrive_for(bar, 2u * q.bytes())) {
              slice_copy<float>(P.SE(st, 0), a.p32, q, bar, P.pol_vec);
              slice_copy<float>(P.SE(st, 1), a.q32, q, bar, P.pol_vec);
            }
          };
          auto work = [&](int s, const BlkDesc &d, unsigned char *st, double(&)[1]) {
            const SliceRange<float> q(d.r0, d.r1);
            const float be = (float)c_beta;
            for (int r = d.r0 + lane; r < d.r1; r += 32) {
              const float pv = slice_get<float>(P.SE(st, 0), a.p32, q, r);
              const float z = slice_get<float>(P.SE(st, 1), a.q32, q, r);
              a.p32[r] = c_first ? z : fmaf(be, pv, z);
            }
          };
          wwalk<0, true>(a, a.te, pe, P, worker, W, false, want, issue, work, fin, load_sys);
        }
        {  // x += s d, plain
          WantCache wc;
          auto want = [&](int b) -> bool { return active_mode(wc, a.te, b, M_XUPD); };
          auto work = [&](int s, const BlkDesc &d, unsigned char *, double(&)[1]) {
            for (int r = d.r0 + lane; r < d.r1; r += 32)
              a.x[r] = fma(c_scale, (double)a.d32[r], a.x[r]);
          };
          wwalk<0, false>(a, a.te, pe, P, worker, W, false, want, no_issue, work, fin, load_sys);
        }
      }
    }
  }

  // ---------------------------------------------------------------- true residual
  if (!gb.sync()) return;
  lap(0);
  {
    auto want = [&](int) -> bool { return true; };
    auto work = [&](int s, const BlkDesc &d, unsigned char *, double(&acc)[1]) {
      if (c_zero) {  // b_s == 0: x_s = 0 exactly, no product needed
        for (int r = d.r0 + lane; r < d.r1; r += 32) a.x[r] = 0.0;
        return;
      }
      for (int r = d.r0 + lane; r < d.r1; r += 32) {
        const double t = a.b[r] - plain_row(a.x, r);
        acc[0] = fma(t, t, acc[0]);
      }
    };
    auto fin = [&](int s, double(&tot)[1]) { a.st[s].tt = tot[0]; };
    wwalk<1, false>(a, a.ta, pa, P, worker, W, false, want, no_issue, work, fin, load_sys);
  }
  lap(4);
  if (timer)
    for (int k = 0; k < 5; ++k) a.ctl->phase_ns[k] = t_acc[k];
}

// ------------------------------------------------------------------ host side

static size_t pcg_smem_for(int nwarps, int ns, int64_t stage_bytes) {
  return (size_t)nwarps * ns * (size_t)stage_bytes + (size_t)nwarps * ns * 8;
}
static size_t pcg_smem(gbs_mat A) { return pcg_smem_for(A->nwarps, A->nstages, A->stage_bytes); }

static BlockTable view(const TableDev &t) {
  return BlockTable{t.nblocks, t.row0, t.nz0, t.sys, t.sys_blk0, t.sys_slot0};
}

template <bool REFINED>
static int raise_smem_limit(size_t smem) {
  cudaFuncAttributes fa;
  GBS_TRY_CUDA(cudaFuncGetAttributes(&fa, k_pcg<REFINED>));
  if (fa.maxDynamicSharedSizeBytes < (int)smem)
    GBS_TRY_CUDA(cudaFuncSetAttribute(k_pcg<REFINED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  return GBS_OK;
}

template <bool REFINED>
static int pcg_grid(gbs_mat A, int *grid) {
  const size_t smem = pcg_smem(A);
  GBS_TRY(raise_smem_limit<REFINED>(smem));
  int per_sm = 0, nsm = 0;
  GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<REFINED>, A->tpb, smem));
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device));
  if (per_sm < 1) {
    set_error("persistent PCG kernel does not fit on an SM (tpb %d, smem %zu)", A->tpb, smem);
    return GBS_ERR_LAUNCH;
  }
  // no more CTAs than the larger table has blocks for its warps
  const int64_t nb = std::max(A->ta.nblocks, A->te.nblocks);
  int64_t g = std::min<int64_t>((int64_t)per_sm * nsm, (nb + A->nwarps - 1) / A->nwarps);
  *grid = (int)std::max<int64_t>(g, 1);
  return GBS_OK;
}

// Slot offsets for W workers: system s owns min(nblocks_s, W) slots per table.
static int ensure_slots(gbs_mat A, int W, cudaStream_t s) {
  const int64_t need = std::max<int64_t>((int64_t)A->ta.nblocks + A->te.nblocks, 1) + 2;
  if (A->part_cap < need) {
    if (A->part) cudaFree(A->part);
    A->part = nullptr;
    GBS_TRY_CUDA(cudaMalloc(&A->part, sizeof(double) * SLOT_STRIDE * need));
    A->part_cap = need;
  }
  if (A->slot_workers != W) {
    for (TableDev *t : {&A->ta, &A->te}) {
      std::vector<int32_t> so(A->nsys + 1, 0);
      for (int32_t q = 0; q < A->nsys; ++q) {
        const int32_t nb = t->sys_blk0_h[q + 1] - t->sys_blk0_h[q];
        so[q + 1] = so[q] + std::min(nb, W);
      }
      GBS_TRY_CUDA(cudaMemcpyAsync(t->sys_slot0, so.data(), sizeof(int32_t) * (A->nsys + 1),
                                   cudaMemcpyHostToDevice, s));
      GBS_TRY_CUDA(cudaStreamSynchronize(s));  // `so` is pageable and goes out of scope
    }
    A->slot_workers = W;
  }
  return GBS_OK;
}

int ensure_solver_workspace(gbs_mat A, bool refined) {
  const size_t n = (size_t)std::max<int64_t>(A->nrows, 1);
  if (!A->r) {
    GBS_TRY_CUDA(cudaMalloc(&A->r, sizeof(double) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->p, sizeof(double) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->q, sizeof(double) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->sys_cnt, sizeof(unsigned) * A->nsys));
    GBS_TRY_CUDA(cudaMalloc(&A->st, sizeof(SysState) * A->nsys));
    GBS_TRY_CUDA(cudaMalloc(&A->ctl, sizeof(DevCtl)));
    GBS_TRY_CUDA(cudaMallocHost(&A->st_host, sizeof(SysState) * A->nsys));
    GBS_TRY_CUDA(cudaMemset(A->sys_cnt, 0, sizeof(unsigned) * A->nsys));
    GBS_TRY_CUDA(cudaMemset(A->ctl, 0, sizeof(DevCtl)));
    A->slot_workers = -1;
  }
  if (refined && !A->r32) {
    GBS_TRY_CUDA(cudaMalloc(&A->r32, sizeof(float) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->p32, sizeof(float) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->q32, sizeof(float) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->d32, sizeof(float) * n));
  }
  return GBS_OK;
}

static void fill_common(PcgArgs &a, const ksp_opts &o) {
  a.rtol = o.rtol;
  a.inner_rtol = o.inner_rtol;
  a.maxit = o.maxit;
  a.inner_maxit = o.inner_maxit;
  a.max_outer = o.max_outer;
  a.nonzero_guess = o.nonzero_guess;
  a.timeout_ns = o.timeout_ns;
  a.barrier_extra = o.debug_barrier_extra;
  a.max_global = o.precision == GBS_FP32_REFINED
                     ? ((int64_t)o.max_outer + 1) * ((int64_t)o.inner_maxit + 3) + 4
                     : (int64_t)o.maxit + 4;
}

static PcgArgs make_args(gbs_mat A, const double *b, double *x, const ksp_opts &o,
                         bool per_system) {
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.nsys = per_system ? A->nsys : 1;
  a.ensemble = per_system ? 0 : 1;
  a.ta = view(A->ta);
  a.te = view(A->te);
  a.cap = A->cap;
  a.Ra = A->Ra;
  a.Re = A->Re;
  a.ns = A->nstages;
  a.stage_bytes = A->stage_bytes;
  a.part_e = A->ta.nblocks + 1;
  a.row_ptr = A->row_ptr;
  a.col = A->col;
  a.val = A->val;
  a.val32 = A->val32;
  a.dinv = A->dinv;
  a.dinv32 = A->dinv32;
  a.b = b;
  a.x = x;
  a.r = A->r;
  a.p = A->p;
  a.q = A->q;
  a.r32 = A->r32;
  a.p32 = A->p32;
  a.q32 = A->q32;
  a.d32 = A->d32;
  a.part = A->part;
  a.sys_cnt = A->sys_cnt;
  a.st = A->st;
  a.ctl = A->ctl;
  fill_common(a, o);
  return a;
}

static int launch_coop(void (*kern)(PcgArgs), PcgArgs &a, int G, int tpb, size_t smem,
                       cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3((unsigned)tpb);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) {
    set_error("cooperative PCG launch (grid %d x %d, smem %zu): %s", G, tpb, smem,
              cudaGetErrorString(e));
    return e == cudaErrorCooperativeLaunchTooLarge ? GBS_ERR_LAUNCH : GBS_ERR_CUDA;
  }
  count_launches(1);
  return GBS_OK;
}

// Enqueue one solve: reset the control words, then the persistent launch.
static int enqueue_solve(gbs_mat A, PcgArgs &a, bool refined, int G, cudaStream_t s) {
  GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
  GBS_TRY_CUDA(cudaMemsetAsync(A->sys_cnt, 0, sizeof(unsigned) * A->nsys, s));
  return refined ? launch_coop(k_pcg<true>, a, G, A->tpb, pcg_smem(A), s)
                 : launch_coop(k_pcg<false>, a, G, A->tpb, pcg_smem(A), s);
}

int solve(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
          bool use_graph, cudaStream_t s) {
  const bool refined = o.precision == GBS_FP32_REFINED;
  GBS_TRY(ensure_solver_workspace(A, refined));
  if (refined && !A->val32_valid) GBS_TRY(launch_to_fp32(A, s));
  A->last_count = per_system ? A->nsys : 1;
  A->last_ensemble = !per_system;
  if (A->ta.nblocks == 0) {  // empty matrix: nothing to iterate
    GBS_TRY_CUDA(cudaMemsetAsync(A->st, 0, sizeof(SysState) * A->nsys, s));
    GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
    return GBS_OK;
  }
  int G = 0;
  GBS_TRY(refined ? pcg_grid<true>(A, &G) : pcg_grid<false>(A, &G));
  if (refined) A->grid_fp32 = G; else A->grid_fp64 = G;
  GBS_TRY(ensure_slots(A, G * A->nwarps, s));
  PcgArgs a = make_args(A, b, x, o, per_system);
  if (!use_graph) return enqueue_solve(A, a, refined, G, s);

  // CUDA graph of (memsets + cooperative launch), re-captured when the
  // arguments change, replayed otherwise.
  uint64_t key[8] = {(uint64_t)(uintptr_t)b, (uint64_t)(uintptr_t)x, 0, 0, 0, 0, 0, 0};
  memcpy(&key[2], &o.rtol, 8);
  memcpy(&key[3], &o.inner_rtol, 8);
  key[4] = ((uint64_t)(uint32_t)o.maxit << 32) | (uint32_t)o.inner_maxit;
  key[5] = ((uint64_t)(uint32_t)o.max_outer << 32) | ((uint32_t)o.nonzero_guess << 1) |
           (refined ? 1u : 0u);
  key[6] = (uint64_t)o.timeout_ns ^ ((uint64_t)o.debug_barrier_extra << 48);
  key[7] = ((uint64_t)G << 32) | (uint64_t)(per_system ? 1 : 0) | ((uint64_t)A->tpb << 8) |
           ((uint64_t)A->nstages << 20) | ((uint64_t)A->Ra << 24);
  if (!A->graph || memcmp(key, A->graph_key, sizeof(key)) != 0) {
    if (A->graph) {
      cudaGraphExecDestroy(A->graph);
      A->graph = nullptr;
    }
    cudaStream_t cs;
    GBS_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int st = GBS_OK;
    if (e == cudaSuccess) {
      st = enqueue_solve(A, a, refined, G, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess && st == GBS_OK) e = cudaGraphInstantiate(&A->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != GBS_OK) return st;
    if (e != cudaSuccess) {
      set_error("capturing the batched PCG graph: %s", cudaGetErrorString(e));
      A->graph = nullptr;
      return GBS_ERR_CUDA;
    }
    memcpy(A->graph_key, key, sizeof(key));
  }
  GBS_TRY_CUDA(cudaGraphLaunch(A->graph, s));
  return GBS_OK;
}

int read_results(gbs_mat A, ksp_result *res, int32_t count, cudaStream_t s) {
  const int32_t n = A->last_count;
  if (count < n) {
    set_error("ksp_get_result: %d results requested, the last solve produced %d", count, n);
    return GBS_ERR_ARG;
  }
  if (!A->st_host) {
    set_error("ksp_get_result: no solve has run on this matrix");
    return GBS_ERR_ARG;
  }
  DevCtl ctl;
  GBS_TRY_CUDA(cudaMemcpyAsync(A->st_host, A->st, sizeof(SysState) * n, cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaMemcpyAsync(&ctl, A->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaStreamSynchronize(s));
  int first = GBS_OK;
  for (int32_t q = 0; q < n; ++q) {
    const SysState &S = A->st_host[q];
    ksp_result &R = res[q];
    R.status = S.status;
    if (S.active) R.status = ctl.err ? ctl.err : GBS_ERR_MAXIT;  // stopped early
    R.iterations = S.iterations;
    R.outer_iterations = S.outer;
    R.reserved = 0;
    R.rnorm0 = S.rnorm0;
    R.rnorm = S.rnorm;
    const double bn = sqrt(S.bb);
    R.true_rel_residual = bn > 0.0 ? sqrt(S.tt) / bn : sqrt(S.tt);
    if (R.status != GBS_OK && first == GBS_OK) first = R.status;
  }
  if (first == GBS_OK && ctl.err) first = ctl.err;
  if (first != GBS_OK) set_error("solve finished with status %d", first);
  return first;
}

}  // namespace gbs

// ------------------------------------------------------------------ no-alloc solve
//
// ksp_solve_cg_noalloc: the same persistent FP64 PCG kernel, for callers that
// must not allocate device memory -- e.g. code that works inside a fixed
// memory budget owned by another allocator, or that cannot afford the device
// synchronisation cudaMalloc / cudaFree imply.  Its scratch (the r, p, q and
// D^-1 vectors, the block tables, the reduction slots and the control words)
// lives in one file-scope __device__ array of fixed size, so the call performs
// no allocation of any kind.  The caller passes the CSR matrix, b and x.
// Limit: n <= NOALLOC_MAX_ROWS rows (the array holds about 8.4 MB and stays
// resident on every GPU that loads the library until the process exits).
// All calls share the array: calls that overlap on the GPU (other streams,
// other host threads) race and must be serialised by the caller.  The first
// call on a device looks the array's device address up (cudaGetSymbolAddress,
// with that device current); make that first call before any stream capture.

namespace {

constexpr int64_t NOALLOC_MAX_ROWS = 262144;
constexpr int NOALLOC_RA = 32, NOALLOC_RE = 256, NOALLOC_NW = 8, NOALLOC_NS = 2;
constexpr int NOALLOC_CAP = 1024;  // staged nonzeros per 32-row block (longer: plain loads)
constexpr int64_t NOALLOC_MAX_BLK_A = NOALLOC_MAX_ROWS / NOALLOC_RA;
constexpr int64_t NOALLOC_MAX_BLK_E = NOALLOC_MAX_ROWS / NOALLOC_RE;

struct NoallocScratch {
  double r[NOALLOC_MAX_ROWS], p[NOALLOC_MAX_ROWS], q[NOALLOC_MAX_ROWS],
      dinv[NOALLOC_MAX_ROWS];
  double part[(NOALLOC_MAX_BLK_A + NOALLOC_MAX_BLK_E + 8) * gbs::SLOT_STRIDE];
  int32_t row0_a[NOALLOC_MAX_BLK_A + 4], nz0_a[NOALLOC_MAX_BLK_A + 4];
  int32_t row0_e[NOALLOC_MAX_BLK_E + 4], nz0_e[NOALLOC_MAX_BLK_E + 4];
  unsigned sys_cnt[4];
  gbs::SysState st[1];
  gbs::DevCtl ctl;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 256;
static void *g_noalloc_addr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device (looked up once
// per device).  In host code the array's name is only a host-side stand-in,
// never a device address, so it must not be handed to a kernel directly.
int noalloc_scratch(NoallocScratch **out) {
  int dev = 0;
  GBS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    gbs::set_error("ksp_solve_cg_noalloc: device ordinal %d out of range", dev);
    return GBS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      gbs::set_error("ksp_solve_cg_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
      return GBS_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<NoallocScratch *>(g_noalloc_addr[dev]);
  return GBS_OK;
}

// D^-1 from the caller's CSR (0 marks a missing or non-positive diagonal) and
// the two block tables (32-row SpMV blocks, 256-row update blocks).
__global__ void k_noalloc_prep(int64_t n, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, const double *__restrict__ val,
                               double *__restrict__ dinv, int32_t *__restrict__ row0_a,
                               int32_t *__restrict__ nz0_a, int32_t nba,
                               int32_t *__restrict__ row0_e, int32_t *__restrict__ nz0_e,
                               int32_t nbe) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t r = i0; r < n; r += stride) {
    double d = 0.0;
    for (int32_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q)
      if (col[q] == r) d = val[q];
    dinv[r] = (d > 0.0) ? 1.0 / d : 0.0;
  }
  for (int64_t b = i0; b <= nba; b += stride) {
    const int64_t r = b * NOALLOC_RA < n ? b * NOALLOC_RA : n;
    row0_a[b] = (int32_t)r;
    nz0_a[b] = row_ptr[r];
  }
  for (int64_t b = i0; b <= nbe; b += stride) {
    const int64_t r = b * NOALLOC_RE < n ? b * NOALLOC_RE : n;
    row0_e[b] = (int32_t)r;
    nz0_e[b] = row_ptr[r];
  }
}

}  // namespace

extern "C" int ksp_solve_cg_noalloc(int64_t n, const int32_t *row_ptr, const int32_t *col,
                                    const double *val, const double *b, double *x,
                                    const ksp_opts *o, ksp_result *res, void *stream) {
  using namespace gbs;
  if (n < 0 || n > NOALLOC_MAX_ROWS) {
    set_error("ksp_solve_cg_noalloc: n = %lld is outside [0, %lld], the size of the "
              "static scratch", (long long)n, (long long)NOALLOC_MAX_ROWS);
    return GBS_ERR_ARG;
  }
  if (n > 0 && (!row_ptr || !col || !val || !b || !x)) {
    set_error("ksp_solve_cg_noalloc: null CSR, b or x pointer");
    return GBS_ERR_ARG;
  }
  if ((((uintptr_t)row_ptr | (uintptr_t)col | (uintptr_t)val | (uintptr_t)b | (uintptr_t)x) &
       15u) != 0) {
    set_error("ksp_solve_cg_noalloc: row_ptr, col, val, b and x must be 16-byte aligned");
    return GBS_ERR_ARG;
  }
  ksp_opts oo;
  ksp_opts_default(&oo);
  if (o) oo = *o;
  if (oo.precision != GBS_FP64) {
    set_error("ksp_solve_cg_noalloc: only GBS_FP64 is supported");
    return GBS_ERR_ARG;
  }
  if (!(oo.rtol >= 0.0) || oo.debug_barrier_extra < 0) {
    set_error("ksp_solve_cg_noalloc: invalid options");
    return GBS_ERR_ARG;
  }
  if (oo.maxit < 0) oo.maxit = (int32_t)std::min<int64_t>(10 * std::max<int64_t>(n, 1), 100000);
  if (oo.timeout_ns <= 0) oo.timeout_ns = 2000000000LL;
  if (n == 0) {
    if (res) memset(res, 0, sizeof(*res));
    return GBS_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NoallocScratch *S = nullptr;
  GBS_TRY(noalloc_scratch(&S));
  const int32_t nba = (int32_t)((n + NOALLOC_RA - 1) / NOALLOC_RA);
  const int32_t nbe = (int32_t)((n + NOALLOC_RE - 1) / NOALLOC_RE);
  const int64_t sb = std::max((spmv_stage_bytes(NOALLOC_CAP, NOALLOC_RA) + 15) & ~15LL,
                              (upd_stage_bytes(NOALLOC_RE) + 15) & ~15LL);
  const size_t smem = pcg_smem_for(NOALLOC_NW, NOALLOC_NS, sb);
  int per_sm = 0, nsm = 0, dev = 0;
  GBS_TRY_CUDA(cudaGetDevice(&dev));
  GBS_TRY(raise_smem_limit<false>(smem));
  GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<false>,
                                                             32 * NOALLOC_NW, smem));
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) {
    set_error("ksp_solve_cg_noalloc: persistent kernel does not fit on an SM");
    return GBS_ERR_LAUNCH;
  }
  const int G = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)per_sm * nsm, (nba + NOALLOC_NW - 1) / NOALLOC_NW));

  // the control words and arrival counters must start at zero on every call
  GBS_TRY_CUDA(cudaMemsetAsync(&S->ctl, 0, sizeof(DevCtl), s));
  GBS_TRY_CUDA(cudaMemsetAsync(S->sys_cnt, 0, sizeof(S->sys_cnt), s));
  k_noalloc_prep<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
      n, row_ptr, col, val, S->dinv, S->row0_a, S->nz0_a, nba, S->row0_e, S->nz0_e, nbe);
  GBS_LAUNCHED(1);

  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.nsys = 1;
  a.ensemble = 1;
  a.ta = BlockTable{nba, S->row0_a, S->nz0_a, nullptr, nullptr, nullptr};
  a.te = BlockTable{nbe, S->row0_e, S->nz0_e, nullptr, nullptr, nullptr};
  a.cap = NOALLOC_CAP;
  a.Ra = NOALLOC_RA;
  a.Re = NOALLOC_RE;
  a.ns = NOALLOC_NS;
  a.stage_bytes = sb;
  a.part_e = nba + 1;
  a.row_ptr = row_ptr;
  a.col = col;
  a.val = val;
  a.dinv = S->dinv;
  a.b = b;
  a.x = x;
  a.r = S->r;
  a.p = S->p;
  a.q = S->q;
  a.part = S->part;
  a.sys_cnt = S->sys_cnt;
  a.st = S->st;
  a.ctl = &S->ctl;
  fill_common(a, oo);
  GBS_TRY(launch_coop(k_pcg<false>, a, G, 32 * NOALLOC_NW, smem, s));
  if (!res) return GBS_OK;

  SysState st;
  DevCtl ctl;
  GBS_TRY_CUDA(cudaMemcpyAsync(&st, S->st, sizeof(SysState), cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaMemcpyAsync(&ctl, &S->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaStreamSynchronize(s));
  res->status = st.active ? (ctl.err ? ctl.err : GBS_ERR_MAXIT) : st.status;
  res->iterations = st.iterations;
  res->outer_iterations = 0;
  res->reserved = 0;
  res->rnorm0 = st.rnorm0;
  res->rnorm = st.rnorm;
  const double bn = sqrt(st.bb);
  res->true_rel_residual = bn > 0.0 ? sqrt(st.tt) / bn : sqrt(st.tt);
  if (res->status != GBS_OK) set_error("ksp_solve_cg_noalloc: solve ended with status %d", res->status);
  return res->status;
}
