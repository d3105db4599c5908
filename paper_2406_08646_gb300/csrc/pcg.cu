// Persistent fused Jacobi-PCG (Sec. 6.1 CG with device-resident scalars and
// no host round trip; Sec. 7 diagonal preconditioning and batched systems;
// Sec. 2 A7 FP32 inner solve under FP64 refinement).
//
// One cooperative launch runs the whole solve.  Rows are cut into work blocks
// of at most rows_per_block rows that never straddle two systems; CTA c
// handles blocks c, c+G, c+2G, ... in every phase.  Per iteration:
//   A: q = A p (staged CSR product) fused with the partial p.q      | barrier
//   B: x += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r     | barrier
//   C: p = z + beta p                                               | barrier
// Reductions are deterministic: each CTA reduces its rows of a system in a
// fixed tree and writes one slot per (system, CTA); the CTA whose slot arrives
// last (atomic arrival counter per system) sums the system's slots in slot
// order and updates that system's scalars (alpha, beta, norms, status).  Every
// CTA then reads those scalars after the next grid barrier, so all CTAs take
// the same decisions and iteration counts are reproducible run to run.
// Converged systems are frozen (their blocks are skipped); the launch ends
// when no system is active.  A final phase recomputes ||b - A x|| per system.
//
// Refined mode (per system state machine; see the M_* modes): an FP32 PCG on
// FP32 copies of A and D^-1 with FP32 vectors and FP32 reductions solves
// A d = r / ||r||; between inner solves the same A/B/C slots run the FP64
// outer step: x += s d (slot C), r = b - A x and ||r|| (slot A), and the
// inner restart r32 = RN(r / s), d = 0 (slot B).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

enum { M_INNER = 0, M_XUPD = 1, M_START = 2 };
constexpr int SLOT_STRIDE = 4;  // doubles per reduction slot
constexpr int PCG_MAX_TPB = 512;

struct PcgArgs {
  int32_t nsys, nblocks, cap, ensemble;
  const int32_t *row_ptr, *col;
  const double *val;
  const float *val32;
  const double *dinv;
  const float *dinv32;
  const int32_t *blk_row0, *blk_sys, *sys_blk0, *sys_slot0;
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

__device__ __forceinline__ int sys_of(const PcgArgs &a, int b) {
  return a.ensemble ? 0 : __ldg(a.blk_sys + b);
}
__device__ __forceinline__ int sys_b0(const PcgArgs &a, int s) {
  return a.ensemble ? 0 : __ldg(a.sys_blk0 + s);
}
__device__ __forceinline__ int sys_nblk(const PcgArgs &a, int s) {
  return a.ensemble ? a.nblocks : __ldg(a.sys_blk0 + s + 1) - __ldg(a.sys_blk0 + s);
}
__device__ __forceinline__ int64_t sys_slot0(const PcgArgs &a, int s) {
  return a.ensemble ? 0 : (int64_t)__ldg(a.sys_slot0 + s);
}

__device__ __forceinline__ void deactivate(const PcgArgs &a, SysState &S, int status) {
  S.status = status;
  S.active = 0;
  atomicSub(&a.ctl->n_active, 1);
}

// Reduce NV per-thread partials of the CTA's run over system s (last block b)
// into the system's slot; the last arriving CTA sums all slots and calls
// fin(s, totals) on thread 0.  f32: FP32 accumulation throughout.
template <int NV, class Fin>
__device__ __forceinline__ void flush(const PcgArgs &a, int s, int b, double (&acc)[NV],
                                      double *red, bool f32, Fin &fin) {
  __shared__ int s_last;
  if (f32) {
    float v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = (float)acc[k];
    block_reduce<float, NV>(v, reinterpret_cast<float *>(red));
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = (double)v[k];
  } else {
    block_reduce<double, NV>(acc, red);
  }
  const int G = gridDim.x;
  const int b0 = sys_b0(a, s), nb = sys_nblk(a, s);
  const int ns = min(nb, G);
  const int slot = (b - b0) % G;
  const int64_t base = sys_slot0(a, s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) a.part[(base + slot) * SLOT_STRIDE + k] = acc[k];
    __threadfence();
    const unsigned prev = atomicAdd(a.sys_cnt + s, 1u);
    s_last = (prev == (unsigned)(ns - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (f32) {
      float tot[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) tot[k] = 0.f;
      for (int t = threadIdx.x; t < ns; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] += (float)ldcg(a.part + (base + t) * SLOT_STRIDE + k);
      block_reduce<float, NV>(tot, reinterpret_cast<float *>(red));
      if (threadIdx.x == 0) {
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
      for (int t = threadIdx.x; t < ns; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] += ldcg(a.part + (base + t) * SLOT_STRIDE + k);
      block_reduce<double, NV>(tot, red);
      if (threadIdx.x == 0) {
        a.sys_cnt[s] = 0u;
        fin(s, tot);
        __threadfence();
      }
    }
  }
  __syncthreads();
}

// Walk this CTA's blocks.  begin(s) -> 0 (skip system), 1 (FP64 run), 2 (FP32
// run, no flush is wanted when NV == 0).  body(s, r0, r1, acc) processes a
// block.  A run is flushed when the system changes and at the end.
template <int NV, class Begin, class Body, class Fin>
__device__ __forceinline__ void run_phase(const PcgArgs &a, double *red, Begin &begin,
                                          Body &body, Fin &fin) {
  int cur_s = -1, cur_b = -1, cur_kind = 0;
  double acc[NV > 0 ? NV : 1];
  for (int b = blockIdx.x; b < a.nblocks; b += gridDim.x) {
    const int s = sys_of(a, b);
    if (s != cur_s) {
      if constexpr (NV > 0) {
        if (cur_kind) flush<NV>(a, cur_s, cur_b, acc, red, cur_kind == 2, fin);
      }
      cur_s = s;
      cur_kind = begin(s);
#pragma unroll
      for (int k = 0; k < (NV > 0 ? NV : 1); ++k) acc[k] = 0.0;
    }
    if (!cur_kind) continue;
    cur_b = b;
    body(s, __ldg(a.blk_row0 + b), __ldg(a.blk_row0 + b + 1), acc);
  }
  if constexpr (NV > 0) {
    if (cur_kind) flush<NV>(a, cur_s, cur_b, acc, red, cur_kind == 2, fin);
  }
}

template <bool REFINED>
__global__ void __launch_bounds__(PCG_MAX_TPB) k_pcg(PcgArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *prod = reinterpret_cast<double *>(smem_raw);
  double *red = prod + a.cap;
  float *prod32 = reinterpret_cast<float *>(smem_raw);
  GridBarrier gb{&a.ctl->bar, &a.ctl->err, 0ull, a.timeout_ns, (unsigned)a.barrier_extra};
  const int tid = threadIdx.x;

  // CTA-uniform copies of the current system's scalars (set by begin()).
  double c_alpha = 0, c_beta = 0, c_scale = 0;
  int c_mode = M_INNER, c_first = 0;
  auto load_sys = [&](int s) -> bool {
    const SysState *S = a.st + s;
    c_alpha = ldcg(&S->alpha);
    c_beta = ldcg(&S->beta);
    c_scale = ldcg(&S->scale);
    c_mode = ldcg(&S->mode);
    c_first = ldcg(&S->first);
    return ldcg(&S->active) != 0;
  };

  // ---------------------------------------------------------------- setup
  {
    auto begin = [&](int s) -> int { return 1; };
    auto body = [&](int s, int r0, int r1, double(&acc)[4]) {
      double t = 0.0;
      if (a.nonzero_guess)
        t = staged_row_product<double>(a.row_ptr, a.col, a.val, a.x, r0, r1, prod, a.cap);
      const int r = r0 + tid;
      if (r < r1) {
        const double bv = a.b[r];
        const double rv = a.nonzero_guess ? bv - t : bv;
        if (!a.nonzero_guess) a.x[r] = 0.0;
        const double dv = a.dinv[r];
        if (REFINED) {
          a.r[r] = rv;
          acc[0] += rv * rv;
        } else {
          const double z = dv * rv;
          a.r[r] = rv;
          a.p[r] = z;
          acc[0] += rv * z;
          acc[1] += rv * rv;
        }
        acc[2] += bv * bv;
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
    run_phase<4>(a, red, begin, body, fin);
  }

  // ---------------------------------------------------------------- iterations
  // Each trip runs one A/B/C round for every active system; the trip cap is a
  // safety net (systems left active when it trips are reported as MAXIT).
  for (int64_t trip = 0;; ++trip) {
    if (!gb.sync()) break;
    if (ld_relaxed_s32(&a.ctl->n_active) == 0) break;
    if (trip >= a.max_global) break;

    // ---- slot A
    {
      auto begin = [&](int s) -> int {
        if (!load_sys(s)) return 0;
        if (!REFINED) return 1;
        if (c_mode == M_INNER) return 2;
        if (c_mode == M_XUPD) return 1;
        return 0;
      };
      auto body = [&](int s, int r0, int r1, double(&acc)[1]) {
        const int r = r0 + tid;
        if (!REFINED) {
          const double qv =
              staged_row_product<double>(a.row_ptr, a.col, a.val, a.p, r0, r1, prod, a.cap);
          if (r < r1) {
            a.q[r] = qv;
            acc[0] += a.p[r] * qv;
          }
        } else if (c_mode == M_INNER) {
          const float qv = staged_row_product<float>(a.row_ptr, a.col, a.val32, a.p32, r0, r1,
                                                     prod32, a.cap);
          if (r < r1) {
            a.q32[r] = qv;
            acc[0] = (double)((float)acc[0] + a.p32[r] * qv);
          }
        } else {  // M_XUPD: FP64 outer residual
          const double t =
              staged_row_product<double>(a.row_ptr, a.col, a.val, a.x, r0, r1, prod, a.cap);
          if (r < r1) {
            const double rv = a.b[r] - t;
            a.r[r] = rv;
            acc[0] += rv * rv;
          }
        }
      };
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
      run_phase<1>(a, red, begin, body, fin);
    }
    if (!gb.sync()) break;

    // ---- slot B
    {
      auto begin = [&](int s) -> int {
        if (!load_sys(s)) return 0;
        if (!REFINED) return 1;
        if (c_mode == M_INNER || c_mode == M_START) return 2;
        return 0;
      };
      auto body = [&](int s, int r0, int r1, double(&acc)[2]) {
        const int r = r0 + tid;
        if (r >= r1) return;
        if (!REFINED) {
          const double pv = a.p[r], qv = a.q[r];
          const double xv = a.x[r] + c_alpha * pv;
          const double rv = a.r[r] - c_alpha * qv;
          const double z = a.dinv[r] * rv;
          a.x[r] = xv;
          a.r[r] = rv;
          acc[0] += rv * z;
          acc[1] += rv * rv;
        } else if (c_mode == M_INNER) {
          const float al = (float)c_alpha;
          const float pv = a.p32[r], qv = a.q32[r];
          const float dv = a.d32[r] + al * pv;
          const float rv = a.r32[r] - al * qv;
          const float z = a.dinv32[r] * rv;
          a.d32[r] = dv;
          a.r32[r] = rv;
          acc[0] = (double)((float)acc[0] + rv * z);
          acc[1] = (double)((float)acc[1] + rv * rv);
        } else {  // M_START: inner restart on the scaled FP64 residual
          const float rv = __double2float_rn(a.r[r] / c_scale);
          const float z = a.dinv32[r] * rv;
          a.r32[r] = rv;
          a.d32[r] = 0.0f;
          acc[0] = (double)((float)acc[0] + rv * z);
          acc[1] = (double)((float)acc[1] + rv * rv);
        }
      };
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
      run_phase<2>(a, red, begin, body, fin);
    }
    if (!gb.sync()) break;
    if (ld_relaxed_s32(&a.ctl->n_active) == 0) break;

    // ---- slot C (no reduction)
    {
      auto begin = [&](int s) -> int {
        if (!load_sys(s)) return 0;
        if (!REFINED) return 1;
        return (c_mode == M_INNER || c_mode == M_XUPD) ? 1 : 0;
      };
      auto body = [&](int s, int r0, int r1, double(&acc)[1]) {
        const int r = r0 + tid;
        if (r >= r1) return;
        if (!REFINED) {
          a.p[r] = a.dinv[r] * a.r[r] + c_beta * a.p[r];
        } else if (c_mode == M_INNER) {
          const float z = a.dinv32[r] * a.r32[r];
          a.p32[r] = c_first ? z : z + (float)c_beta * a.p32[r];
        } else {  // M_XUPD: x += s d
          a.x[r] += c_scale * (double)a.d32[r];
        }
      };
      auto fin = [&](int s, double(&tot)[1]) {};
      run_phase<0>(a, red, begin, body, fin);
    }
  }

  // ---------------------------------------------------------------- true residual
  if (!gb.sync()) return;
  {
    int c_zero = 0;
    auto begin = [&](int s) -> int {
      c_zero = ldcg(&a.st[s].zero_x);
      return 1;
    };
    auto body = [&](int s, int r0, int r1, double(&acc)[1]) {
      const int r = r0 + tid;
      if (c_zero) {  // b_s == 0: x_s = 0 exactly, no product needed
        if (r < r1) a.x[r] = 0.0;
        return;
      }
      const double t =
          staged_row_product<double>(a.row_ptr, a.col, a.val, a.x, r0, r1, prod, a.cap);
      if (r < r1) {
        const double d = a.b[r] - t;
        acc[0] += d * d;
      }
    };
    auto fin = [&](int s, double(&tot)[1]) {
      SysState &S = a.st[s];
      S.tt = tot[0];
    };
    run_phase<1>(a, red, begin, body, fin);
  }
}

// ------------------------------------------------------------------ host side

static size_t pcg_smem(gbs_mat A) { return (size_t)A->cap * sizeof(double) + 4 * 32 * sizeof(double); }

template <bool REFINED>
static int pcg_grid(gbs_mat A, int *grid) {
  static int configured_smem[2] = {0, 0};
  const size_t smem = pcg_smem(A);
  if ((int)smem > configured_smem[REFINED]) {
    GBS_TRY_CUDA(cudaFuncSetAttribute(k_pcg<REFINED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    configured_smem[REFINED] = (int)smem;
  }
  int per_sm = 0, nsm = 0;
  GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<REFINED>, A->tpb, smem));
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device));
  if (per_sm < 1) {
    set_error("persistent PCG kernel does not fit on an SM (tpb %d, smem %zu)", A->tpb, smem);
    return GBS_ERR_LAUNCH;
  }
  int64_t g = (int64_t)per_sm * nsm;
  if (g > A->nblocks) g = A->nblocks;
  if (g < 1) g = 1;
  *grid = (int)g;
  return GBS_OK;
}

// Slot offsets for grid size G: system s owns min(nblocks_s, G) slots.
static int ensure_slots(gbs_mat A, int G, cudaStream_t s) {
  const int64_t need = std::max<int64_t>((int64_t)A->nblocks, 1) + G;
  if (A->part_cap < need) {
    if (A->part) cudaFree(A->part);
    A->part = nullptr;
    GBS_TRY_CUDA(cudaMalloc(&A->part, sizeof(double) * SLOT_STRIDE * need));
    A->part_cap = need;
  }
  if (A->slot_grid != G) {
    std::vector<int32_t> so(A->nsys + 1, 0);
    for (int32_t q = 0; q < A->nsys; ++q) {
      const int32_t nb = A->sys_blk0_h[q + 1] - A->sys_blk0_h[q];
      so[q + 1] = so[q] + std::min(nb, G);
    }
    GBS_TRY_CUDA(cudaMemcpyAsync(A->sys_slot0, so.data(), sizeof(int32_t) * (A->nsys + 1),
                                 cudaMemcpyHostToDevice, s));
    GBS_TRY_CUDA(cudaStreamSynchronize(s));  // `so` is pageable and goes out of scope
    A->slot_grid = G;
  }
  return GBS_OK;
}

int ensure_solver_workspace(gbs_mat A, bool refined) {
  const size_t n = (size_t)std::max<int64_t>(A->nrows, 1);
  if (!A->r) {
    GBS_TRY_CUDA(cudaMalloc(&A->r, sizeof(double) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->p, sizeof(double) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->q, sizeof(double) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->sys_slot0, sizeof(int32_t) * (A->nsys + 1)));
    GBS_TRY_CUDA(cudaMalloc(&A->sys_cnt, sizeof(unsigned) * A->nsys));
    GBS_TRY_CUDA(cudaMalloc(&A->st, sizeof(SysState) * A->nsys));
    GBS_TRY_CUDA(cudaMalloc(&A->ctl, sizeof(DevCtl)));
    GBS_TRY_CUDA(cudaMallocHost(&A->st_host, sizeof(SysState) * A->nsys));
    GBS_TRY_CUDA(cudaMemset(A->sys_cnt, 0, sizeof(unsigned) * A->nsys));
    A->slot_grid = -1;
  }
  if (refined && !A->r32) {
    GBS_TRY_CUDA(cudaMalloc(&A->r32, sizeof(float) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->p32, sizeof(float) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->q32, sizeof(float) * n));
    GBS_TRY_CUDA(cudaMalloc(&A->d32, sizeof(float) * n));
  }
  return GBS_OK;
}

static PcgArgs make_args(gbs_mat A, const double *b, double *x, const ksp_opts &o,
                         bool per_system) {
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.nsys = per_system ? A->nsys : 1;
  a.ensemble = per_system ? 0 : 1;
  a.nblocks = A->nblocks;
  a.cap = A->cap;
  a.row_ptr = A->row_ptr;
  a.col = A->col;
  a.val = A->val;
  a.val32 = A->val32;
  a.dinv = A->dinv;
  a.dinv32 = A->dinv32;
  a.blk_row0 = A->blk_row0;
  a.blk_sys = A->blk_sys;
  a.sys_blk0 = A->sys_blk0;
  a.sys_slot0 = A->sys_slot0;
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
  return a;
}

template <bool REFINED>
static int launch_pcg(gbs_mat A, PcgArgs &a, int G, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3((unsigned)A->tpb);
  cfg.dynamicSmemBytes = pcg_smem(A);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_pcg<REFINED>, a);
  if (e != cudaSuccess) {
    set_error("cooperative PCG launch (grid %d x %d, smem %zu): %s", G, A->tpb, pcg_smem(A),
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
  return refined ? launch_pcg<true>(A, a, G, s) : launch_pcg<false>(A, a, G, s);
}

int solve(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
          bool use_graph, cudaStream_t s) {
  const bool refined = o.precision == GBS_FP32_REFINED;
  GBS_TRY(ensure_solver_workspace(A, refined));
  if (refined && !A->val32_valid) GBS_TRY(launch_to_fp32(A, s));
  A->last_count = per_system ? A->nsys : 1;
  A->last_ensemble = !per_system;
  if (A->nblocks == 0) {  // empty matrix: nothing to iterate
    GBS_TRY_CUDA(cudaMemsetAsync(A->st, 0, sizeof(SysState) * A->nsys, s));
    GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
    return GBS_OK;
  }
  int G = 0;
  GBS_TRY(refined ? pcg_grid<true>(A, &G) : pcg_grid<false>(A, &G));
  if (refined) A->grid_fp32 = G; else A->grid_fp64 = G;
  GBS_TRY(ensure_slots(A, G, s));
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
           ((uint64_t)A->cap << 20);
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
// D^-1 vectors, the block table, the reduction slots and the control words)
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
constexpr int NOALLOC_R = 256, NOALLOC_TPB = 256, NOALLOC_CAP = 2048;
constexpr int64_t NOALLOC_MAX_BLOCKS = NOALLOC_MAX_ROWS / NOALLOC_R;

struct NoallocScratch {
  double r[NOALLOC_MAX_ROWS], p[NOALLOC_MAX_ROWS], q[NOALLOC_MAX_ROWS],
      dinv[NOALLOC_MAX_ROWS];
  double part[(NOALLOC_MAX_BLOCKS + 8) * gbs::SLOT_STRIDE];
  int32_t blk_row0[NOALLOC_MAX_BLOCKS + 1];
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
// the block table of ceil(n / NOALLOC_R) blocks.
__global__ void k_noalloc_prep(int64_t n, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, const double *__restrict__ val,
                               double *__restrict__ dinv, int32_t *__restrict__ blk_row0,
                               int32_t nblocks) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    double d = 0.0;
    for (int32_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q)
      if (col[q] == r) d = val[q];
    dinv[r] = (d > 0.0) ? 1.0 / d : 0.0;
  }
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nblocks; b += stride)
    blk_row0[b] = (int32_t)(b * NOALLOC_R < n ? b * NOALLOC_R : n);
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
  const int32_t nblocks = (int32_t)((n + NOALLOC_R - 1) / NOALLOC_R);
  const size_t smem = (size_t)NOALLOC_CAP * sizeof(double) + 4 * 32 * sizeof(double);
  int per_sm = 0, nsm = 0, dev = 0;
  GBS_TRY_CUDA(cudaGetDevice(&dev));
  GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<false>, NOALLOC_TPB,
                                                             smem));
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) {
    set_error("ksp_solve_cg_noalloc: persistent kernel does not fit on an SM");
    return GBS_ERR_LAUNCH;
  }
  const int G = (int)std::min<int64_t>((int64_t)per_sm * nsm, nblocks);
  {  // the kernel's dynamic shared-memory limit may have been set lower by
     // another launch configuration; raise it if needed, never lower it
    cudaFuncAttributes fa;
    GBS_TRY_CUDA(cudaFuncGetAttributes(&fa, k_pcg<false>));
    if (fa.maxDynamicSharedSizeBytes < (int)smem)
      GBS_TRY_CUDA(cudaFuncSetAttribute(k_pcg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
  }

  // the control words and arrival counters must start at zero on every call
  GBS_TRY_CUDA(cudaMemsetAsync(&S->ctl, 0, sizeof(DevCtl), s));
  GBS_TRY_CUDA(cudaMemsetAsync(S->sys_cnt, 0, sizeof(S->sys_cnt), s));
  k_noalloc_prep<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
      n, row_ptr, col, val, S->dinv, S->blk_row0, nblocks);
  GBS_LAUNCHED(1);

  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.nsys = 1;
  a.ensemble = 1;
  a.nblocks = nblocks;
  a.cap = NOALLOC_CAP;
  a.row_ptr = row_ptr;
  a.col = col;
  a.val = val;
  a.dinv = S->dinv;
  a.blk_row0 = S->blk_row0;
  a.b = b;
  a.x = x;
  a.r = S->r;
  a.p = S->p;
  a.q = S->q;
  a.part = S->part;
  a.sys_cnt = S->sys_cnt;
  a.st = S->st;
  a.ctl = &S->ctl;
  a.rtol = oo.rtol;
  a.maxit = oo.maxit;
  a.nonzero_guess = oo.nonzero_guess;
  a.timeout_ns = oo.timeout_ns;
  a.barrier_extra = oo.debug_barrier_extra;
  a.max_global = (int64_t)oo.maxit + 4;

  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3((unsigned)NOALLOC_TPB);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_pcg<false>, a);
  if (e != cudaSuccess) {
    set_error("ksp_solve_cg_noalloc: cooperative launch failed: %s", cudaGetErrorString(e));
    return e == cudaErrorCooperativeLaunchTooLarge ? GBS_ERR_LAUNCH : GBS_ERR_CUDA;
  }
  count_launches(1);
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
