// Jacobi-PCG driver (Sec. 6.1 CG with device-resident scalars and no host
// round trip; Sec. 7 diagonal preconditioning and batched systems; Sec. 2 A7
// FP32 inner solve under FP64 refinement).  The phase bodies are in
// phases.cuh.
//
// A solve is one CUDA graph, built once per (precision, batched) shape and
// matrix plan and replayed for every call:
//
//   memset control words -> setup -> WHILE(cond) { A -> B -> C } -> final
//
// The WHILE body repeats while its condition is non-zero; the last CTA of
// phase C sets it on the device (cudaGraphSetConditional), so the count is
// decided where the scalars live and the host never waits inside the loop.
// The per-call arguments (b, x, tolerances, limits) sit in a small device
// struct written by a one-thread kernel ahead of the graph, so one
// instantiated graph serves every call.  Each phase is its own kernel at full
// occupancy: no CTA ever waits for another, so no in-kernel wait exists that
// could hang.
//
// With ksp_opts.host_loop, and always in ksp_solve_cg_noalloc (which may not
// instantiate a graph), the same phase kernels run from a host loop instead:
// trips are launched in chunks and each trip checks a stop flag written by
// the previous one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "device_util.cuh"
#include "internal.cuh"
#include "cta.cuh"
#include "phases.cuh"

namespace gbs {

// ------------------------------------------------------------------ kernels

// Kernels with row products (setup, A, final) on the sliced-ELL layout
// (L == 0) are held to 32 registers so that four 512-thread CTAs (64 warps)
// fit per SM: the sliced product is latency-bound and needs every warp slot
// to keep HBM busy.  MB = 2: the same kernels for plans that cap the grids at
// one or two CTAs per SM anyway, with 64 registers a thread (no spills; C2
// FP64 product phase at two CTAs per SM 62.9 -> 51.9 us per iteration with
// column patterns).
#define GBS_ROWS_BOUNDS(L, MB) __launch_bounds__(PHASE_TPB, (L) == 0 ? (MB) : 1)

template <bool REFINED, int L, int MB = SELL_MIN_CTAS>
__global__ void GBS_ROWS_BOUNDS(L, MB) k_pcg_setup(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t t = (int64_t)global_ns();
    a.ctl->t_start = t;
    a.ctl->stamp = t;
    a.ctl->last_phase = 0;
  }
  phase_setup<REFINED, L>(a, red);
}

template <bool REFINED, int L, int MB = SELL_MIN_CTAS>
__global__ void GBS_ROWS_BOUNDS(L, MB) k_pcg_spmv(PcgArgs a) {
  __shared__ double red[RED_SCRATCH1];
  if (!trip_live(a)) return;
  stamp_phase(a, 1);
  phase_A<REFINED, L>(a, red);
}

template <bool REFINED>
__global__ void __launch_bounds__(PHASE_TPB) k_pcg_update(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  if (!trip_live(a)) return;
  stamp_phase(a, 2);
  phase_B<REFINED>(a, red);
}

template <bool REFINED>
__global__ void __launch_bounds__(PHASE_TPB) k_pcg_direction(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  const bool live = trip_live(a);
  loop_control(a, live);
  if (!live) return;
  stamp_phase(a, 3);
  phase_C<REFINED>(a, red);
}

template <int L, int MB = SELL_MIN_CTAS>
__global__ void GBS_ROWS_BOUNDS(L, MB) k_pcg_final(PcgArgs a) {
  __shared__ double red[RED_SCRATCH];
  stamp_phase(a, 4);
  phase_final<L>(a, red);
  if (blockIdx.x == 0 && threadIdx.x == 0)
    a.ctl->phase_ns[4] += (int64_t)global_ns() - a.ctl->stamp;
}

// Writes the call arguments; with ctl, also stamps the solve's start (the
// per-CTA solver's time limit counts from it).
__global__ void k_put_call(CallArgs *dst, CallArgs v, DevCtl *ctl) {
  *dst = v;
  if (ctl) ctl->t_start = (int64_t)global_ns();
}

struct PhaseKernels {
  void (*setup)(PcgArgs);
  void (*spmv)(PcgArgs);
  void (*update)(PcgArgs);
  void (*direction)(PcgArgs);
  void (*final_)(PcgArgs);
};

template <bool R, int L, int MB = SELL_MIN_CTAS>
static PhaseKernels kernels_for() {
  return PhaseKernels{k_pcg_setup<R, L, MB>, k_pcg_spmv<R, L, MB>, k_pcg_update<R>,
                      k_pcg_direction<R>, k_pcg_final<L, MB>};
}

// wide: the plan caps the grids at one or two CTAs per SM (wide_rows), so the
// sliced-ELL row kernels compiled for two CTAs per SM run.
static PhaseKernels phase_kernels(bool refined, int lanes, bool wide = false) {
  if (lanes == GBS_SPMV_SELL && wide)
    return refined ? kernels_for<true, 0, 2>() : kernels_for<false, 0, 2>();
  switch (lanes) {
    case 1: return refined ? kernels_for<true, 1>() : kernels_for<false, 1>();
    case 2: return refined ? kernels_for<true, 2>() : kernels_for<false, 2>();
    case 8: return refined ? kernels_for<true, 8>() : kernels_for<false, 8>();
    case 4: return refined ? kernels_for<true, 4>() : kernels_for<false, 4>();
    case 32: return refined ? kernels_for<true, 32>() : kernels_for<false, 32>();
    default: return refined ? kernels_for<true, 0>() : kernels_for<false, 0>();
  }
}

// ------------------------------------------------------------------ host side

// CTAs per SM that fit at once for the kernels walking the SpMV table (setup,
// A, final) and the update table (B, C), FP64 and refined, for the plan's
// row-product kernel.
int phase_occupancy(int lanes, int *rows, int *upd) {
  const PhaseKernels K[2] = {phase_kernels(false, lanes), phase_kernels(true, lanes)};
  int r = 1 << 20, u = 1 << 20;
  for (const PhaseKernels &k : K) {
    for (void (*f)(PcgArgs) : {k.setup, k.spmv, k.final_}) {
      int n = 0;
      GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, PHASE_TPB, 0));
      r = std::min(r, n);
    }
    for (void (*f)(PcgArgs) : {k.update, k.direction}) {
      int n = 0;
      GBS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, PHASE_TPB, 0));
      u = std::min(u, n);
    }
  }
  *rows = std::max(r, 1);
  *upd = std::max(u, 1);
  return GBS_OK;
}

static BlockTable view(const TableDev &t) {
  return BlockTable{t.nblocks, t.row0, t.sys, t.sys_blk0, t.sys_slot0, t.slice0, t.row1, t.slice1};
}

void drop_graphs(gbs_mat A) {
  for (auto &row : A->graph)
    for (auto &g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

// The solver's buffers, allocated on the first solve that needs them (on
// stream s; the stream is synchronised after an allocation, so the buffers
// are ready for any stream).
int ensure_solver_workspace(gbs_mat A, bool refined, cudaStream_t s) {
  const size_t n = (size_t)std::max<int64_t>(A->nrows, 1);
  bool grew = false;
  if (!A->r) {
    GBS_TRY(dev_alloc(&A->r, n, s));
    GBS_TRY(dev_alloc(&A->p, n, s));
    GBS_TRY(dev_alloc(&A->q, n, s));
    GBS_TRY(dev_alloc(&A->sys_cnt, A->nsys, s));
    GBS_TRY(dev_alloc(&A->st, A->nsys, s));
    GBS_TRY(dev_alloc(&A->ctl, 1, s));
    GBS_TRY(dev_alloc(&A->call, 1, s));
    GBS_TRY_CUDA(cudaMallocHost(&A->st_host, sizeof(SysState) * A->nsys));
    GBS_TRY_CUDA(cudaMemsetAsync(A->sys_cnt, 0, sizeof(unsigned) * A->nsys, s));
    GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
    grew = true;
  }
  if (refined && !A->r32) {
    GBS_TRY(dev_alloc(&A->r32, n, s));
    GBS_TRY(dev_alloc(&A->p32, n, s));
    GBS_TRY(dev_alloc(&A->q32, n, s));
    GBS_TRY(dev_alloc(&A->d32, n, s));
    drop_graphs(A);  // a cached refined graph would hold null FP32 pointers
    grew = true;
  }
  // reduction slots: table A's, table E's, and a third region the size of
  // table E's for partial sums of E's slots
  const int64_t need = std::max(A->ta.nslots + 2 * A->te.nslots, A->sa.nslots + 2 * A->se.nslots) + 1;
  if (A->part_cap < need) {
    if (A->part) {
      GBS_TRY_CUDA(cudaStreamSynchronize(s));
      dev_free(A->part, s);
    }
    A->part = nullptr;
    A->part_cap = 0;
    GBS_TRY(dev_alloc(&A->part, SLOT_STRIDE * (size_t)need, s));
    A->part_cap = need;
    drop_graphs(A);  // cached graphs hold the old pointer
    grew = true;
  }
  // the one-kernel CG's flags, one per CTA of table A
  if (A->halo_cap < A->ta.grid) {
    if (A->halo_flags) {
      GBS_TRY_CUDA(cudaStreamSynchronize(s));
      dev_free(A->halo_flags, s);
    }
    A->halo_flags = nullptr;
    A->halo_cap = 0;
    GBS_TRY(dev_alloc(&A->halo_flags, (size_t)A->ta.grid, s));
    A->halo_cap = A->ta.grid;
    drop_graphs(A);
    grew = true;
  }
  if (grew) GBS_TRY_CUDA(cudaStreamSynchronize(s));
  return GBS_OK;
}

// Loop-trip cap: a safety net only (each trip advances every active system).
static int64_t max_trips_for(const ksp_opts &o) {
  if (o.method == GBS_KSP_PIPECG)  // an iteration, a confirmation and a restart at most
    return 3 * (int64_t)o.maxit + 8;
  return o.precision == GBS_FP32_REFINED
             ? ((int64_t)o.max_outer + 1) * ((int64_t)o.inner_maxit + 3) + 4
             : (int64_t)o.maxit + 4;
}

CallArgs call_args(const double *b, double *x, const ksp_opts &o) {
  CallArgs c;
  memset(&c, 0, sizeof(c));
  c.b = b;
  c.x = x;
  c.rtol = o.rtol;
  c.inner_rtol = o.inner_rtol;
  c.maxit = o.maxit;
  c.inner_maxit = o.inner_maxit;
  c.max_outer = o.max_outer;
  c.nonzero_guess = o.nonzero_guess;
  c.max_trips = max_trips_for(o);
  c.timeout_ns = o.timeout_ns > 0 ? o.timeout_ns : 0;
  return c;
}

int put_call(CallArgs *dst, const CallArgs &c, cudaStream_t s, DevCtl *ctl) {
  k_put_call<<<1, 1, 0, s>>>(dst, c, ctl);
  GBS_LAUNCHED(1);
  return GBS_OK;
}

PcgArgs make_args(gbs_mat A, bool per_system, bool refined) {
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.nsys = per_system ? A->nsys : 1;
  a.ensemble = per_system ? 0 : 1;
  a.ta = view(A->ta);
  a.te = view(A->te);
  a.part_e = A->ta.nslots;
  a.grid_a = A->ta.grid;
  a.grid_e = A->te.grid;
  a.row_ptr = A->row_ptr;
  a.col = A->col;
  a.val = A->val;
  a.val32 = A->val32;
  a.sv = sell_view(A);
  a.sval = A->sell_val;
  a.sval32 = A->sell_val32;
  a.stream_matrix = stream_matrix(A, refined ? 8 : 12);
  a.dinv = A->dinv;
  a.dinv32 = A->dinv32;
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
  a.call = A->call;
  a.halo_flags = A->halo_flags;
  a.halo_lo = A->halo_lo;
  a.halo_n = A->halo_n;
  if (A->kv)
    for (int k = 0; k < KRYLOV_NVEC; ++k) a.kv[k] = A->kv + (size_t)k * (size_t)A->nrows;
  if (A->At) {
    a.tv = sell_view(A->At);
    a.tval = A->At->sell_val;
  }
  return a;
}

static cudaKernelNodeParams kernel_node(void (*k)(PcgArgs), int grid, void **args) {
  cudaKernelNodeParams p = {};
  p.func = (void *)k;
  p.gridDim = dim3((unsigned)std::max(grid, 1));
  p.blockDim = dim3(PHASE_TPB);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  return p;
}

// CG's loop: setup, WHILE { A (table A), B, C (table E) }, final (table A).
static LoopPlan cg_plan(bool refined, int lanes, bool wide = false) {
  const PhaseKernels K = phase_kernels(refined, lanes, wide);
  LoopPlan P;
  memset(&P, 0, sizeof(P));
  P.npre = 1;
  P.pre[0] = K.setup;
  P.nbody = 3;
  P.body[0] = K.spmv;
  P.body[1] = K.update;
  P.body[2] = K.direction;
  P.body_e[1] = P.body_e[2] = true;
  P.npost = 1;
  P.post[0] = K.final_;
  return P;
}

// Trips per evaluation of the graph's WHILE condition.  Each evaluation costs
// about 4 us on GB300 (measured: the per-iteration time of CG, TFQMR and
// pipelined CG on 1k-262k-row problems drops by that much with 8 trips per
// body); the price is up to GRAPH_UNROLL - 1 trips after the last system has
// finished, whose kernels find no active system and return.  Every trip
// sets the condition; its value only falls (systems never reactivate), so
// the body's last trip decides.
constexpr int GRAPH_UNROLL = 8;

// The solve graph of a loop plan:
//   memset control words -> memset counters -> start-up kernels ->
//   WHILE { GRAPH_UNROLL copies of the body } -> closing kernels.
int build_loop_graph(gbs_mat A, const LoopPlan &P, PcgArgs a, cudaGraphExec_t *out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  GBS_TRY_CUDA(cudaGraphCreate(&g, 0));
  cudaError_t e = cudaSuccess;
  auto fail = [&](const char *what) {
    set_error("building the solve graph (%s): %s", what, cudaGetErrorString(e));
    cudaGraphDestroy(g);
    return GBS_ERR_CUDA;
  };
  cudaGraphConditionalHandle h;
  // default 1: the body runs at least once per launch; its first trip finds
  // every system the setup already retired frozen and clears the condition
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail("conditional handle");
  a.cond = h;
  a.stepped = 0;
  a.trip = 0;
  void *args[] = {&a};
  auto grid = [&](bool e_table) { return e_table ? a.grid_e : a.grid_a; };

  cudaGraphNode_t n_ctl, n_cnt, n_loop;
  cudaMemsetParams ms;
  memset(&ms, 0, sizeof(ms));
  ms.dst = A->ctl;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = sizeof(DevCtl) / 4;
  ms.height = 1;
  e = cudaGraphAddMemsetNode(&n_ctl, g, nullptr, 0, &ms);
  if (e != cudaSuccess) return fail("memset");
  ms.dst = A->sys_cnt;
  ms.width = (size_t)A->nsys;
  e = cudaGraphAddMemsetNode(&n_cnt, g, &n_ctl, 1, &ms);
  if (e != cudaSuccess) return fail("memset");
  // every system's state starts cleared (a system without rows is never
  // visited by a kernel and reports OK with no iterations)
  cudaGraphNode_t n_st;
  ms.dst = A->st;
  ms.width = sizeof(SysState) * (size_t)A->nsys / 4;
  e = cudaGraphAddMemsetNode(&n_st, g, &n_cnt, 1, &ms);
  if (e != cudaSuccess) return fail("memset");
  n_cnt = n_st;
  if (P.body_coop) {  // the one-kernel CG's flags start below every iteration number
    cudaGraphNode_t n_fl;
    ms.dst = A->halo_flags;
    ms.width = (size_t)A->ta.grid;
    e = cudaGraphAddMemsetNode(&n_fl, g, &n_cnt, 1, &ms);
    if (e != cudaSuccess) return fail("memset");
    n_cnt = n_fl;
  }
  cudaKernelNodeParams kp;
  cudaGraphNode_t prev = n_cnt;
  for (int k = 0; k < P.npre; ++k) {
    cudaGraphNode_t n;
    kp = kernel_node(P.pre[k], grid(P.pre_e[k]), args);
    e = cudaGraphAddKernelNode(&n, g, &prev, 1, &kp);
    if (e != cudaSuccess) return fail("start-up node");
    prev = n;
  }

  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};  // other members zeroed
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(&n_loop, g, &prev, nullptr, 1, &cp);
  if (e != cudaSuccess) return fail("conditional node");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  prev = nullptr;
  for (int k = 0; k < P.nbody * GRAPH_UNROLL; ++k) {
    cudaGraphNode_t n;
    kp = kernel_node(P.body[k % P.nbody], grid(P.body_e[k % P.nbody]), args);
    e = cudaGraphAddKernelNode(&n, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
    if (e != cudaSuccess) return fail("loop body node");
    if (P.body_coop) {
      cudaLaunchAttributeValue v;
      memset(&v, 0, sizeof(v));
      v.cooperative = 1;
      e = cudaGraphKernelNodeSetAttribute(n, cudaLaunchAttributeCooperative, &v);
      if (e != cudaSuccess) return fail("cooperative loop body node");
    }
    prev = n;
  }
  prev = n_loop;
  for (int k = 0; k < P.npost; ++k) {
    cudaGraphNode_t n;
    kp = kernel_node(P.post[k], grid(P.post_e[k]), args);
    e = cudaGraphAddKernelNode(&n, g, &prev, 1, &kp);
    if (e != cudaSuccess) return fail("closing node");
    prev = n;
  }

  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    set_error("instantiating the solve graph: %s", cudaGetErrorString(e));
    return GBS_ERR_CUDA;
  }
  return GBS_OK;
}

constexpr int STEP_CHUNK = 16;  // host-stepped loop: trips launched between stop checks

// The loop without a graph: trips are launched STEP_CHUNK at a time; each
// trip's kernels skip their work once the previous trip has stopped the loop
// (DevCtl::stop), and the host reads the stop flag after every chunk.  The
// control words must be zero and the call arguments in place; setup runs
// first, the closing kernels last.
int run_loop_stepped(const LoopPlan &P, PcgArgs a, int grid_a, int grid_e, int64_t cap,
                     DevCtl *ctl, cudaStream_t s) {
  a.stepped = 1;
  a.trip = 0;
  auto grid = [&](bool e_table) { return (unsigned)(e_table ? grid_e : grid_a); };
  for (int q = 0; q < P.npre; ++q) P.pre[q]<<<grid(P.pre_e[q]), PHASE_TPB, 0, s>>>(a);
  GBS_LAUNCHED(P.npre);
  for (int64_t t = 0;;) {
    for (int k = 0; k < STEP_CHUNK; ++k, ++t) {
      a.trip = (int32_t)(t & 1);
      for (int q = 0; q < P.nbody; ++q) {
        if (P.body_coop) {
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3(grid(P.body_e[q]));
          cfg.blockDim = dim3(PHASE_TPB);
          cfg.stream = s;
          cudaLaunchAttribute at;
          at.id = cudaLaunchAttributeCooperative;
          at.val.cooperative = 1;
          cfg.attrs = &at;
          cfg.numAttrs = 1;
          GBS_TRY_CUDA(cudaLaunchKernelEx(&cfg, P.body[q], a));
        } else {
          P.body[q]<<<grid(P.body_e[q]), PHASE_TPB, 0, s>>>(a);
        }
      }
      GBS_LAUNCHED(P.nbody);
    }
    int32_t stop = 0;  // written by the last trip launched, for the next one
    GBS_TRY_CUDA(cudaMemcpyAsync(&stop, &ctl->stop[t & 1], sizeof(stop), cudaMemcpyDeviceToHost, s));
    GBS_TRY_CUDA(cudaStreamSynchronize(s));
    if (stop || t > cap) break;
  }
  for (int q = 0; q < P.npost; ++q) P.post[q]<<<grid(P.post_e[q]), PHASE_TPB, 0, s>>>(a);
  GBS_LAUNCHED(P.npost);
  return GBS_OK;
}

// The per-CTA solver takes systems small enough that one SM iterates them
// faster than the phase kernels' launch and reduction latency allows, and
// batches with enough systems to fill every SM with CTAs.  A CTA has one
// SM's FP64 rate (2 FMAs per clock), so its iteration costs about one FP64
// operation per nonzero plus eight per row; measured on GB300, up to about
// 40,000 of those it beats a phase-kernel CG iteration (about 14-16 us at
// small sizes): q1_hex 8^3 (729 rows, 15,625 nonzeros) 13.6 against 21.9
// us, poisson2d 64^2 (4,096 rows, 20,224 nonzeros) 18.4 against 14.0 us.
bool cta_size_rule(gbs_mat A, bool per_system, int systems_per_sm) {
  const int64_t nz = per_system ? A->max_sys_nnz : A->nnz;
  const int64_t rows = per_system ? A->max_sys_rows : A->nrows;
  return nz + 8 * rows <= CTA_AUTO_WORK ||
         (per_system && A->nsys >= (int64_t)systems_per_sm * sm_count(A));
}

// The per-CTA PCG solver for a.cta_n systems: one CTA per SM (each system
// then has an SM and 64 registers a thread to itself while it runs), or two
// (32 registers) when the plan caps the grids at two or more CTAs per SM and
// there are more systems than SMs; at most cta_n CTAs, which take the systems
// beyond the grid from a queue (k_cta_pcg).
static void launch_cta_pcg(gbs_mat A, const PcgArgs &a, bool refined, cudaStream_t s) {
  const int64_t per = A->ctas_per_sm >= 2 && a.cta_n > sm_count(A) ? 2 : 1;
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.cta_n, per * sm_count(A)));
  if (per == 1) {
    if (refined) k_cta_pcg<true, 1><<<grid, CTA_TPB, 0, s>>>(a);
    else k_cta_pcg<false, 1><<<grid, CTA_TPB, 0, s>>>(a);
  } else {
    if (refined) k_cta_pcg<true, 2><<<grid, CTA_TPB, 0, s>>>(a);
    else k_cta_pcg<false, 2><<<grid, CTA_TPB, 0, s>>>(a);
  }
}

int sm_count(gbs_mat A) {
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device);
  return nsm;
}

bool use_cta_solver(gbs_mat A, bool per_system) {
  const int32_t sv = solver_for(A, per_system);
  if (sv == GBS_SOLVER_CTA) return true;
  if (sv == GBS_SOLVER_PHASES || A->lanes != GBS_SPMV_SELL) return false;
  if (sv == GBS_SOLVER_SPLIT && per_system) return false;  // solve() splits the batch
  return cta_size_rule(A, per_system, 2);  // two 1024-thread PCG CTAs fit an SM
}

int solve(gbs_mat A, const double *b, double *x, const ksp_opts &o, bool per_system,
          cudaStream_t s) {
  const bool refined = o.precision == GBS_FP32_REFINED;
  // the sliced copy (a no-op once built; rebuilt here if switching its
  // column patterns could not rebuild it)
  if (A->lanes == GBS_SPMV_SELL) GBS_TRY(sell_build(A, s));
  // the handle's CG form: FP64 CG on the phase kernels may run as the
  // single-reduction loop (same iterates in exact arithmetic, two kernels per
  // iteration instead of three, or one)
  const bool split =
      per_system && solver_for(A, per_system) == GBS_SOLVER_SPLIT && A->lanes == GBS_SPMV_SELL;
  if (!refined && A->cg_form != GBS_CG_TEXTBOOK && A->lanes == GBS_SPMV_SELL && !split &&
      !use_cta_solver(A, per_system)) {
    ksp_opts sr = o;
    sr.method = GBS_KSP_CGSR;
    return solve_krylov(A, b, x, sr, per_system, s);
  }
  GBS_TRY(ensure_solver_workspace(A, refined, s));
  if (refined && !A->val32_valid) GBS_TRY(launch_to_fp32(A, s));
  A->last_count = per_system ? A->nsys : 1;
  A->last_ensemble = !per_system;
  A->trips_counted = true;
  A->last_solver = GBS_SOLVER_PHASES;
  if (A->ta.nblocks == 0) {  // empty matrix: nothing to iterate
    GBS_TRY_CUDA(cudaMemsetAsync(A->st, 0, sizeof(SysState) * A->nsys, s));
    GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
    return GBS_OK;
  }
  if (use_cta_solver(A, per_system)) {
    if (A->lanes != GBS_SPMV_SELL) {
      set_error("the per-CTA solver needs the sliced-ELL row products (plan kernel)");
      return GBS_ERR_ARG;
    }
    A->last_solver = GBS_SOLVER_CTA;
    GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
    GBS_TRY(put_call(A->call, call_args(b, x, o), s, A->ctl));
    PcgArgs a = make_args(A, per_system, refined);
    a.order = per_system ? A->cta_order : nullptr;
    a.cta_n = per_system ? A->nsys : 1;
    launch_cta_pcg(A, a, refined, s);
    GBS_LAUNCHED(1);
    return GBS_OK;
  }
  if (split) {
    // the systems of at least split_rows rows on the phase kernels (the
    // others are skipped by every phase: walk), then the rest -- a suffix of
    // cta_order, which lists the systems by decreasing rows -- on the
    // per-CTA solver, after the loop (whose graph clears every system's state
    // first) on the same stream
    const int32_t nbig = split_count(A);
    A->last_solver = GBS_SOLVER_SPLIT;
    if (nbig > 0) {
      GBS_TRY(build_split_tables(A, s));
      GBS_TRY(ensure_solver_workspace(A, refined, s));  // the split tables' slots
      PcgArgs a = make_args(A, per_system, refined);
      a.ta = view(A->sa);
      a.te = view(A->se);
      a.part_e = A->sa.nslots;
      a.grid_a = A->sa.grid;
      a.grid_e = A->se.grid;
      GBS_TRY(run_loop(A, cg_plan(refined, A->lanes, wide_rows(A)), refined ? GBS_GRAPH_CG32 : GBS_GRAPH_CG,
                       a, b, x, o, per_system, s));
    } else {
      GBS_TRY_CUDA(cudaMemsetAsync(A->st, 0, sizeof(SysState) * A->nsys, s));
      GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
      GBS_TRY(put_call(A->call, call_args(b, x, o), s, A->ctl));
    }
    if (nbig < A->nsys) {
      PcgArgs a = make_args(A, per_system, refined);
      a.order = A->cta_order + nbig;
      a.cta_n = A->nsys - nbig;
      GBS_TRY_CUDA(cudaMemsetAsync(&A->ctl->queue, 0, sizeof(int32_t), s));
      launch_cta_pcg(A, a, refined, s);
      GBS_LAUNCHED(1);
    }
    return GBS_OK;
  }
  return run_loop(A, cg_plan(refined, A->lanes, wide_rows(A)), refined ? GBS_GRAPH_CG32 : GBS_GRAPH_CG,
                  make_args(A, per_system, refined), b, x, o, per_system, s);
}

// Systems with at least split_rows rows (a prefix of cta_order).
int32_t split_count(gbs_mat A) {
  int32_t k = 0;
  for (int32_t q = 0; q < A->nsys; ++q)
    if (A->row_off_h[q + 1] - A->row_off_h[q] >= A->split_rows) ++k;
  return k;
}

// Runs a loop plan on the phase kernels: host-stepped (o.host_loop) or as the
// cached graph of its kind.
int run_loop(gbs_mat A, const LoopPlan &P, int kind, const PcgArgs &a, const double *b,
             double *x, const ksp_opts &o, bool per_system, cudaStream_t s) {
  A->loop_body = P.nbody;
  if (o.host_loop) {
    GBS_TRY_CUDA(cudaMemsetAsync(A->ctl, 0, sizeof(DevCtl), s));
    GBS_TRY_CUDA(cudaMemsetAsync(A->sys_cnt, 0, sizeof(unsigned) * A->nsys, s));
    GBS_TRY_CUDA(cudaMemsetAsync(A->st, 0, sizeof(SysState) * A->nsys, s));
    if (P.body_coop)
      GBS_TRY_CUDA(cudaMemsetAsync(A->halo_flags, 0, sizeof(int32_t) * A->ta.grid, s));
    GBS_TRY(put_call(A->call, call_args(b, x, o), s));
    return run_loop_stepped(P, a, a.grid_a, a.grid_e, max_trips_for(o), A->ctl, s);
  }
  cudaGraphExec_t &G = A->graph[kind][per_system ? 1 : 0];
  if (!G) GBS_TRY(build_loop_graph(A, P, a, &G));
  GBS_TRY(put_call(A->call, call_args(b, x, o), s));
  GBS_TRY_CUDA(cudaGraphLaunch(G, s));
  count_launches(P.npre + P.npost);  // the loop's kernels are counted when read
  A->trips_counted = false;
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
  if (!A->trips_counted) {
    count_launches(A->loop_body * ctl.trips);
    A->trips_counted = true;
  }
  int first = GBS_OK;
  for (int32_t q = 0; q < n; ++q) {
    const SysState &S = A->st_host[q];
    ksp_result &R = res[q];
    R.status = S.status;
    if (S.active) R.status = ctl.err ? ctl.err : GBS_ERR_MAXIT;  // stopped early
    R.iterations = S.iterations;
    R.outer_iterations = S.outer;
    R.solver = A->last_solver;
    if (R.solver == GBS_SOLVER_SPLIT)  // the engine this system ran on
      R.solver = A->row_off_h[q + 1] - A->row_off_h[q] >= A->split_rows ? GBS_SOLVER_PHASES
                                                                         : GBS_SOLVER_CTA;
    R.rnorm0 = S.rnorm0;
    R.rnorm = S.rnorm;
    const double bn = sqrt(S.bb);
    R.true_rel_residual = bn > 0.0 ? sqrt(S.tt) / bn : sqrt(S.tt);
    if (R.status != GBS_OK && first == GBS_OK) first = R.status;
  }
  if (first != GBS_OK) set_error("solve finished with status %d", first);
  return first;
}

int read_phase_ns(gbs_mat A, int64_t *phase_ns, cudaStream_t s) {
  DevCtl c;
  GBS_TRY_CUDA(cudaMemcpyAsync(&c, A->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 5; ++k) phase_ns[k] = c.phase_ns[k];
  return GBS_OK;
}

}  // namespace gbs

// ------------------------------------------------------------------ no-alloc solve
//
// ksp_solve_cg_noalloc: the same FP64 phase kernels, for callers that must not
// allocate device memory -- e.g. code that works inside a fixed memory budget
// owned by another allocator, or that cannot afford the device
// synchronisation cudaMalloc / cudaFree imply.  Its scratch (the r, p, q and
// D^-1 vectors, the block tables, the reduction slots, the control words and
// the call arguments) lives in one file-scope __device__ array of fixed size,
// so the call performs no allocation of any kind; it builds no CUDA graph
// either (instantiation allocates), and steps the loop from the host.  The
// caller passes the CSR matrix, b and x.  Limit: n <= NOALLOC_MAX_ROWS rows
// (the array holds about 8.5 MB and stays resident on every GPU that loads the
// library until the process exits).  All calls share the array: calls that
// overlap on the GPU (other streams, other host threads) race and must be
// serialised by the caller.  The first call on a device looks the array's
// device address up (cudaGetSymbolAddress, with that device current); make
// that first call before any stream capture.  The looked-up address is kept
// for the life of the process: after a cudaDeviceReset on that device the
// module is loaded again and the kept address is stale, so a process that
// resets a device must not call this entry point on it afterwards.

namespace {

constexpr int64_t NOALLOC_MAX_ROWS = 262144;
constexpr int NOALLOC_RA = 256, NOALLOC_RE = 512, NOALLOC_LANES = 4;
constexpr int64_t NOALLOC_MAX_BLK_A = NOALLOC_MAX_ROWS / NOALLOC_RA;
constexpr int64_t NOALLOC_MAX_BLK_E = NOALLOC_MAX_ROWS / NOALLOC_RE;

struct NoallocScratch {
  double r[NOALLOC_MAX_ROWS], p[NOALLOC_MAX_ROWS], q[NOALLOC_MAX_ROWS],
      dinv[NOALLOC_MAX_ROWS];
  double part[(NOALLOC_MAX_BLK_A + NOALLOC_MAX_BLK_E + 8) * gbs::SLOT_STRIDE];
  int32_t row0_a[NOALLOC_MAX_BLK_A + 4];
  int32_t row0_e[NOALLOC_MAX_BLK_E + 4];
  unsigned sys_cnt[4];
  gbs::SysState st[1];
  gbs::DevCtl ctl;
  gbs::CallArgs call;
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
// the two block tables (256-row SpMV blocks, 512-row update blocks).
__global__ void k_noalloc_prep(int64_t n, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, const double *__restrict__ val,
                               double *__restrict__ dinv, int32_t *__restrict__ row0_a,
                               int32_t nba, int32_t *__restrict__ row0_e, int32_t nbe) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t r = i0; r < n; r += stride) {
    double d = 0.0;
    for (int32_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q)
      if (col[q] == r) d = val[q];
    dinv[r] = (d > 0.0) ? 1.0 / d : 0.0;
  }
  for (int64_t b = i0; b <= nba; b += stride)
    row0_a[b] = (int32_t)(b * NOALLOC_RA < n ? b * NOALLOC_RA : n);
  for (int64_t b = i0; b <= nbe; b += stride)
    row0_e[b] = (int32_t)(b * NOALLOC_RE < n ? b * NOALLOC_RE : n);
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
  if (oo.method != GBS_KSP_CG) {
    set_error("ksp_solve_cg_noalloc: o->method must be GBS_KSP_CG");
    return GBS_ERR_ARG;
  }
  if (!(oo.rtol >= 0.0) || !std::isfinite(oo.rtol)) {
    set_error("ksp_solve_cg_noalloc: rtol must be finite and >= 0");
    return GBS_ERR_ARG;
  }
  if (oo.host_loop != 0 && oo.host_loop != 1) {
    set_error("ksp_solve_cg_noalloc: host_loop must be 0 or 1");
    return GBS_ERR_ARG;
  }
  if (oo.maxit < 0) oo.maxit = (int32_t)std::min<int64_t>(10 * std::max<int64_t>(n, 1), 100000);
  if (oo.timeout_ns < 0) oo.timeout_ns = 0;
  if (n == 0) {
    if (res) memset(res, 0, sizeof(*res));
    return GBS_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NoallocScratch *S = nullptr;
  GBS_TRY(noalloc_scratch(&S));
  const int32_t nba = (int32_t)((n + NOALLOC_RA - 1) / NOALLOC_RA);
  const int32_t nbe = (int32_t)((n + NOALLOC_RE - 1) / NOALLOC_RE);

  // the control words and arrival counters must start at zero on every call
  GBS_TRY_CUDA(cudaMemsetAsync(&S->ctl, 0, sizeof(DevCtl), s));
  GBS_TRY_CUDA(cudaMemsetAsync(S->sys_cnt, 0, sizeof(S->sys_cnt), s));
  k_noalloc_prep<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
      n, row_ptr, col, val, S->dinv, S->row0_a, nba, S->row0_e, nbe);
  GBS_LAUNCHED(1);
  GBS_TRY(put_call(&S->call, call_args(b, x, oo), s));

  // one CTA per block: each table has as many slots as blocks
  PcgArgs a;
  memset(&a, 0, sizeof(a));
  a.nsys = 1;
  a.ensemble = 1;
  a.ta = BlockTable{nba, S->row0_a, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  a.te = BlockTable{nbe, S->row0_e, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  a.part_e = nba;
  a.grid_a = nba;
  a.grid_e = nbe;
  a.row_ptr = row_ptr;
  a.col = col;
  a.val = val;
  a.dinv = S->dinv;
  a.r = S->r;
  a.p = S->p;
  a.q = S->q;
  a.part = S->part;
  a.sys_cnt = S->sys_cnt;
  a.st = S->st;
  a.ctl = &S->ctl;
  a.call = &S->call;
  GBS_TRY(run_loop_stepped(cg_plan(false, NOALLOC_LANES), a, nba, nbe, max_trips_for(oo),
                           &S->ctl, s));

  // the loop has synchronised the stream once per chunk already; one more
  // small read gives the status, returned whether or not res is given
  SysState st;
  DevCtl ctl;
  GBS_TRY_CUDA(cudaMemcpyAsync(&st, S->st, sizeof(SysState), cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaMemcpyAsync(&ctl, &S->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
  GBS_TRY_CUDA(cudaStreamSynchronize(s));
  const int status = st.active ? (ctl.err ? ctl.err : GBS_ERR_MAXIT) : st.status;
  if (res) {
    res->status = status;
    res->iterations = st.iterations;
    res->outer_iterations = 0;
    res->solver = GBS_SOLVER_PHASES;
    res->rnorm0 = st.rnorm0;
    res->rnorm = st.rnorm;
    const double bn = sqrt(st.bb);
    res->true_rel_residual = bn > 0.0 ? sqrt(st.tt) / bn : sqrt(st.tt);
  }
  if (status != GBS_OK) set_error("ksp_solve_cg_noalloc: solve ended with status %d", status);
  return status;
}
