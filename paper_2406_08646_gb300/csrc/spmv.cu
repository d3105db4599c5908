// MatMult (Sec. 6.1): y = A x on the assembled CSR, FP64, and the launch plan
// (block tables, lanes per row, grid caps) shared with the solves.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"
#include "phases.cuh"

namespace gbs {

constexpr int SPMV_ROWS = PHASE_TPB;  // rows per CTA pass of the CSR-vector SpMV (32 per warp)

// y = A x with the CSR-vector row product of the solves (csr_rows), over
// chunks of 32 rows per warp.
template <int L>
__global__ void __launch_bounds__(PHASE_TPB) k_spmv(const int32_t *__restrict__ row_ptr,
                                                    const int32_t *__restrict__ col,
                                                    const double *__restrict__ val,
                                                    const double *__restrict__ x,
                                                    double *__restrict__ y, int32_t n) {
  auto f = [&](int r, double s) { y[r] = s; };
  for (int64_t r0 = (int64_t)blockIdx.x * SPMV_ROWS; r0 < n;
       r0 += (int64_t)gridDim.x * SPMV_ROWS) {
    const int r1 = (int)(r0 + SPMV_ROWS < n ? r0 + SPMV_ROWS : n);
    csr_rows<double, L>(row_ptr, col, val, x, (int)r0, r1, f);
  }
}

// y = A x with the sliced-ELL row product (sell_rows), 8 slices per CTA pass.
__global__ void __launch_bounds__(PHASE_TPB, SELL_MIN_CTAS)
    k_spmv_sell(const SellView S, const double *__restrict__ sval,
                const double *__restrict__ x, double *__restrict__ y, int32_t nslices,
                int32_t stream_matrix) {
  auto f = [&](int r, double s) { y[r] = s; };
  const int per = PHASE_TPB / 32;
  for (int64_t s0 = (int64_t)blockIdx.x * per; s0 < nslices; s0 += (int64_t)gridDim.x * per) {
    const int s1 = (int)(s0 + per < nslices ? s0 + per : nslices);
    if (stream_matrix)
      sell_rows<double, true, GATHER_NC>(S, sval, x, (int)s0, s1, f);
    else sell_rows<double, false, GATHER_NC>(S, sval, x, (int)s0, s1, f);
  }
}

int launch_spmv(gbs_mat A, const double *x, double *y, cudaStream_t s) {
  if (A->nrows == 0) return GBS_OK;
  const int32_t n = (int32_t)A->nrows;
  if (A->lanes == GBS_SPMV_SELL) {
    GBS_TRY(sell_build(A, s));  // a no-op once built
    const int64_t ns = A->nslices, per = PHASE_TPB / 32;
    const unsigned grid = (unsigned)std::min<int64_t>((ns + per - 1) / per, 1 << 20);
    k_spmv_sell<<<grid, PHASE_TPB, 0, s>>>(sell_view(A), A->sell_val, x, y, (int32_t)ns,
                                           stream_matrix(A, 12));
    GBS_LAUNCHED(1);
    return GBS_OK;
  }
  const int64_t chunks = (A->nrows + SPMV_ROWS - 1) / SPMV_ROWS;
  const unsigned grid = (unsigned)std::min<int64_t>(chunks, 1 << 20);
  switch (A->lanes) {
    case 1: k_spmv<1><<<grid, PHASE_TPB, 0, s>>>(A->row_ptr, A->col, A->val, x, y, n); break;
    case 2: k_spmv<2><<<grid, PHASE_TPB, 0, s>>>(A->row_ptr, A->col, A->val, x, y, n); break;
    case 8: k_spmv<8><<<grid, PHASE_TPB, 0, s>>>(A->row_ptr, A->col, A->val, x, y, n); break;
    case 32: k_spmv<32><<<grid, PHASE_TPB, 0, s>>>(A->row_ptr, A->col, A->val, x, y, n); break;
    default: k_spmv<4><<<grid, PHASE_TPB, 0, s>>>(A->row_ptr, A->col, A->val, x, y, n); break;
  }
  GBS_LAUNCHED(1);
  return GBS_OK;
}

// 1 when the sliced copy (bytes_per_entry per padded entry) is larger than
// half of L2: its loads then carry the evict-first hint.
int32_t stream_matrix(gbs_mat A, int bytes_per_entry) {
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, A->device) != cudaSuccess) l2 = 0;
  return (double)A->sell_nnz * bytes_per_entry > 0.5 * (double)l2 ? 1 : 0;
}

// Lanes per row from the mean row length: enough lanes that a warp's loads
// cover whole 32-byte sectors of the value stream, few enough that masked
// slots and the cross-lane adds stay a small part of the FP64 work.
int auto_lanes(int64_t nnz, int64_t nrows) {
  const double m = nrows > 0 ? (double)nnz / (double)nrows : 0.0;
  if (m < 3.0) return 1;
  if (m < 12.0) return 2;
  if (m < 48.0) return 4;
  if (m < 160.0) return 8;
  return 32;
}

void free_table(TableDev &t) {
  dev_free(t.row0, nullptr);  // one buffer holds all five arrays (build_table)
  t.row0 = t.sys = t.sys_blk0 = t.sys_slot0 = t.slice0 = t.row1 = t.slice1 = nullptr;
  t.nblocks = 0;
  t.grid = 0;
  t.nslots = 0;
  t.sys_blk0_h.clear();
}

// Each system's rows cut into ceil(n_s / R) blocks of R rows (the last one
// ragged); blocks never straddle systems.  R is a multiple of 32, so a block
// is a whole number of the 32-row slices of the sliced-ELL layout (slice0).
// The kernels walking the table run min(blocks, cap_per_sm x SMs) CTAs;
// system s owns min(blocks_s, grid) reduction slots.
// min_rows > 0: only the systems of at least min_rows rows get blocks (the
// size split's table; the others have none and are never visited).
static int build_table(gbs_mat A, int32_t R, int32_t cap_per_sm, TableDev &t, cudaStream_t st,
                       int64_t min_rows = 0) {
  std::vector<int32_t> row0, sys, sb0(A->nsys + 1, 0), sl0, row1, sl1;
  int32_t slices = 0;
  for (int32_t q = 0; q < A->nsys; ++q) {
    const int64_t a = A->row_off_h[q], e = A->row_off_h[q + 1];
    for (int64_t r = a; r < e && e - a >= min_rows; r += R) {
      const int64_t re = std::min<int64_t>(r + R, e);
      row0.push_back((int32_t)r);
      sys.push_back(q);
      sl0.push_back(slices + (int32_t)((r - a) / 32));
      row1.push_back((int32_t)re);
      sl1.push_back(slices + (int32_t)((re - a + 31) / 32));
    }
    slices += (int32_t)((e - a + 31) / 32);
    sb0[q + 1] = (int32_t)row0.size();
  }
  row0.push_back((int32_t)A->nrows);
  sl0.push_back(slices);
  const int32_t nb = (int32_t)sys.size();
  int nsm = 0;
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device));
  int64_t grid = std::min<int64_t>(nb, (int64_t)std::max(cap_per_sm, 1) * nsm);
  grid = std::max<int64_t>(grid, 1);
  std::vector<int32_t> so(A->nsys + 1, 0);
  for (int32_t q = 0; q < A->nsys; ++q)
    so[q + 1] = so[q] + (int32_t)std::min<int64_t>(sb0[q + 1] - sb0[q], grid);
  free_table(t);
  // one buffer: row0 (nb + 1), slice0 (nb + 1), sys (nb), sys_blk0, sys_slot0 (nsys + 1
  // each), and with gaps (min_rows > 0) row1, slice1 (nb each)
  const bool ends = min_rows > 0;
  const size_t tot = 3 * (size_t)nb + 2 + 2 * ((size_t)A->nsys + 1) + (ends ? 2 * (size_t)nb : 0);
  std::vector<int32_t> h;
  h.reserve(tot);
  h.insert(h.end(), row0.begin(), row0.end());
  h.insert(h.end(), sl0.begin(), sl0.end());
  h.insert(h.end(), sys.begin(), sys.end());
  h.insert(h.end(), sb0.begin(), sb0.end());
  h.insert(h.end(), so.begin(), so.end());
  if (ends) {
    h.insert(h.end(), row1.begin(), row1.end());
    h.insert(h.end(), sl1.begin(), sl1.end());
  }
  int32_t *d = nullptr;
  GBS_TRY(dev_alloc(&d, tot, st));
  GBS_TRY_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(int32_t) * tot, cudaMemcpyHostToDevice, st));
  t.row0 = d;
  t.slice0 = d + nb + 1;
  t.sys = d + 2 * (size_t)nb + 2;
  t.sys_blk0 = t.sys + nb;
  t.sys_slot0 = t.sys_blk0 + A->nsys + 1;
  t.row1 = ends ? t.sys_slot0 + A->nsys + 1 : nullptr;
  t.slice1 = ends ? t.row1 + nb : nullptr;
  t.sys_blk0_h = sb0;
  t.nblocks = nb;
  t.grid = (int32_t)grid;
  t.nslots = std::max<int64_t>(so[A->nsys], 1);
  return GBS_OK;
}

// The one-kernel CG's wait window over table A (blocks of R rows per
// system, grid G, CTA c taking blocks c, c + G, ...): block b's row products
// read rows within col_span of its own, i.e. blocks b - lo_b .. b + hi_b;
// with lo and hi the largest lo_b and hi_b, CTA c's blocks need only CTAs
// c - lo .. c + hi (mod G).  halo_lo = lo, halo_n = lo + hi + 1, or the
// whole grid (halo_lo = 0, halo_n = G) when that window would wrap onto
// itself.
static void halo_window(gbs_mat A, int32_t R, const TableDev &t) {
  std::vector<int64_t> row0;
  for (int32_t q = 0; q < A->nsys; ++q)
    for (int64_t r = A->row_off_h[q]; r < A->row_off_h[q + 1]; r += R) row0.push_back(r);
  const int64_t nb = (int64_t)row0.size();
  row0.push_back(A->nrows);
  const int64_t span = A->col_span;
  auto blk = [&](int64_t r) {  // the block holding row r, 0 <= r < nrows
    return (int64_t)(std::upper_bound(row0.begin(), row0.end() - 1, r) - row0.begin()) - 1;
  };
  int64_t lo = 0, hi = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t a = std::max<int64_t>(0, row0[b] - span);
    const int64_t e = std::min<int64_t>(A->nrows - 1, row0[b + 1] - 1 + span);
    lo = std::max(lo, b - blk(a));
    hi = std::max(hi, blk(e) - b);
  }
  const int64_t G = std::max<int32_t>(t.grid, 1);
  if (nb == 0) {
    A->halo_lo = A->halo_n = 0;
  } else if (lo + hi + 1 >= G) {
    A->halo_lo = 0;
    A->halo_n = (int32_t)G;
  } else {
    A->halo_lo = (int32_t)lo;
    A->halo_n = (int32_t)(lo + hi + 1);
  }
}

// The size split's tables: the systems of at least split_rows rows, cut into
// blocks sized for them alone (about one block per CTA of a one-wave grid, as
// the plan's automatic sizes are for the whole batch), at the plan's
// occupancy.  Rebuilt when the split or the plan changes.
int build_split_tables(gbs_mat A, cudaStream_t st) {
  if (A->split_built == A->split_rows && A->sa.row0) return GBS_OK;
  int occ_rows = 1, occ_upd = 1, nsm = 1;
  GBS_TRY(phase_occupancy(A->lanes, &occ_rows, &occ_upd));
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device));
  const int cap_a = A->ctas_per_sm ? A->ctas_per_sm : occ_rows;
  const int cap_e = A->ctas_per_sm ? A->ctas_per_sm : occ_upd;
  int64_t rows = 0;
  for (int32_t q = 0; q < A->nsys; ++q) {
    const int64_t n = A->row_off_h[q + 1] - A->row_off_h[q];
    if (n >= A->split_rows) rows += n;
  }
  auto auto_rows = [&](int cap) {
    const int64_t per = (rows + (int64_t)cap * nsm - 1) / ((int64_t)cap * nsm);
    return (int32_t)std::min<int64_t>(65536, std::max<int64_t>(PHASE_TPB, (per + 31) / 32 * 32));
  };
  GBS_TRY(build_table(A, auto_rows(cap_a), cap_a, A->sa, st, A->split_rows));
  GBS_TRY(build_table(A, auto_rows(cap_e), cap_e, A->se, st, A->split_rows));
  A->split_built = A->split_rows;
  return GBS_OK;
}

// nnz_off[q] = row_ptr[first row of system q] (q = 0 .. nsys).
__global__ void k_system_nnz(int32_t nsys, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ row0,
                             const int32_t *__restrict__ sys_blk0, int32_t *__restrict__ nnz_off) {
  const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q <= nsys) nnz_off[q] = row_ptr[row0[sys_blk0[q]]];
}

// Systems in decreasing row count (ties by index): the per-CTA solver hands
// them to CTAs in this order, so the longest solves start first.  Also the
// largest system's rows and nonzeros (the solver choice uses them; a batch's
// per-system counts are read back, which synchronises st).
static int build_cta_order(gbs_mat A, cudaStream_t st) {
  std::vector<int32_t> ord(A->nsys), noff(A->nsys + 1, 0);
  if (A->nsys == 1) {
    noff[1] = (int32_t)A->nnz;
  } else {
    int32_t *d = nullptr;
    GBS_TRY(dev_alloc(&d, A->nsys + 1, st));
    k_system_nnz<<<(A->nsys + 256) / 256, 256, 0, st>>>(A->nsys, A->row_ptr, A->ta.row0,
                                                        A->ta.sys_blk0, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(noff.data(), d, sizeof(int32_t) * (A->nsys + 1), cudaMemcpyDeviceToHost,
                          st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(d, st);
    count_launches(1);
    GBS_TRY_CUDA(e);
  }
  A->max_sys_rows = A->max_sys_nnz = 0;
  for (int32_t q = 0; q < A->nsys; ++q) {
    ord[q] = q;
    A->max_sys_rows = std::max(A->max_sys_rows, A->row_off_h[q + 1] - A->row_off_h[q]);
    A->max_sys_nnz = std::max<int64_t>(A->max_sys_nnz, noff[q + 1] - noff[q]);
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t u, int32_t v) {
    return A->row_off_h[u + 1] - A->row_off_h[u] > A->row_off_h[v + 1] - A->row_off_h[v];
  });
  if (!A->cta_order) GBS_TRY(dev_alloc(&A->cta_order, A->nsys, st));
  GBS_TRY_CUDA(cudaMemcpyAsync(A->cta_order, ord.data(), sizeof(int32_t) * A->nsys,
                               cudaMemcpyHostToDevice, st));
  GBS_TRY_CUDA(cudaStreamSynchronize(st));  // ord is a local vector
  return GBS_OK;
}

// Plan: SpMV-phase blocks of Ra rows, update-phase blocks of Re rows (both
// multiples of 32), the row-product kernel (GBS_SPMV_AUTO, GBS_SPMV_SELL or
// CSR-vector lanes per row) and a cap of CTAs per SM on the grids (0: as many
// as fit on an SM at once, so each phase kernel runs in one wave).  Cached graphs are dropped: they bake in the tables and grids.
// Work is ordered on stream st; the host copies of the tables are synchronous.
int build_plan(gbs_mat A, int32_t Ra, int32_t Re, int32_t kernel, int32_t ctas_per_sm,
               cudaStream_t st) {
  const bool bad_ra = Ra != 0 && (Ra < 32 || Ra > 65536 || (Ra % 32) != 0);
  const bool bad_re = Re != 0 && (Re < 32 || Re > 65536 || (Re % 32) != 0);
  if (bad_ra || bad_re ||
      !(kernel == GBS_SPMV_AUTO || kernel == GBS_SPMV_SELL || kernel == 1 || kernel == 2 ||
        kernel == 4 || kernel == 8 || kernel == 32) ||
      ctas_per_sm < 0 || ctas_per_sm > 64) {
    set_error("plan: spmv_rows %d and update_rows %d must be 0 (auto) or multiples of 32 in "
              "[32, 65536], "
              "kernel %d one of -1 (auto), 0 (sliced ELL), 1, 2, 4, 8, 32 (CSR lanes), "
              "ctas_per_sm %d in [0, 64]",
              Ra, Re, kernel, ctas_per_sm);
    return GBS_ERR_ARG;
  }
  drop_graphs(A);
  free_table(A->sa);  // the size split's tables follow the plan
  free_table(A->se);
  A->split_built = 0;
  if (kernel == GBS_SPMV_AUTO) {
    GBS_TRY(sell_shape(A, st));
    kernel = (A->sell_ptr && (double)A->sell_nnz_rows <= 1.2 * (double)A->nnz)
                 ? GBS_SPMV_SELL
                 : auto_lanes(A->nnz, A->nrows);
  }
  if (kernel == GBS_SPMV_SELL) GBS_TRY(sell_build(A, st));
  // grids: one wave of the phase kernels unless capped explicitly; automatic
  // block sizes give about one block per CTA of that wave (at least one row
  // per thread, so every warp of a CTA has rows)
  int occ_rows = 1, occ_upd = 1, nsm = 1;
  GBS_TRY(phase_occupancy(kernel, &occ_rows, &occ_upd));
  GBS_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, A->device));
  const int cap_a = ctas_per_sm ? ctas_per_sm : occ_rows;
  const int cap_e = ctas_per_sm ? ctas_per_sm : occ_upd;
  auto auto_rows = [&](int cap) {
    const int64_t per = (A->nrows + (int64_t)cap * nsm - 1) / ((int64_t)cap * nsm);
    return (int32_t)std::min<int64_t>(65536, std::max<int64_t>(PHASE_TPB, (per + 31) / 32 * 32));
  };
  if (Ra == 0) Ra = auto_rows(cap_a);
  if (Re == 0) Re = auto_rows(cap_e);
  GBS_TRY(build_table(A, Ra, cap_a, A->ta, st));
  halo_window(A, Ra, A->ta);
  GBS_TRY(build_table(A, Re, cap_e, A->te, st));
  GBS_TRY(build_cta_order(A, st));
  A->Ra = Ra;
  A->Re = Re;
  A->lanes = kernel;
  A->ctas_per_sm = ctas_per_sm;
  return GBS_OK;
}

}  // namespace gbs
