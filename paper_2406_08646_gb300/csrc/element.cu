// Device-side COO generation for the two model problems (Sec. 3: the user's
// Jacobian callback fills the COO values on the device and hands them to
// MatSetValuesCOO; Sec. 5: element e writes its block at an offset of its
// own, here 64 e for a Q1 hexahedron and 4 e for a graph edge).
//
// Q1 hexahedra on ne^3 elements of the unit cube, h = 1/ne:
//   node g = ix + nn (iy + nn iz), nn = ne + 1; element e = ex + ne (ey + ne ez);
//   local node a = ax + 2 ay + 4 az; COO entry 64 e + 8 a + b holds
//   (g(e, a), g(e, b), (kappa_e h) K_ref[a][b]),
//   K_ref[a][b] = integral over the unit cube of grad N_a . grad N_b, by the
//   number of coordinates in which a and b differ: 0 -> 1/3, 1 -> 0,
//   2 or 3 -> -1/12.
//   Dirichlet on the outer faces with every row and the 27-point pattern
//   kept: an entry a != b touching a boundary node is 0, and a boundary node's
//   diagonal entry is 1/m, m = the node's element multiplicity (1, 2 or 4:
//   corner, edge or face node), so its assembled diagonal is exactly 1.
// Edges (variable-coefficient graph Laplacian): edge e between nodes a and b
//   with conductivity kappa_e writes (+k, +k, -k, -k) at 4 e .. 4 e + 3 for
//   the entries (a, a), (b, b), (a, b), (b, a); the indices are the caller's.
//
// The values are rounded in the order written above (kappa_e h first, then
// the product with K_ref), so they are the same bits a host program gets
// with the same two roundings.  Every kernel is a pure streaming write
// (HBM-bound: 8 bytes per value written, 8 per element read); the FP64
// multiplies, which on this part would otherwise bound the values kernel,
// are formed once per element (three), not once per value (64).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

constexpr int GEN_TPB = 256;

// Per-element data one warp shares: node coordinates of the element's corner
// and its three distinct products (kappa_e h) K_ref -- FP64 is scarce on this
// part, so each element's products are formed once, by one lane, and every
// value of its block is a selection among them.
struct ElemInfo {
  double p_diag, p_edge, p_face;  // (kappa h)/3, (kappa h)(-1/12), (kappa h) 0
  int32_t ex, ey, ez, pad;
};

// Warp w takes elements 32 w .. 32 w + 31: lane l forms element 32 w + l's
// products (three FP64 multiplies per element in all), then the warp writes
// the 32 blocks one after the other, lane l storing entries 2 l, 2 l + 1 of
// the block (local row a = l / 4, columns b = 2 (l % 4), b + 1) as one
// 16-byte store: 512 contiguous bytes per store instruction.
__global__ void __launch_bounds__(GEN_TPB)
    k_q1_values(int32_t ne, double h, const double *__restrict__ kappa,
                double2 *__restrict__ v) {
  __shared__ ElemInfo info[GEN_TPB];
  const int32_t nelem = ne * ne * ne;
  const int lane = threadIdx.x & 31;
  ElemInfo *wi = info + (threadIdx.x & ~31);
  const int a = lane >> 2, b0 = (lane & 3) * 2;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < nelem;
       w += nwarps) {
    const int32_t e0 = (int32_t)(w * 32);
    const int32_t e = e0 + lane;
    __syncwarp();
    if (e < nelem) {
      const double ke = __dmul_rn(__ldg(kappa + e), h);
      ElemInfo E;
      E.p_diag = __dmul_rn(ke, 1.0 / 3.0);
      E.p_edge = __dmul_rn(ke, -1.0 / 12.0);
      E.p_face = __dmul_rn(ke, 0.0);
      E.ex = e % ne;
      E.ey = (e / ne) % ne;
      E.ez = e / (ne * ne);
      E.pad = 0;
      wi[lane] = E;
    }
    __syncwarp();
    const int cnt = nelem - e0 < 32 ? nelem - e0 : 32;
    for (int j = 0; j < cnt; ++j) {
      const ElemInfo E = wi[j];
      double out[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int b = b0 + u;
        // boundary tests of local nodes a and b (coordinate 0 or ne)
        const int ax = E.ex + (a & 1), ay = E.ey + ((a >> 1) & 1), az = E.ez + (a >> 2);
        const int bx = E.ex + (b & 1), by = E.ey + ((b >> 1) & 1), bz = E.ez + (b >> 2);
        const bool fax = ax == 0 || ax == ne, fay = ay == 0 || ay == ne, faz = az == 0 || az == ne;
        const bool fbx = bx == 0 || bx == ne, fby = by == 0 || by == ne, fbz = bz == 0 || bz == ne;
        const bool ba = fax || fay || faz, bb = fbx || fby || fbz;
        double val;
        if (a == b) {
          // a boundary node's diagonal: 1/m with m = 1, 2 or 4 elements
          const int nf = (int)fax + (int)fay + (int)faz;  // faces it lies on
          val = ba ? (nf == 3 ? 1.0 : (nf == 2 ? 0.5 : 0.25)) : E.p_diag;
        } else if (ba || bb) {
          val = 0.0;
        } else {  // K_ref: 0 for one differing coordinate, -1/12 for two or three
          val = __popc(a ^ b) == 1 ? E.p_face : E.p_edge;
        }
        out[u] = val;
      }
      v[(int64_t)(e0 + j) * 32 + lane] = make_double2(out[0], out[1]);
    }
  }
}

// Row and column indices of the element blocks: entry 64 e + 8 a + b is
// (g(e, a), g(e, b)).  Warp w takes elements 32 w .. 32 w + 31; lane l
// computes element 32 w + l's first node, then the warp writes the blocks
// one after the other, lane l storing entries 2 l, 2 l + 1 of i and of j
// (8-byte stores, 256 contiguous bytes per instruction).
__global__ void __launch_bounds__(GEN_TPB)
    k_q1_indices(int32_t ne, int2 *__restrict__ i2, int2 *__restrict__ j2) {
  __shared__ int32_t g0s[GEN_TPB];
  const int32_t nelem = ne * ne * ne;
  const int32_t nn = ne + 1;
  const int lane = threadIdx.x & 31;
  int32_t *wg = g0s + (threadIdx.x & ~31);
  const int a = lane >> 2, b0 = (lane & 3) * 2;
  // offsets of local nodes a, b0, b0 + 1 from the element's first node
  auto off = [&](int q) { return (q & 1) + nn * (((q >> 1) & 1) + nn * (q >> 2)); };
  const int32_t oa = off(a), ob0 = off(b0), ob1 = off(b0 + 1);
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < nelem;
       w += nwarps) {
    const int32_t e0 = (int32_t)(w * 32);
    const int32_t e = e0 + lane;
    __syncwarp();
    if (e < nelem) wg[lane] = e % ne + nn * ((e / ne) % ne + nn * (e / (ne * ne)));
    __syncwarp();
    const int cnt = nelem - e0 < 32 ? nelem - e0 : 32;
    for (int j = 0; j < cnt; ++j) {
      const int32_t g0 = wg[j];
      const int64_t q = (int64_t)(e0 + j) * 32 + lane;
      i2[q] = make_int2(g0 + oa, g0 + oa);
      j2[q] = make_int2(g0 + ob0, g0 + ob1);
    }
  }
}

// Edge e: (+k, +k, -k, -k) at 4 e .. 4 e + 3, two 16-byte stores.
__global__ void __launch_bounds__(GEN_TPB)
    k_edge_values(int64_t nedges, const double *__restrict__ kappa, double2 *__restrict__ v) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nedges;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double k = __ldg(kappa + e);
    v[2 * e] = make_double2(k, k);
    v[2 * e + 1] = make_double2(-k, -k);
  }
}

static unsigned gen_grid(int64_t work) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + GEN_TPB - 1) / GEN_TPB, 1 << 20));
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ne^3 * 64 entries must stay below 2^31 (int32 COO indices downstream).
static bool q1_size_ok(int32_t ne) {
  return ne >= 1 && (int64_t)ne * ne * ne * 64 < 2147483648LL;
}

}  // namespace gbs

using namespace gbs;

extern "C" int q1_hex_element_coo(int32_t ne, int32_t *i, int32_t *j, void *stream) {
  if (!q1_size_ok(ne)) {
    set_error("q1_hex_element_coo: ne = %d must be >= 1 with 64 ne^3 < 2^31", ne);
    return GBS_ERR_ARG;
  }
  if (!i || !j || !aligned16(i) || !aligned16(j)) {
    set_error("q1_hex_element_coo: i and j must be non-null 16-byte aligned device pointers");
    return GBS_ERR_ARG;
  }
  const int64_t warps = ((int64_t)ne * ne * ne + 31) / 32;
  k_q1_indices<<<gen_grid(32 * warps), GEN_TPB, 0, (cudaStream_t)stream>>>(
      ne, reinterpret_cast<int2 *>(i), reinterpret_cast<int2 *>(j));
  GBS_LAUNCHED(1);
  return GBS_OK;
}

extern "C" int q1_hex_element_values(int32_t ne, const double *kappa, double *v, void *stream) {
  if (!q1_size_ok(ne)) {
    set_error("q1_hex_element_values: ne = %d must be >= 1 with 64 ne^3 < 2^31", ne);
    return GBS_ERR_ARG;
  }
  if (!kappa || !v || !aligned16(v) || ((uintptr_t)kappa & 7u) != 0) {
    set_error("q1_hex_element_values: kappa (8-byte aligned) and v (16-byte aligned) must be "
              "non-null device pointers");
    return GBS_ERR_ARG;
  }
  const int64_t warps = ((int64_t)ne * ne * ne + 31) / 32;
  k_q1_values<<<gen_grid(32 * warps), GEN_TPB, 0, (cudaStream_t)stream>>>(
      ne, 1.0 / (double)ne, kappa, reinterpret_cast<double2 *>(v));
  GBS_LAUNCHED(1);
  return GBS_OK;
}

extern "C" int edge_coo_values(int64_t nedges, const double *kappa, double *v, void *stream) {
  if (nedges < 0 || nedges * 4 >= 2147483648LL) {
    set_error("edge_coo_values: nedges = %lld must be in [0, 2^29)", (long long)nedges);
    return GBS_ERR_ARG;
  }
  if (nedges == 0) return GBS_OK;
  if (!kappa || !v || !aligned16(v) || ((uintptr_t)kappa & 7u) != 0) {
    set_error("edge_coo_values: kappa (8-byte aligned) and v (16-byte aligned) must be "
              "non-null device pointers");
    return GBS_ERR_ARG;
  }
  k_edge_values<<<gen_grid(nedges), GEN_TPB, 0, (cudaStream_t)stream>>>(
      nedges, kappa, reinterpret_cast<double2 *>(v));
  GBS_LAUNCHED(1);
  return GBS_OK;
}
