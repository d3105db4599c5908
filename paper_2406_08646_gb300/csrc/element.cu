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
// (HBM-bound: 8 bytes per value written, 8 per element read).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.cuh"

namespace gbs {

constexpr int GEN_TPB = 256;

// Thread t writes entries 2 t and 2 t + 1 of the element blocks (one 16-byte
// store): element e = t / 32, local row a = (t / 4) % 8, columns b, b + 1
// with b = 2 (t % 4).
__global__ void __launch_bounds__(GEN_TPB)
    k_q1_values(int32_t ne, const double *__restrict__ kappa, double2 *__restrict__ v) {
  const int64_t nelem = (int64_t)ne * ne * ne;
  const int64_t npairs = nelem * 32;
  const double h = 1.0 / (double)ne;
  const double kd = 1.0 / 3.0, k2 = -1.0 / 12.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npairs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t >> 5;
    const int a = (int)((t >> 2) & 7), b0 = (int)(t & 3) * 2;
    const int32_t ex = (int32_t)(e % ne), ey = (int32_t)((e / ne) % ne),
                  ez = (int32_t)(e / ((int64_t)ne * ne));
    const double ke = __dmul_rn(__ldg(kappa + e), h);
    double out[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int b = b0 + u;
      // boundary tests of local nodes a and b (coordinate 0 or ne on a face)
      const int ax = ex + (a & 1), ay = ey + ((a >> 1) & 1), az = ez + (a >> 2);
      const int bx = ex + (b & 1), by = ey + ((b >> 1) & 1), bz = ez + (b >> 2);
      const bool fax = ax == 0 || ax == ne, fay = ay == 0 || ay == ne, faz = az == 0 || az == ne;
      const bool fbx = bx == 0 || bx == ne, fby = by == 0 || by == ne, fbz = bz == 0 || bz == ne;
      const bool ba = fax || fay || faz, bb = fbx || fby || fbz;
      double val;
      if (a == b) {
        if (ba) {
          const int m = (fax ? 1 : 2) * (fay ? 1 : 2) * (faz ? 1 : 2);
          val = 1.0 / (double)m;  // 1, 1/2, 1/4 or 1/8: exact
        } else {
          val = __dmul_rn(ke, kd);
        }
      } else if (ba || bb) {
        val = 0.0;
      } else {  // K_ref: 0 for one differing coordinate, -1/12 for two or three
        val = __dmul_rn(ke, __popc(a ^ b) == 1 ? 0.0 : k2);
      }
      out[u] = val;
    }
    v[t] = make_double2(out[0], out[1]);
  }
}

// Row and column indices of the element blocks: entry 64 e + 8 a + b is
// (g(e, a), g(e, b)).  Thread t writes the 8 entries of row a of element e
// (t = 8 e + a): two 16-byte stores of i (all g(e, a)) and two of j.
__global__ void __launch_bounds__(GEN_TPB)
    k_q1_indices(int32_t ne, int4 *__restrict__ i4, int4 *__restrict__ j4) {
  const int64_t nrow = (int64_t)ne * ne * ne * 8;
  const int32_t nn = ne + 1;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nrow;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t >> 3;
    const int a = (int)(t & 7);
    const int32_t ex = (int32_t)(e % ne), ey = (int32_t)((e / ne) % ne),
                  ez = (int32_t)(e / ((int64_t)ne * ne));
    const int32_t g0 = ex + nn * (ey + nn * ez);
    int32_t g[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) g[b] = g0 + (b & 1) + nn * (((b >> 1) & 1) + nn * (b >> 2));
    const int32_t ga = g0 + (a & 1) + nn * (((a >> 1) & 1) + nn * (a >> 2));
    i4[2 * t] = make_int4(ga, ga, ga, ga);
    i4[2 * t + 1] = make_int4(ga, ga, ga, ga);
    j4[2 * t] = make_int4(g[0], g[1], g[2], g[3]);
    j4[2 * t + 1] = make_int4(g[4], g[5], g[6], g[7]);
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
  const int64_t nrow = (int64_t)ne * ne * ne * 8;
  k_q1_indices<<<gen_grid(nrow), GEN_TPB, 0, (cudaStream_t)stream>>>(
      ne, reinterpret_cast<int4 *>(i), reinterpret_cast<int4 *>(j));
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
  const int64_t npairs = (int64_t)ne * ne * ne * 32;
  k_q1_values<<<gen_grid(npairs), GEN_TPB, 0, (cudaStream_t)stream>>>(
      ne, kappa, reinterpret_cast<double2 *>(v));
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
