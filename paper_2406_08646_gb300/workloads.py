"""Seeded synthetic workloads (COO triples, right-hand sides, targets).

This module is the ONE piece shared by the CUDA path and the CPU oracle: it
only draws random numbers and lays out the COO triples a user's Jacobian
callback would produce (Sec. 3's user callback filling v, Sec. 5's
element-offset layout).  It holds none of the method's arithmetic: no
assembly, no duplicate summation, no SpMV, no solve.

All draws use numpy's PCG64 ``default_rng(seed)``.  Log-uniform means
``10 ** rng.uniform(-1, 1)``; normal means ``rng.standard_normal``.

Workloads (sizes at the defaults):
  * ``poisson2d``      -- 2D 5-point Poisson on an m x m interior grid,
                          h = 1/(m+1), A = h^-2 [4; -1 x4], missing neighbours
                          written as column -1 (ignored entries, Sec. 5);
                          b = 2 pi^2 sin(pi x) sin(pi y).  m = 64: n = 4096,
                          nnz = 20,224.
  * ``q1_hex``         -- 3D Q1 hexahedral FE Poisson on ne^3 elements of the
                          unit cube, 8x8 element blocks stored contiguously
                          (COO index 64 e + 8 a + b), kappa_e log-uniform,
                          Dirichlet on the outer faces (see the function).
                          ne = 96: n = 912,673, ncoo = 56,623,104,
                          nnz = 24,137,569.
  * ``poisson3d``      -- 3D 7-point Laplacian on m^3, h = 1/(m+1), ghosts as -1,
                          b normal.  m = 192: n = 7,077,888, nnz = 49,324,032.
  * ``edge_diffusion`` -- variable-coefficient graph Laplacian of a 2D/3D grid:
                          each edge e=(a,b) adds (a,a,+k), (b,b,+k), (a,b,-k),
                          (b,a,-k); an edge to a Dirichlet ghost uses index -1.
                          1024^2: n = 1,048,576, edges 2,099,200, nnz = 5,238,784.
  * ``batch``          -- 512 independent edge-diffusion systems, even s 2D,
                          odd s 3D, row counts ~ U[1000, 200000].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_C2, SEED_C3, SEED_C4, SEED_C4_SMALL, SEED_C5 = 1002, 1003, 1004, 1014, 1005
SEED_C6 = 1006  # nonsymmetric (convection-diffusion) batches
SEED_C7 = 1007  # right-hand sides of the 2D stencil sweep (time per solve vs NNZ)


@dataclass
class Problem:
    """One linear system given as COO triples plus a right-hand side."""
    name: str
    nrows: int
    ncols: int
    i: np.ndarray            # int32[ncoo], -1 = ignored entry
    j: np.ndarray            # int32[ncoo]
    v: np.ndarray            # float64[ncoo]
    b: np.ndarray            # float64[nrows]
    extra: dict = field(default_factory=dict)

    @property
    def ncoo(self) -> int:
        return int(self.i.shape[0])


@dataclass
class Batch:
    """Independent systems; COO indices are LOCAL to each system and the
    per-system arrays are concatenated in system order."""
    name: str
    nrows: np.ndarray        # int64[nsys]
    ncoo: np.ndarray         # int64[nsys]
    i: np.ndarray            # int32[sum ncoo], local row, -1 = ignored
    j: np.ndarray            # int32[sum ncoo], local col, -1 = ignored
    v: np.ndarray            # float64[sum ncoo]
    b: np.ndarray            # float64[sum nrows]
    extra: dict = field(default_factory=dict)

    @property
    def nsys(self) -> int:
        return int(self.nrows.shape[0])

    @property
    def row_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.nrows)]).astype(np.int64)

    @property
    def coo_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.ncoo)]).astype(np.int64)

    def global_coo(self):
        """Indices shifted to the block-diagonal numbering (ignored stay -1)."""
        shift = np.repeat(self.row_off[:-1], self.ncoo)
        gi = np.where(self.i >= 0, self.i + shift, -1).astype(np.int32)
        gj = np.where(self.j >= 0, self.j + shift, -1).astype(np.int32)
        return gi, gj


# --------------------------------------------------------------------------
# 2D / 3D constant-coefficient stencils (ghost neighbours written as -1)
# --------------------------------------------------------------------------

def _stencil_coo(shape, diag, off):
    """Row-major COO of a (2d+1)-point stencil on an interior grid (x fastest).

    Entry order per row: centre, then -x, +x, -y, +y (, -z, +z); a neighbour
    outside the grid gets column -1."""
    dims = len(shape)
    n = int(np.prod(shape))
    g = np.arange(n, dtype=np.int64)
    coords = []
    rem = g.copy()
    for d in range(dims):
        coords.append(rem % shape[d])
        rem //= shape[d]
    stride = [int(np.prod(shape[:d])) for d in range(dims)]
    cols = [g]
    for d in range(dims):
        for sgn in (-1, 1):
            c = coords[d] + sgn
            ok = (c >= 0) & (c < shape[d])
            cols.append(np.where(ok, g + sgn * stride[d], -1))
    J = np.stack(cols, axis=1).astype(np.int32)            # [n, 2d+1]
    I = np.repeat(np.arange(n, dtype=np.int32), J.shape[1]).reshape(J.shape)
    V = np.empty(J.shape, np.float64)
    V[:, 0] = diag
    V[:, 1:] = off
    return I.reshape(-1), J.reshape(-1), V.reshape(-1)


def poisson2d(m: int = 64) -> Problem:
    """2D 5-point Poisson, Dirichlet, manufactured u = sin(pi x) sin(pi y).

    Interior points x_i = i h, i = 1..m, h = 1/(m+1); node g = (ix-1) + m (iy-1).
    A = h^-2 [4 on the diagonal, -1 per neighbour]; b = 2 pi^2 sin(pi x) sin(pi y)."""
    h = 1.0 / (m + 1)
    I, J, V = _stencil_coo((m, m), 4.0 / h ** 2, -1.0 / h ** 2)
    t = np.arange(1, m + 1) * h
    X, Y = np.meshgrid(t, t, indexing="xy")       # X varies along the fast axis
    u = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1)
    b = 2.0 * np.pi ** 2 * u
    return Problem(f"poisson2d_{m}", m * m, m * m, I, J, V, b,
                   {"h": h, "m": m, "u_exact": u})


def poisson3d(m: int = 192, seed: int = SEED_C3) -> Problem:
    """3D 7-point Laplacian h^-2 [6; -1 x6], h = 1/(m+1), b ~ N(0,1)."""
    h = 1.0 / (m + 1)
    rng = np.random.default_rng(seed)
    I, J, V = _stencil_coo((m, m, m), 6.0 / h ** 2, -1.0 / h ** 2)
    b = rng.standard_normal(m ** 3)
    return Problem(f"poisson3d_{m}", m ** 3, m ** 3, I, J, V, b, {"h": h, "m": m})


def convdiff2d(m: int, bx: float, by: float, seed: int = SEED_C6) -> Problem:
    """2D convection-diffusion -lap u + (bx, by) . grad u on an m x m interior
    grid, h = 1/(m+1), first-order upwind convection (a nonsymmetric M-matrix):
    row = h^-2 [4; -1 x4] plus, for the x direction, |bx|/h on the diagonal
    and -|bx|/h on the upwind neighbour (west if bx > 0, east if bx < 0); the
    same for y.  Entry order per row as _stencil_coo; b ~ N(0,1)."""
    h = 1.0 / (m + 1)
    I, J, V = _stencil_coo((m, m), 4.0 / h ** 2, -1.0 / h ** 2)
    V = V.reshape(-1, 5).copy()
    V[:, 0] += (abs(bx) + abs(by)) / h
    V[:, 1 if bx > 0 else 2] -= abs(bx) / h      # -x or +x neighbour
    V[:, 3 if by > 0 else 4] -= abs(by) / h      # -y or +y neighbour
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(m * m)
    return Problem(f"convdiff2d_{m}", m * m, m * m, I, J, V.reshape(-1), b,
                   {"h": h, "m": m, "velocity": (bx, by)})


def convdiff_batch(nsys: int = 512, seed: int = SEED_C6, size_range=(1000, 50000),
                   peclet=(1.0, 100.0)) -> Batch:
    """Independent 2D convection-diffusion systems (convdiff2d): side
    L = round(sqrt(n_s)) with n_s ~ U_int[lo, hi]; velocity angle ~ U[0, 2 pi)
    and magnitude ~ log-uniform[peclet] (times 1, the domain length).
    Draws in order: all sizes; all angles; all magnitudes; all b."""
    rng = np.random.default_rng(seed)
    target = rng.integers(size_range[0], size_range[1], size=nsys, endpoint=True)
    ang = rng.uniform(0.0, 2.0 * np.pi, size=nsys)
    mag = 10.0 ** rng.uniform(np.log10(peclet[0]), np.log10(peclet[1]), size=nsys)
    Is, Js, Vs, nrows, ncoo = [], [], [], [], []
    for s in range(nsys):
        L = max(2, int(round(float(target[s]) ** 0.5)))
        p = convdiff2d(L, mag[s] * np.cos(ang[s]), mag[s] * np.sin(ang[s]))
        Is.append(p.i); Js.append(p.j); Vs.append(p.v)
        nrows.append(p.nrows); ncoo.append(p.i.shape[0])
    nrows = np.array(nrows, np.int64)
    b = rng.standard_normal(int(nrows.sum()))
    return Batch(f"convdiff_batch_{nsys}", nrows, np.array(ncoo, np.int64),
                 np.concatenate(Is), np.concatenate(Js), np.concatenate(Vs), b,
                 {"angle": ang, "magnitude": mag})


# --------------------------------------------------------------------------
# Q1 hexahedral finite elements (8x8 element blocks, Sec. 5 element offsets)
# --------------------------------------------------------------------------

def q1_reference_stiffness() -> np.ndarray:
    """K_ref[a][b] = integral over the unit cube of grad N_a . grad N_b for the
    trilinear basis, local node a = ax + 2 ay + 4 az.  Closed form by the number
    of coordinates in which a and b differ: 0 -> 1/3, 1 -> 0, 2 -> -1/12,
    3 -> -1/12."""
    table = {0: 1.0 / 3.0, 1: 0.0, 2: -1.0 / 12.0, 3: -1.0 / 12.0}
    K = np.empty((8, 8), np.float64)
    for a in range(8):
        for b in range(8):
            K[a, b] = table[bin(a ^ b).count("1")]
    return K


def q1_load_vector(ne: int = 96, seed: int = SEED_C2 + 100):
    """Element load vector of the Q1 mesh of q1_hex: element e contributes 8
    COO entries (node g(e, a), f_e / 8) in element order, f_e ~ U[0.1, 10].
    Returns (n, i int32[8 ne^3], v float64[8 ne^3])."""
    nn = ne + 1
    rng = np.random.default_rng(seed)
    E = ne ** 3
    e = np.arange(E, dtype=np.int64)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    loc = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], np.int64)
    node = ((ex[:, None] + loc[None, :, 0])
            + nn * ((ey[:, None] + loc[None, :, 1]) + nn * (ez[:, None] + loc[None, :, 2])))
    f = rng.uniform(0.1, 10.0, size=E)
    v = np.repeat(f / 8.0, 8)
    return nn ** 3, node.reshape(-1).astype(np.int32), v


def q1_hex(ne: int = 96, seed: int = SEED_C2, kappa: np.ndarray | None = None) -> Problem:
    """3D Q1 FE Poisson on ne^3 hex elements of the unit cube, h = 1/ne.

    Node g = ix + nn (iy + nn iz), nn = ne + 1; element e = ex + ne (ey + ne ez);
    COO index 64 e + 8 a + b holds (g(e,a), g(e,b), kappa_e h K_ref[a][b]).
    Dirichlet on the outer faces, keeping all nn^3 rows and the full 27-point
    pattern: element entries (a != b) touching a boundary node are set to 0,
    and a boundary node's diagonal element entry is 1/m with m its element
    multiplicity (1, 2 or 4), so that its assembled diagonal is exactly 1.
    kappa_e ~ log-uniform[0.1, 10] (first draw), then b ~ N(0,1) with b = 0 on
    the boundary (second draw)."""
    nn = ne + 1
    h = 1.0 / ne
    rng = np.random.default_rng(seed)
    E = ne ** 3
    if kappa is None:
        kappa = 10.0 ** rng.uniform(-1.0, 1.0, size=E)
    else:
        kappa = np.broadcast_to(np.asarray(kappa, np.float64), (E,)).copy()
        rng.uniform(-1.0, 1.0, size=E)  # keep the draw sequence identical
    n = nn ** 3
    b = rng.standard_normal(n)

    e = np.arange(E, dtype=np.int64)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    loc = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], np.int64)
    node = ((ex[:, None] + loc[None, :, 0])
            + nn * ((ey[:, None] + loc[None, :, 1]) + nn * (ez[:, None] + loc[None, :, 2])))
    node = node.astype(np.int32)                               # [E, 8]
    I = np.repeat(node, 8, axis=1)                             # I[e, 8a+b] = node[e,a]
    J = np.tile(node, (1, 8))                                  # J[e, 8a+b] = node[e,b]
    K = q1_reference_stiffness().reshape(64)
    V = (kappa * h)[:, None] * K[None, :]

    g = np.arange(n, dtype=np.int64)
    gx, gy, gz = g % nn, (g // nn) % nn, g // (nn * nn)
    on = lambda c: (c == 0) | (c == ne)
    bnd = on(gx) | on(gy) | on(gz)
    mult = (np.where(on(gx), 1, 2) * np.where(on(gy), 1, 2) * np.where(on(gz), 1, 2))
    diag_slot = np.zeros(64, bool)
    diag_slot[[9 * a for a in range(8)]] = True
    touch = bnd[I] | bnd[J]
    V[touch & ~diag_slot[None, :]] = 0.0
    dmask = diag_slot[None, :] & bnd[I]
    V[dmask] = 1.0 / mult[I[dmask]]
    b[bnd] = 0.0
    return Problem(f"q1hex_{ne}", n, n, I.reshape(-1), J.reshape(-1), V.reshape(-1), b,
                   {"h": h, "ne": ne, "kappa": kappa, "boundary": bnd})


# --------------------------------------------------------------------------
# Variable-coefficient edge Laplacians (2D / 3D grids)
# --------------------------------------------------------------------------

def grid_edges(shape) -> tuple[np.ndarray, np.ndarray]:
    """Edges of a grid with Dirichlet ghosts, direction-major (x, then y, then
    z), lexicographic with x fastest inside a direction.  Returns (a, b) node
    indices (node = x + nx (y + ny z)); a ghost end is -1."""
    dims = len(shape)
    A, B = [], []
    for d in range(dims):
        eshape = list(shape)
        eshape[d] += 1
        cnt = int(np.prod(eshape))
        k = np.arange(cnt, dtype=np.int64)
        coords, rem = [], k.copy()
        for dd in range(dims):
            coords.append(rem % eshape[dd])
            rem //= eshape[dd]
        def node(cs):
            g = np.zeros(cnt, np.int64)
            s = 1
            for dd in range(dims):
                g += cs[dd] * s
                s *= shape[dd]
            return g
        lo = list(coords)
        lo[d] = coords[d] - 1
        a = np.where(coords[d] >= 1, node(lo), -1)
        b = np.where(coords[d] < shape[d], node(coords), -1)
        A.append(a)
        B.append(b)
    return (np.concatenate(A).astype(np.int32), np.concatenate(B).astype(np.int32))


EDGE_SIGNS = np.array([1.0, 1.0, -1.0, -1.0])


def edge_coo(ea: np.ndarray, eb: np.ndarray, kappa: np.ndarray):
    """4 COO entries per edge, edge-contiguous: (a,a,+k), (b,b,+k), (a,b,-k),
    (b,a,-k).  Any entry touching a ghost (-1) keeps index -1 (ignored)."""
    I = np.stack([ea, eb, ea, eb], axis=1)
    J = np.stack([ea, eb, eb, ea], axis=1)
    gh = (ea < 0) | (eb < 0)
    I[gh, 2:] = -1
    J[gh, 2:] = -1
    V = kappa[:, None] * EDGE_SIGNS[None, :]
    return I.reshape(-1).astype(np.int32), J.reshape(-1).astype(np.int32), V.reshape(-1)


def edge_diffusion(m: int = 1024, seed: int = SEED_C4) -> Problem:
    """2D variable-coefficient 5-point diffusion on m x m: kappa per edge
    log-uniform[0.1, 10] (first draw), b ~ N(0,1) (second), x_target ~ N(0,1)
    (third).  extra carries the edge list and kappa for gradients."""
    rng = np.random.default_rng(seed)
    ea, eb = grid_edges((m, m))
    kappa = 10.0 ** rng.uniform(-1.0, 1.0, size=ea.shape[0])
    b = rng.standard_normal(m * m)
    xt = rng.standard_normal(m * m)
    I, J, V = edge_coo(ea, eb, kappa)
    return Problem(f"edge2d_{m}", m * m, m * m, I, J, V, b,
                   {"edges": (ea, eb), "kappa": kappa, "x_target": xt, "m": m})


def batch(nsys: int = 512, seed: int = SEED_C5, size_range=(1000, 200000)) -> Batch:
    """Independent edge-diffusion systems: s even -> 2D (side L = round(n^(1/2))),
    s odd -> 3D (L = round(n^(1/3))), with n_s ~ U_int[lo, hi] inclusive.
    Draws in order: all sizes; kappa system by system; all b; all x_target."""
    rng = np.random.default_rng(seed)
    target = rng.integers(size_range[0], size_range[1], size=nsys, endpoint=True)
    shapes, nrows = [], []
    for s in range(nsys):
        d = 2 if s % 2 == 0 else 3
        L = max(1, int(round(float(target[s]) ** (1.0 / d))))
        shapes.append((L,) * d)
        nrows.append(L ** d)
    Is, Js, Vs, ncoo, kap, edges = [], [], [], [], [], []
    for s in range(nsys):
        ea, eb = grid_edges(shapes[s])
        k = 10.0 ** rng.uniform(-1.0, 1.0, size=ea.shape[0])
        I, J, V = edge_coo(ea, eb, k)
        Is.append(I); Js.append(J); Vs.append(V); ncoo.append(I.shape[0])
        kap.append(k); edges.append((ea, eb))
    nrows = np.array(nrows, np.int64)
    b = rng.standard_normal(int(nrows.sum()))
    xt = rng.standard_normal(int(nrows.sum()))
    return Batch(f"batch_{nsys}", nrows, np.array(ncoo, np.int64),
                 np.concatenate(Is), np.concatenate(Js), np.concatenate(Vs), b,
                 {"shapes": shapes, "kappa": kap, "edges": edges, "x_target": xt})
