"""Pins of the oracle's SpMV (MatMult, Sec. 6.1) and of the workload generators
(closed-form Laplacian eigenpairs, the Q1 element stencil, exact pattern
counts)."""
import numpy as np
import pytest

import oracle
from paper_2406_08646_gb300 import workloads as W


def assemble(p):
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(A, p.v)
    return A


def dense(A):
    D = np.zeros((A.nrows, A.ncols))
    for r in range(A.nrows):
        for q in range(A.row_ptr[r], A.row_ptr[r + 1]):
            D[r, A.col[q]] = A.val[q]
    return D


def test_spmv_matches_dense_matvec():
    rng = np.random.default_rng(1)
    n = 120
    i = rng.integers(0, n, 2000).astype(np.int32)
    j = rng.integers(0, n, 2000).astype(np.int32)
    A = oracle.coo_symbolic(n, n, i, j)
    oracle.coo_numeric(A, rng.standard_normal(2000))
    x = rng.standard_normal(n)
    y = oracle.spmv(A, x)
    D = dense(A)
    bound = np.abs(D) @ np.abs(x)
    assert np.all(np.abs(y - D @ x) <= 1e-14 * bound)
    # an empty row gives exactly 0
    E = oracle.coo_symbolic(3, 3, np.array([0, 2], np.int32), np.array([1, 2], np.int32))
    oracle.coo_numeric(E, np.array([2.0, 3.0]))
    assert oracle.spmv(E, np.ones(3)).tolist() == [2.0, 0.0, 3.0]


@pytest.mark.parametrize("jk", [(1, 1), (2, 3), (5, 1), (15, 16), (16, 16)])
def test_laplacian_eigenpairs(jk):
    m = 16
    p = W.poisson2d(m)
    A = assemble(p)
    h = p.extra["h"]
    j, k = jk
    t = np.arange(1, m + 1) * h
    X, Y = np.meshgrid(t, t, indexing="xy")
    v = (np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)).reshape(-1)
    lam = 4.0 / h ** 2 * (np.sin(j * np.pi * h / 2) ** 2 + np.sin(k * np.pi * h / 2) ** 2)
    y = oracle.spmv(A, v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13 * lam * np.max(np.abs(v))


def test_c1_counts_and_rhs_is_eigenvector():
    p = W.poisson2d(64)
    A = assemble(p)
    assert p.nrows == 4096 and A.nnz == 20224 and p.ncoo == 5 * 4096
    h = p.extra["h"]
    lam11 = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    y = oracle.spmv(A, p.b)
    assert np.max(np.abs(y - lam11 * p.b)) <= 1e-12 * lam11 * np.max(np.abs(p.b))
    assert abs(2 * np.pi ** 2 / lam11 - 1.00019469) < 1e-8


def test_q1_reference_stiffness_by_quadrature():
    """K_ref from 2-point Gauss quadrature of the trilinear basis gradients
    (exact for these polynomial integrands), independent of the closed form."""
    g = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    K = np.zeros((8, 8))
    def grad(a, x, y, z):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        f = lambda c, s: c if s else 1 - c
        df = lambda s: 1.0 if s else -1.0
        return np.array([df(ax) * f(y, ay) * f(z, az),
                         f(x, ax) * df(ay) * f(z, az),
                         f(x, ax) * f(y, ay) * df(az)])
    for x in g:
        for y in g:
            for z in g:
                G = np.array([grad(a, x, y, z) for a in range(8)])
                K += 0.125 * G @ G.T
    assert np.allclose(K, W.q1_reference_stiffness(), atol=1e-15)


def test_q1_assembled_constant_kappa_stencil():
    ne = 6
    p = W.q1_hex(ne, kappa=1.0)
    A = assemble(p)
    nn = ne + 1
    assert A.nnz == (3 * nn - 2) ** 3
    h = p.extra["h"]
    bnd = p.extra["boundary"]
    cls = {0: 8.0 / 3.0, 1: 0.0, 2: -1.0 / 6.0, 3: -1.0 / 12.0}
    for r in range(A.nrows):
        cols = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        vals = A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
        rx, ry, rz = r % nn, (r // nn) % nn, r // (nn * nn)
        if bnd[r]:
            assert vals[cols == r].tolist() == [1.0]          # exactly 1 (dyadic sum)
            assert np.all(vals[cols != r] == 0.0)
            continue
        for c, v in zip(cols, vals):
            cx, cy, cz = c % nn, (c // nn) % nn, c // (nn * nn)
            d = int(abs(cx - rx) + abs(cy - ry) + abs(cz - rz) > 0) * \
                sum(int(a != b) for a, b in ((cx, rx), (cy, ry), (cz, rz)))
            expect = 0.0 if bnd[c] and c != r else h * cls[d]
            assert abs(v - expect) <= 1e-15 * h * 3, (r, c, v, expect)
    # rows away from the boundary sum to zero (constant kappa)
    y = oracle.spmv(A, np.ones(A.nrows))
    deep = [r for r in range(A.nrows)
            if all(1 < c < ne - 1 for c in (r % nn, (r // nn) % nn, r // (nn * nn)))]
    assert np.max(np.abs(y[deep])) <= 1e-15


def test_q1_full_size_counts():
    nn = 97
    assert nn ** 3 == 912_673 and 96 ** 3 * 64 == 56_623_104 and (3 * nn - 2) ** 3 == 24_137_569


def test_edge_counts_and_symmetry():
    p = W.edge_diffusion(16, seed=3)
    A = assemble(p)
    m = 16
    ea, eb = p.extra["edges"]
    assert ea.shape[0] == 2 * m * (m + 1)
    assert A.nnz == 5 * m * m - 4 * m
    assert oracle.is_symmetric(A)
    # graph Laplacian plus boundary terms: A 1 = sum of ghost-edge kappas per row
    ghost = (ea < 0) | (eb < 0)
    expect = np.zeros(m * m)
    real = np.where(ea >= 0, ea, eb)
    np.add.at(expect, real[ghost], p.extra["kappa"][ghost])
    y = oracle.spmv(A, np.ones(m * m))
    assert np.allclose(y, expect, rtol=1e-13, atol=1e-13)
    assert 2 * 1024 * 1025 == 2_099_200 and 5 * 1024 ** 2 - 4 * 1024 == 5_238_784


def test_3d_edges_and_stencil_counts():
    ea, eb = W.grid_edges((3, 4, 5))
    assert ea.shape[0] == 4 * 4 * 5 + 3 * 5 * 5 + 3 * 4 * 6
    p = W.poisson3d(6, seed=1)
    A = assemble(p)
    assert A.nnz == 7 * 216 - 6 * 36
    assert 7 * 192 ** 3 - 6 * 192 ** 2 == 49_324_032
