"""Pins of the oracle's Jacobi-PCG (Sec. 6.1 CG with the diagonal preconditioner
of Sec. 7), FP32-refined form (Sec. 2 multiprecision), adjoint (Sec. 1) and
batched form (Sec. 7): dense solves, closed forms, finite termination, the CG
error bound, finite differences and the error paths."""
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
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    D[rows, A.col] = A.val
    return D


def from_dense(D):
    i, j = np.nonzero(D)
    A = oracle.coo_symbolic(D.shape[0], D.shape[1], i.astype(np.int32), j.astype(np.int32))
    oracle.coo_numeric(A, D[i, j])
    return A


# ---------------------------------------------------------------- FP64 PCG

@pytest.mark.parametrize("make", [lambda: W.edge_diffusion(12, seed=5),
                                  lambda: W.q1_hex(5, seed=6),
                                  lambda: W.poisson3d(7, seed=7)])
def test_pcg_matches_dense_solve(make):
    p = make()
    A = assemble(p)
    x, res = oracle.pcg(A, p.b, rtol=1e-10)
    assert res["status"] == oracle.OK
    D = dense(A)
    xs = np.linalg.solve(D, p.b)
    cond = np.linalg.cond(D)
    assert res["true_rel_residual"] <= 1e-10 * 1.01
    assert np.linalg.norm(x - xs) <= cond * 1e-10 * np.linalg.norm(xs) * 2
    assert np.linalg.norm(D @ x - p.b) <= 1.01e-10 * np.linalg.norm(p.b)


def test_c1_closed_form_one_iteration():
    p = W.poisson2d(64)
    A = assemble(p)
    x, res = oracle.pcg(A, p.b, rtol=1e-8)
    h = p.extra["h"]
    lam11 = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    xc = 2 * np.pi ** 2 / lam11 * p.extra["u_exact"]
    assert res["status"] == oracle.OK and 1 <= res["iterations"] <= 2
    assert np.max(np.abs(x - xc)) <= 1e-12
    # discrete solution approximates u = sin(pi x) sin(pi y) to O(h^2)
    assert np.max(np.abs(x - p.extra["u_exact"])) <= 2 * h ** 2


def test_finite_termination_three_eigenvectors():
    m = 20
    p = W.poisson2d(m)
    A = assemble(p)
    t = np.arange(1, m + 1) * p.extra["h"]
    X, Y = np.meshgrid(t, t, indexing="xy")
    b = sum(c * np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)
            for c, (j, k) in zip((1.0, 0.5, 2.0), ((1, 1), (3, 2), (7, 9)))).reshape(-1)
    x, res = oracle.pcg(A, b, rtol=1e-10)
    assert res["status"] == oracle.OK and res["iterations"] == 3


def test_cg_error_bound():
    """||e_k||_A <= 2 ((sqrt k - 1)/(sqrt k + 1))^k ||e_0||_A with the closed-form
    condition number of the 2D Laplacian (Jacobi is a constant scaling here)."""
    m = 24
    p = W.poisson2d(m)
    A = assemble(p)
    D = dense(A)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(m * m)
    xs = np.linalg.solve(D, b)
    h = p.extra["h"]
    kappa = np.sin(m * np.pi * h / 2) ** 2 / np.sin(np.pi * h / 2) ** 2
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    anorm = lambda e: np.sqrt(e @ D @ e)
    e0 = anorm(xs)
    for k in (1, 5, 10, 20, 40):
        x, res = oracle.pcg(A, b, rtol=1e-14, maxit=k)
        assert res["status"] == oracle.ERR_MAXIT and res["iterations"] == k
        assert anorm(x - xs) <= 2 * q ** k * e0 * (1 + 1e-9)


def test_pcg_error_paths():
    rng = np.random.default_rng(4)
    D = np.diag([2.0, 0.0, 3.0]) + 0.1 * (np.ones((3, 3)) - np.eye(3))
    x, r = oracle.pcg(from_dense(D), np.ones(3))
    assert r["status"] == oracle.ERR_NOT_SPD              # missing / zero diagonal
    D = np.diag([2.0, -1.0, 3.0])
    assert oracle.pcg(from_dense(D), np.ones(3))[1]["status"] == oracle.ERR_NOT_SPD
    D = np.array([[1.0, 3.0], [3.0, 1.0]])                 # indefinite, positive diagonal
    assert oracle.pcg(from_dense(D), np.array([1.0, -1.0]))[1]["status"] == oracle.ERR_BREAKDOWN
    A = assemble(W.poisson2d(8))
    b = rng.standard_normal(64)
    b[5] = np.nan
    assert oracle.pcg(A, b)[1]["status"] == oracle.ERR_NAN
    x, r = oracle.pcg(A, rng.standard_normal(64), maxit=1)
    assert r["status"] == oracle.ERR_MAXIT and r["iterations"] == 1
    x, r = oracle.pcg(A, np.zeros(64))
    assert r["status"] == oracle.OK and r["iterations"] == 0 and np.all(x == 0)


def test_nonzero_initial_guess():
    p = W.edge_diffusion(10, seed=2)
    A = assemble(p)
    xs = np.linalg.solve(dense(A), p.b)
    x, r = oracle.pcg(A, p.b, rtol=1e-8, x0=xs)
    assert r["status"] == oracle.OK and r["iterations"] == 0
    x1, r1 = oracle.pcg(A, p.b, rtol=1e-10, x0=0.5 * xs)
    assert r1["status"] == oracle.OK and r1["true_rel_residual"] <= 1.01e-10


# ---------------------------------------------------------------- FP32-refined

@pytest.mark.parametrize("make", [lambda: W.q1_hex(6, seed=11),
                                  lambda: W.poisson3d(10, seed=12)])
def test_refined_reaches_fp64_residual(make):
    p = make()
    A = assemble(p)
    x, r = oracle.pcg_refined(A, p.b, rtol=1e-10, inner_rtol=1e-4)
    assert r["status"] == oracle.OK
    assert r["true_rel_residual"] <= 1e-10
    assert r["outer_iterations"] >= 2
    D = dense(A)
    xs = np.linalg.solve(D, p.b)
    assert np.linalg.norm(x - xs) <= np.linalg.cond(D) * 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(D @ x - p.b) <= 1.0001e-10 * np.linalg.norm(p.b)


def test_refined_fp32_inner_is_really_fp32():
    """One outer step with an exact inner solve cannot beat FP32 rounding: the
    residual after the first correction is ~1e-7, not ~1e-15."""
    p = W.poisson3d(8, seed=13)
    A = assemble(p)
    x, r = oracle.pcg_refined(A, p.b, rtol=1e-30, inner_rtol=1e-12, max_outer=1)
    assert r["status"] == oracle.ERR_MAXIT and r["outer_iterations"] == 1
    assert 1e-9 < r["true_rel_residual"] < 1e-4


def test_refined_stagnation_and_maxit():
    p = W.poisson3d(10, seed=14)
    A = assemble(p)
    x, r = oracle.pcg_refined(A, p.b, rtol=1e-10, inner_rtol=0.9, inner_maxit=1)
    assert r["status"] == oracle.ERR_STAGNATION
    x, r = oracle.pcg_refined(A, p.b, rtol=1e-10, max_outer=1)
    assert r["status"] == oracle.ERR_MAXIT and r["outer_iterations"] == 1


# ---------------------------------------------------------------- adjoint

def _loss_dense(D_of_kappa, b, xt):
    D = D_of_kappa
    x = np.linalg.solve(D, b)
    return 0.5 * np.sum((x - xt) ** 2), x


def _edge_dense(m, ea, eb, kappa):
    n = m * m
    D = np.zeros((n, n))
    for a, b_, k in zip(ea, eb, kappa):
        if a >= 0:
            D[a, a] += k
        if b_ >= 0:
            D[b_, b_] += k
        if a >= 0 and b_ >= 0:
            D[a, b_] -= k
            D[b_, a] -= k
    return D


def _kappa_grad_from_dldv(dldv, nedges):
    return (dldv.reshape(nedges, 4) * W.EDGE_SIGNS[None, :]).sum(axis=1)


def test_adjoint_dense_reference_and_finite_differences():
    p = W.edge_diffusion(32, seed=W.SEED_C4_SMALL)
    m = 32
    ea, eb = p.extra["edges"]
    kappa = p.extra["kappa"]
    xt = p.extra["x_target"]
    A = assemble(p)
    assert oracle.is_symmetric(A)
    x, r = oracle.pcg(A, p.b, rtol=1e-13)
    assert r["status"] == oracle.OK
    lam, dlda, dldv, ra = oracle.adjoint(A, x, x - xt, rtol=1e-13)
    assert ra["status"] == oracle.OK
    gk = _kappa_grad_from_dldv(dldv, ea.shape[0])

    # (i) dense reference gradient: lambda = A^-1 (x - xt), dL/dk = -(l_a - l_b)(x_a - x_b)
    D = _edge_dense(m, ea, eb, kappa)
    xd = np.linalg.solve(D, p.b)
    ld = np.linalg.solve(D, xd - xt)
    la = np.where(ea >= 0, ld[ea], 0.0)
    lb = np.where(eb >= 0, ld[eb], 0.0)
    xa = np.where(ea >= 0, xd[ea], 0.0)
    xb = np.where(eb >= 0, xd[eb], 0.0)
    gref = -(la - lb) * (xa - xb)
    assert np.linalg.norm(gk - gref) <= 1e-10 * np.linalg.norm(gref)
    assert np.linalg.norm(lam - ld) <= 1e-10 * np.linalg.norm(ld)

    # (ii) central finite differences on kappa: 128 sampled edges + 4 directions
    rng = np.random.default_rng(0)
    L = lambda kap, bb=p.b: _loss_dense(_edge_dense(m, ea, eb, kap), bb, xt)[0]
    for e in rng.choice(ea.shape[0], 128, replace=False):
        eps = 1e-6 * kappa[e]
        kp, km = kappa.copy(), kappa.copy()
        kp[e] += eps
        km[e] -= eps
        Lp, Lm = L(kp), L(km)
        fd = (Lp - Lm) / (2 * eps)
        # 1e-6 relative, plus the rounding of the two loss values (a few ulps of L)
        noise = 20 * np.finfo(float).eps * abs(Lp) / eps
        assert abs(fd - gk[e]) <= 1e-6 * abs(gk[e]) + noise, e
    for _ in range(4):
        d = rng.standard_normal(ea.shape[0]) * kappa
        eps = 1e-6
        fd = (L(kappa + eps * d) - L(kappa - eps * d)) / (2 * eps)
        assert abs(fd - gk @ d) <= 1e-6 * abs(gk @ d)
    # (iii) finite differences on b along random directions: dL/db = lambda
    for _ in range(4):
        d = rng.standard_normal(m * m)
        eps = 1e-6
        fd = (L(kappa, p.b + eps * d) - L(kappa, p.b - eps * d)) / (2 * eps)
        assert abs(fd - lam @ d) <= 1e-6 * abs(lam @ d)


def test_adjoint_requires_symmetry():
    D = np.array([[2.0, 0.5], [0.1, 2.0]])
    A = from_dense(D)
    lam, dlda, dldv, r = oracle.adjoint(A, np.ones(2), np.ones(2))
    assert r["status"] == oracle.ERR_ARG


# ---------------------------------------------------------------- batched

def test_batched_each_system_matches_dense():
    bt = W.batch(6, seed=21, size_range=(50, 700))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    A = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(A, bt.v)
    D = dense(A)
    ro = bt.row_off
    for prec in (0, 1):
        x, rs = oracle.pcg_batched(A, ro, bt.b, rtol=1e-10, precision=prec)
        for s in range(bt.nsys):
            sl = slice(ro[s], ro[s + 1])
            Ds = D[sl, sl]
            assert np.count_nonzero(D[sl, :]) == np.count_nonzero(Ds)   # block diagonal
            assert rs[s]["status"] == oracle.OK
            assert np.linalg.norm(Ds @ x[sl] - bt.b[sl]) <= 1.01e-10 * np.linalg.norm(bt.b[sl])
            xs = np.linalg.solve(Ds, bt.b[sl])
            assert np.linalg.norm(x[sl] - xs) <= np.linalg.cond(Ds) * 2e-10 * np.linalg.norm(xs)


def test_batched_degenerate_systems_closed_forms():
    """A batch holding a 2 x 2 SPD block, an empty system, a 1 x 1 system and a
    system with b = 0: CG's finite termination (at most n iterations, here 2
    and 1), x = b / a for the 1 x 1 block (Jacobi-PCG takes alpha = 1 there),
    x = 0 with no iteration for b = 0, and nothing to do for the empty one --
    in FP64 and in the refined form."""
    blocks = [np.array([[4.0, 1.0], [1.0, 3.0]]), np.zeros((0, 0)), np.array([[2.5]]),
              np.array([[2.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 2.0]])]
    N = sum(B_.shape[0] for B_ in blocks)
    D = np.zeros((N, N))
    off = [0]
    for B_ in blocks:
        o, n = off[-1], B_.shape[0]
        D[o:o + n, o:o + n] = B_
        off.append(o + n)
    A = from_dense(D)
    b = np.array([1.0, 2.0, 5.0, 0.0, 0.0, 0.0])
    for prec in (0, 1):
        x, rs = oracle.pcg_batched(A, np.array(off), b, rtol=1e-12, precision=prec)
        assert [r["status"] for r in rs] == [oracle.OK] * 4
        assert rs[1]["iterations"] == 0 and rs[3]["iterations"] == 0
        assert not np.any(x[3:])                                   # b = 0: x = 0 exactly
        xs = np.linalg.solve(blocks[0], b[:2])
        assert np.linalg.norm(x[:2] - xs) <= 1e-12 * np.linalg.norm(xs) * 10
        assert abs(x[2] - 5.0 / 2.5) <= 4 * np.spacing(2.0)
        if prec == 0:
            assert rs[0]["iterations"] == 2 and rs[2]["iterations"] == 1


def test_all_cores_build_gives_the_same_bits():
    """The OpenMP build of the oracle (the all-cores CPU baseline) splits only
    loops whose iterations write separate elements and keeps the inner
    products sequential: assembly, SpMV and the PCG solve are bit-identical
    to the one-thread build."""
    p = W.q1_hex(10, seed=4)
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    v1 = oracle.coo_numeric(A, p.v).copy()
    v2 = oracle.coo_numeric(A, p.v, omp=True).copy()
    assert v1.tobytes() == v2.tobytes()
    y1, y2 = oracle.spmv(A, p.b), oracle.spmv(A, p.b, omp=True)
    assert y1.tobytes() == y2.tobytes()
    x1, r1 = oracle.pcg(A, p.b, rtol=1e-10)
    x2, r2 = oracle.pcg(A, p.b, rtol=1e-10, omp=True)
    assert x1.tobytes() == x2.tobytes() and r1 == r2
