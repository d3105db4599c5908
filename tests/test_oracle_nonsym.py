"""Pins of the oracle's nonsymmetric solvers (Sec. 7's batched BiCG and TFQMR
with the diagonal preconditioner): dense solves, BiCG = PCG operation for
operation on symmetric input, TFQMR's quasi-residual bound, finite
termination on tiny systems, and batched = one system at a time."""
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
            D[r, A.col[q]] += A.val[q]
    return D


@pytest.mark.parametrize("make", [lambda: W.poisson2d(12), lambda: W.q1_hex(4, seed=3),
                                  lambda: W.edge_diffusion(9, seed=5)])
def test_bicg_is_pcg_on_symmetric_input(make):
    p = make()
    A = assemble(p)
    xb, rb = oracle.bicg(A, p.b, rtol=1e-10)
    xc, rc = oracle.pcg(A, p.b, rtol=1e-10)
    assert rb["status"] == rc["status"] == oracle.OK
    assert rb["iterations"] == rc["iterations"]
    assert xb.tobytes() == xc.tobytes()


@pytest.mark.parametrize("solver", [oracle.bicg, oracle.tfqmr])
@pytest.mark.parametrize("vel", [(5.0, 0.0), (-20.0, 7.0), (60.0, -80.0)])
def test_nonsymmetric_against_dense_solve(solver, vel):
    p = W.convdiff2d(14, *vel, seed=4)
    A = assemble(p)
    D = dense(A)
    assert not np.allclose(D, D.T)
    xs = np.linalg.solve(D, p.b)
    x, r = solver(A, p.b, rtol=1e-10)
    assert r["status"] == oracle.OK, r
    tr = np.linalg.norm(p.b - D @ x) / np.linalg.norm(p.b)
    # BiCG stops on its updated residual, TFQMR on its quasi-residual bound;
    # in FP64 both can sit a little above the true residual (residual gap)
    assert tr <= (1.5e-10 if solver is oracle.bicg else 5e-10), tr
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr + 1e-15
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.cond(D) * np.linalg.norm(xs)


def test_tfqmr_quasi_residual_bounds_the_true_residual():
    """tau sqrt(m+1) bounds ||b - A x_m|| at every stop, converged or not."""
    p = W.convdiff2d(20, 30.0, -10.0, seed=7)
    A = assemble(p)
    bn = np.linalg.norm(p.b)
    for maxit in (3, 8, 21, 50):
        x, r = oracle.tfqmr(A, p.b, rtol=1e-14, maxit=maxit)
        assert r["status"] == oracle.ERR_MAXIT
        assert r["true_rel_residual"] * bn <= r["rnorm"] * (1 + 1e-9)


@pytest.mark.parametrize("solver", [oracle.bicg, oracle.tfqmr])
def test_finite_termination_on_a_tiny_system(solver):
    rng = np.random.default_rng(2)
    n = 6
    D = rng.standard_normal((n, n)) + 8.0 * np.eye(n)
    i, j = np.nonzero(np.ones((n, n)))
    A = oracle.coo_symbolic(n, n, i.astype(np.int32), j.astype(np.int32))
    oracle.coo_numeric(A, D[i, j])
    b = rng.standard_normal(n)
    x, r = solver(A, b, rtol=1e-12)
    assert r["status"] == oracle.OK
    # Krylov space of dimension n: n products for BiCG, about 2n for TFQMR
    assert r["iterations"] <= (n + 2 if solver is oracle.bicg else 2 * n + 4)
    assert np.linalg.norm(D @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_batched_equals_one_at_a_time():
    bt = W.convdiff_batch(6, seed=11, size_range=(50, 400))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    A = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(A, bt.v)
    ro, co = bt.row_off, bt.coo_off
    for method, solver in ((oracle.BICG, oracle.bicg), (oracle.TFQMR, oracle.tfqmr)):
        x, rs = oracle.krylov_batched(A, ro, bt.b, method, rtol=1e-9)
        for s in range(bt.nsys):
            sl = slice(int(co[s]), int(co[s + 1]))
            As = oracle.coo_symbolic(int(bt.nrows[s]), int(bt.nrows[s]), bt.i[sl], bt.j[sl])
            oracle.coo_numeric(As, bt.v[sl])
            xs, r = solver(As, bt.b[ro[s]:ro[s + 1]], rtol=1e-9)
            assert x[ro[s]:ro[s + 1]].tobytes() == xs.tobytes()
            assert rs[s]["iterations"] == r["iterations"] and r["status"] == oracle.OK


def test_error_statuses():
    p = W.convdiff2d(6, 3.0, 3.0, seed=1)
    A = assemble(p)
    b = p.b.copy()
    b[0] = np.nan
    for solver in (oracle.bicg, oracle.tfqmr):
        assert solver(A, b)[1]["status"] == oracle.ERR_NAN
        x, r = solver(A, np.zeros(p.nrows))
        assert r["status"] == oracle.OK and r["iterations"] == 0 and not x.any()
        assert solver(A, p.b, rtol=1e-14, maxit=2)[1]["status"] == oracle.ERR_MAXIT


@pytest.mark.parametrize("method", ["bicg", "tfqmr"])
def test_batched_degenerate_systems(method):
    """A batch holding a 2 x 2 nonsymmetric block, an empty system, a 1 x 1
    system and a system with b = 0: the 2 x 2 and 1 x 1 solves reach the dense
    solution within BiCG's n-step finite termination (TFQMR: two half steps
    per BiCG step, plus its closing one), x = 0 with no iteration where b = 0,
    and nothing to do for the empty system."""
    blocks = [np.array([[4.0, 1.5], [-0.5, 3.0]]), np.zeros((0, 0)), np.array([[2.5]]),
              np.array([[2.0, -1.3, 0.0], [-0.7, 2.0, -1.0], [0.0, -1.0, 2.0]])]
    N = sum(B_.shape[0] for B_ in blocks)
    D = np.zeros((N, N))
    off = [0]
    for B_ in blocks:
        o, n = off[-1], B_.shape[0]
        D[o:o + n, o:o + n] = B_
        off.append(o + n)
    i, j = np.nonzero(D)
    A = oracle.coo_symbolic(N, N, i.astype(np.int32), j.astype(np.int32))
    oracle.coo_numeric(A, D[i, j])
    b = np.array([1.0, 2.0, 5.0, 0.0, 0.0, 0.0])
    m = oracle.BICG if method == "bicg" else oracle.TFQMR
    x, rs = oracle.krylov_batched(A, np.array(off), b, m, rtol=1e-12)
    assert [r["status"] for r in rs] == [oracle.OK] * 4
    assert rs[1]["iterations"] == 0 and rs[3]["iterations"] == 0
    assert not np.any(x[3:])
    xs = np.linalg.solve(blocks[0], b[:2])
    assert np.linalg.norm(x[:2] - xs) <= 1e-11 * np.linalg.norm(xs)
    assert abs(x[2] - 2.0) <= 4 * np.spacing(2.0)
    steps = [2, 0, 1, 0]
    for r, n in zip(rs, steps):
        limit = n if method == "bicg" else 2 * n + (n > 0)
        assert r["iterations"] <= limit, (method, r, n)
