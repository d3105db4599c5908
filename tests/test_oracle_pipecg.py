"""Pins of the oracle's pipelined Jacobi-PCG (one reduction per iteration,
Ghysels-Vanroose; the latency-bound regime of Sec. 6.2's asynchronous
solvers): PCG's iterates in exact arithmetic (same counts, same solutions),
the auxiliary recurrences' invariants (u = M^-1 r, w = A u, s = A p,
q = M^-1 s, z = A q, r = b - A x), dense solves, finite termination with
three eigenvectors, the error paths, the batched driver, and the restart
that brings the true residual to the tolerance where the recursive one
drifted below it."""
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


MAKERS = [lambda: W.edge_diffusion(16, seed=5), lambda: W.q1_hex(6, seed=6),
          lambda: W.poisson3d(9, seed=7), lambda: W.poisson2d(40)]


@pytest.mark.parametrize("make", MAKERS)
def test_same_iterates_as_pcg(make):
    """In exact arithmetic pipelined PCG and PCG produce the same iterates:
    equal iteration counts (to one, for rounding at the threshold) and
    solutions that agree far below the tolerance's scale."""
    p = make()
    A = assemble(p)
    x, r = oracle.pipecg(A, p.b, rtol=1e-10)
    xc, rc = oracle.pcg(A, p.b, rtol=1e-10)
    assert r["status"] == rc["status"] == oracle.OK
    assert abs(r["iterations"] - rc["iterations"]) <= 1, (r, rc)
    assert np.linalg.norm(x - xc) <= 1e-7 * np.linalg.norm(xc)
    assert r["true_rel_residual"] <= 1e-9
    assert r["rnorm0"] == rc["rnorm0"]


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_recurrence_invariants(k):
    """After k iterations the recursively updated vectors still satisfy their
    definitions to rounding: a dropped term, a wrong sign or a swapped vector
    in any of the eight updates breaks one of these."""
    p = W.edge_diffusion(14, seed=3)
    A = assemble(p)
    D = dense(A)
    dinv = 1.0 / np.diag(D)
    x, r, v = oracle.pipecg(A, p.b, rtol=1e-15, maxit=k, want_aux=True)
    assert r["status"] == oracle.ERR_MAXIT and r["iterations"] == k
    scale = np.linalg.norm(D, 2)

    def close(lhs, rhs, ref):
        return np.linalg.norm(lhs - rhs) <= 1e-11 * max(np.linalg.norm(ref), 1e-300) * 10

    assert close(v["r"], p.b - D @ x, scale * np.linalg.norm(x) + np.linalg.norm(p.b))
    assert close(v["u"], dinv * v["r"], dinv.max() * np.linalg.norm(v["r"]))
    assert close(v["w"], D @ v["u"], scale * np.linalg.norm(v["u"]))
    assert close(v["s"], D @ v["p"], scale * np.linalg.norm(v["p"]))
    assert close(v["q"], dinv * v["s"], dinv.max() * np.linalg.norm(v["s"]))
    assert close(v["z"], D @ v["q"], scale * np.linalg.norm(v["q"]))
    # the first step's direction is the preconditioned residual
    x1, r1, v1 = oracle.pipecg(A, p.b, rtol=1e-15, maxit=1, want_aux=True)
    u0 = dinv * p.b
    assert np.allclose(v1["p"], u0, rtol=0, atol=1e-14 * np.abs(u0).max())


def test_dense_spd_solve():
    rng = np.random.default_rng(4)
    n = 30
    G = rng.standard_normal((n, n))
    D = G @ G.T + n * np.eye(n)
    A = from_dense(D)
    b = rng.standard_normal(n)
    x, r = oracle.pipecg(A, b, rtol=1e-12)
    assert r["status"] == oracle.OK
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_finite_termination_three_eigenvectors():
    """Constant diagonal (Jacobi is a scaling) and b in the span of three
    Laplacian eigenvectors: three iterations, as for CG."""
    m = 20
    p = W.poisson2d(m)
    A = assemble(p)
    t = np.arange(1, m + 1) * p.extra["h"]
    X, Y = np.meshgrid(t, t, indexing="xy")
    b = sum(c * np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)
            for c, (j, k) in zip((1.0, 0.5, 2.0), ((1, 1), (3, 2), (7, 9)))).reshape(-1)
    x, res = oracle.pipecg(A, b, rtol=1e-10)
    assert res["status"] == oracle.OK and res["iterations"] == 3


def test_error_paths():
    p = W.poisson2d(8)
    A = assemble(p)
    x, r = oracle.pipecg(A, np.zeros(p.nrows))
    assert r["status"] == oracle.OK and r["iterations"] == 0 and not np.any(x)
    b = p.b.copy()
    b[3] = np.nan
    x, r = oracle.pipecg(A, b)
    assert r["status"] == oracle.ERR_NAN
    rb = np.random.default_rng(9).standard_normal(p.nrows)   # (p.b is an eigenvector)
    x, r = oracle.pipecg(A, rb, rtol=1e-14, maxit=4)
    assert r["status"] == oracle.ERR_MAXIT and r["iterations"] == 4
    D = dense(A)
    D[5, 5] = 0.0
    x, r = oracle.pipecg(from_dense(D), p.b)
    assert r["status"] == oracle.ERR_NOT_SPD
    # an indefinite matrix breaks down (the alpha denominator is p.Ap)
    E = np.diag([2.0, 1.0, 1.0])
    E[0, 1] = E[1, 0] = 3.0
    x, r = oracle.pipecg(from_dense(E), np.array([1.0, -1.0, 0.5]), rtol=1e-12)
    assert r["status"] == oracle.ERR_BREAKDOWN


def test_nonzero_guess():
    p = W.edge_diffusion(10, seed=8)
    A = assemble(p)
    x0 = np.random.default_rng(5).standard_normal(p.nrows)
    x, r = oracle.pipecg(A, p.b, rtol=1e-11, x0=x0)
    xs = np.linalg.solve(dense(A), p.b)
    assert r["status"] == oracle.OK
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert r["rnorm0"] == pytest.approx(np.linalg.norm(p.b - dense(A) @ x0), rel=1e-12)


def test_batched_equals_one_at_a_time():
    bt = W.batch(5, seed=12, size_range=(30, 300))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    A = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(A, bt.v)
    ro, co = bt.row_off, bt.coo_off
    x, rs = oracle.krylov_batched(A, ro, bt.b, oracle.PIPECG, rtol=1e-9)
    for s in range(bt.nsys):
        sl = slice(int(co[s]), int(co[s + 1]))
        As = oracle.coo_symbolic(int(bt.nrows[s]), int(bt.nrows[s]), bt.i[sl], bt.j[sl])
        oracle.coo_numeric(As, bt.v[sl])
        xs, r = oracle.pipecg(As, bt.b[ro[s]:ro[s + 1]], rtol=1e-9)
        assert x[ro[s]:ro[s + 1]].tobytes() == xs.tobytes()
        assert rs[s]["iterations"] == r["iterations"] and r["status"] == oracle.OK


def test_restart_confirms_the_true_residual():
    """On a 512 x 512 Laplacian (kappa ~ 1e5) the recursive residual of
    pipelined CG falls below rtol ||b|| while b - A x is still above it; the
    confirmation catches that and restarts the recurrences from x, and the
    solve ends with the true residual within the tolerance, after about as
    many x updates as CG needs."""
    m = 512
    p = W.poisson2d(m)
    b = np.random.default_rng(1007 + m).standard_normal(p.nrows)
    A = assemble(p)
    x, r = oracle.pipecg(A, b, rtol=1e-8)
    xc, rc = oracle.pcg(A, b, rtol=1e-8)
    assert r["status"] == oracle.OK
    assert r["outer_iterations"] >= 1                      # at least one restart
    assert r["true_rel_residual"] <= 1e-8 * (1 + 1e-6)
    assert abs(r["rnorm"] / np.linalg.norm(b) - r["true_rel_residual"]) <= 1e-12
    assert rc["iterations"] <= r["iterations"] <= 1.2 * rc["iterations"]


def test_restart_reinitialises_the_recurrences():
    """After a restart the invariants hold again (u = M^-1 r, w = A u, and
    p, s, q, z consistent), checked at the end of the solve, some iterations
    past the restart: the drift the recurrences accumulate after it is a few
    parts in a million of these small vectors; a restart that left any of
    them stale would be off by order one."""
    m = 512
    p = W.poisson2d(m)
    b = np.random.default_rng(1007 + m).standard_normal(p.nrows)
    A = assemble(p)
    x0, r0 = oracle.pipecg(A, b, rtol=1e-8)
    k = r0["iterations"]                   # an iteration limit just past the restart
    x, r, v = oracle.pipecg(A, b, rtol=1e-8, maxit=k, want_aux=True)
    import scipy.sparse as sp
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.nrows, A.nrows))
    dinv = 1.0 / S.diagonal()
    nr = lambda t: np.linalg.norm(t)
    assert nr(v["r"] - (b - S @ x)) <= 1e-6 * nr(b)
    assert r["outer_iterations"] >= 1
    assert nr(v["u"] - dinv * v["r"]) <= 1e-4 * nr(dinv * v["r"])
    assert nr(v["w"] - S @ v["u"]) <= 1e-4 * nr(S @ v["u"])
    assert nr(v["s"] - S @ v["p"]) <= 1e-4 * nr(S @ v["p"])
    assert nr(v["q"] - dinv * v["s"]) <= 1e-4 * nr(dinv * v["s"])


def test_batched_degenerate_systems():
    """A batch holding a 2 x 2 SPD block, an empty system, a 1 x 1 system and a
    system with b = 0: CG's finite termination carries over to the pipelined
    recurrences (2 and 1 iterations), x = b / a for the 1 x 1 block, x = 0
    with no iteration where b = 0, nothing to do for the empty system."""
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
    x, rs = oracle.krylov_batched(A, np.array(off), b, oracle.PIPECG, rtol=1e-12)
    assert [r["status"] for r in rs] == [oracle.OK] * 4
    assert [r["iterations"] for r in rs] == [2, 0, 1, 0]
    assert all(r["outer_iterations"] == 0 for r in rs)          # no restart needed
    assert not np.any(x[3:])
    xs = np.linalg.solve(blocks[0], b[:2])
    assert np.linalg.norm(x[:2] - xs) <= 1e-12 * np.linalg.norm(xs) * 10
    assert abs(x[2] - 2.0) <= 4 * np.spacing(2.0)
