"""GPU parity of the pipelined Jacobi-PCG (one fused kernel and one reduction
per iteration; the latency-bound regime of Sec. 6.2's asynchronous solvers)
against the oracle's pipelined PCG, through ksp_solve / ksp_solve_batched.

Bars: statuses equal to the oracle's; iteration counts within max(2, 1%) of
the oracle's (only the summation order of the three dot products differs),
equal under an iteration limit (iterates equal to 1e-10); the relative true
residual recomputed by the oracle from the GPU's x at most
2 max(rtol, the oracle's own true residual) (the pipelined recurrences let
the recursive residual drift from b - A x more than CG's do); the GPU's
closing true residual within 1e-3 of the recomputation; the iteration count
within 2 of the GPU's own CG (same iterates in exact arithmetic)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_08646_gb300 import binding as B
from paper_2406_08646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def iters_close(a, b):
    return abs(a - b) <= max(2, int(np.ceil(0.01 * max(a, b))))


def resid_ok(tr, ro, rtol):
    return tr <= 2 * max(rtol, ro["true_rel_residual"])


def true_rel(O, b, x):
    return np.linalg.norm(b - oracle.spmv(O, x)) / np.linalg.norm(b)


def single(p):
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    A.set_values(t(p.v))
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    return A, O


def with_random_rhs(p, seed):
    p.b = np.random.default_rng(seed).standard_normal(p.nrows)
    return p


@pytest.mark.parametrize("name,make,rtol", [
    ("poisson2d_64", lambda: with_random_rhs(W.poisson2d(64), 1), 1e-8),
    ("q1hex_12", lambda: W.q1_hex(12, seed=W.SEED_C2), 1e-8),
    ("poisson3d_24", lambda: W.poisson3d(24, seed=W.SEED_C3), 1e-10),
    ("edge_32", lambda: W.edge_diffusion(32, seed=W.SEED_C4_SMALL), 1e-8),
    ("edge_300", lambda: W.edge_diffusion(300, seed=9), 1e-8),
])
def test_pipecg_parity(name, make, rtol):
    p = make()
    A, O = single(p)
    x, r = A.solve(t(p.b), rtol=rtol, method=B.KSP_PIPECG)
    xo, ro = oracle.pipecg(O, p.b, rtol=rtol)
    assert r["status"] == ro["status"] == B.OK, (r, ro)
    assert r["solver"] == B.SOLVER_PHASES
    assert iters_close(r["iterations"], ro["iterations"]), (r, ro)
    tr = true_rel(O, p.b, x.cpu().numpy())
    assert resid_ok(tr, ro, rtol), (tr, ro)
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr + 1e-15
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    assert r["outer_iterations"] == ro["outer_iterations"]   # restarts (none here)
    xc, rc = A.solve(t(p.b), rtol=rtol)                 # the GPU's CG
    assert abs(r["iterations"] - rc["iterations"]) <= 2, (r, rc)
    A.close()


def test_restart_when_the_recursive_residual_drifts():
    """512 x 512 Laplacian, random rhs: the recursive residual meets rtol
    before b - A x does; the confirmation restarts the recurrences, as in the
    oracle, and the solve ends with the true residual within rtol."""
    m = 512
    p = W.poisson2d(m)
    p.b = np.random.default_rng(1007 + m).standard_normal(p.nrows)
    A, O = single(p)
    x, r = A.solve(t(p.b), rtol=1e-8, method=B.KSP_PIPECG)
    xo, ro = oracle.pipecg(O, p.b, rtol=1e-8)
    assert r["status"] == ro["status"] == B.OK
    assert r["outer_iterations"] >= 1 and ro["outer_iterations"] >= 1
    tr = true_rel(O, p.b, x.cpu().numpy())
    assert tr <= 1.05e-8, tr
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr
    assert abs(r["iterations"] - ro["iterations"]) <= max(5, 0.03 * ro["iterations"]), (r, ro)
    A.close()


def test_iteration_limit_counts_exactly():
    p = W.edge_diffusion(40, seed=3)
    A, O = single(p)
    for maxit in (1, 2, 7):
        x, r = A.solve(t(p.b), rtol=1e-14, maxit=maxit, method=B.KSP_PIPECG)
        xo, ro = oracle.pipecg(O, p.b, rtol=1e-14, maxit=maxit)
        assert r["status"] == ro["status"] == B.ERR_MAXIT
        assert r["iterations"] == ro["iterations"] == maxit
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
    A.close()


def test_batched_and_ensemble():
    bt = W.batch(12, seed=41, size_range=(100, 6000))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    x, rs = A.solve_batched(t(bt.b), rtol=1e-9, method=B.KSP_PIPECG)
    xo, ros = oracle.krylov_batched(O, bt.row_off, bt.b, oracle.PIPECG, rtol=1e-9)
    resid = bt.b - oracle.spmv(O, x.cpu().numpy())
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.OK, (s, rs[s], ros[s])
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"]), (s, rs[s], ros[s])
        sl = slice(ro[s], ro[s + 1])
        tr = np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl])
        assert resid_ok(tr, ros[s], 1e-9), (s, tr)
    # the stacked ensemble: one set of scalars, one global norm
    xe, re = A.solve(t(bt.b), rtol=1e-9, method=B.KSP_PIPECG)
    xeo, reo = oracle.pipecg(O, bt.b, rtol=1e-9)
    assert re["status"] == reo["status"] == B.OK
    assert iters_close(re["iterations"], reo["iterations"])
    assert resid_ok(true_rel(O, bt.b, xe.cpu().numpy()), reo, 1e-9)
    A.close()


def test_host_loop_matches_graph_and_reruns_are_identical():
    p = W.edge_diffusion(120, seed=6)
    A, O = single(p)
    x1, r1 = A.solve(t(p.b), rtol=1e-9, method=B.KSP_PIPECG)
    x2, r2 = A.solve(t(p.b), rtol=1e-9, method=B.KSP_PIPECG, host_loop=True)
    x3, r3 = A.solve(t(p.b), rtol=1e-9, method=B.KSP_PIPECG)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert r1["iterations"] == r2["iterations"] == r3["iterations"]
    A.close()


def test_degenerate_and_error_paths():
    p = W.edge_diffusion(20, seed=2)
    A, O = single(p)
    x, r = A.solve(torch.zeros(p.nrows, dtype=torch.float64, device=DEV),
                   method=B.KSP_PIPECG)
    assert r["status"] == B.OK and r["iterations"] == 0 and not torch.any(x)
    x0 = np.random.default_rng(3).standard_normal(p.nrows)
    x, r = A.solve(t(p.b), x=t(x0.copy()), rtol=1e-10, nonzero_guess=True,
                   method=B.KSP_PIPECG)
    xo, ro = oracle.pipecg(O, p.b, rtol=1e-10, x0=x0)
    assert r["status"] == ro["status"] == B.OK
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    assert iters_close(r["iterations"], ro["iterations"])
    x, r = A.solve(t(p.b), rtol=1e-15, maxit=100000, timeout_ns=1, method=B.KSP_PIPECG)
    assert r["status"] == B.ERR_TIMEOUT
    with pytest.raises(B.GbsError):
        A.solve(t(p.b), method=B.KSP_PIPECG, precision=B.FP32_REFINED)
    A.close()
    v = p.v.copy()
    v[(p.i == 7) & (p.j == 7)] = 0.0                  # zero diagonal
    A, O = single(W.Problem("zd", p.nrows, p.ncols, p.i, p.j, v, p.b))
    x, r = A.solve(t(p.b), method=B.KSP_PIPECG)
    assert r["status"] == B.ERR_NOT_SPD
    A.close()


def test_one_kernel_per_iteration():
    p = W.edge_diffusion(64, seed=4)
    A, O = single(p)
    A.solve(t(p.b), rtol=1e-9, method=B.KSP_PIPECG)        # builds the graph
    n0 = B.launch_count()
    x, r = A.solve(t(p.b), rtol=1e-9, method=B.KSP_PIPECG)
    n = B.launch_count() - n0
    # call arguments + two start-up kernels + closing residual + one kernel
    # per trip: one trip per iteration, then the trip that sees no active
    # system, rounded up to the graph body's 8 trips
    trips = n - 4
    assert trips % 8 == 0 and r["iterations"] + 1 <= trips <= r["iterations"] + 8, (n, r)
    A.close()
