"""GPU parity of the cluster solver (FP64 Jacobi-PCG with one thread-block
cluster per system, reductions through distributed shared memory) against
the FP64 oracle, through the C-ABI.

Bars as for the other CG engines: statuses equal to the oracle's, iteration
counts within max(2, 1%), relative true residual recomputed by the oracle
from the GPU's x at most 1.05 rtol, the GPU's own closing residual within
1e-3 of the recomputation, bit-identical reruns."""
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


def true_rel(O, b, x):
    return np.linalg.norm(b - oracle.spmv(O, x)) / np.linalg.norm(b)


def single(p):
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    A.set_values(t(p.v))
    A.set_solver(B.SOLVER_CLUSTER)
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    return A, O


def random_rhs(p, seed):
    p.b = np.random.default_rng(seed).standard_normal(p.nrows)
    return p


@pytest.mark.parametrize("name,make,rtol", [
    ("poisson2d_20", lambda: random_rhs(W.poisson2d(20), 2), 1e-8),
    ("poisson2d_128", lambda: random_rhs(W.poisson2d(128), 3), 1e-8),
    ("q1hex_16", lambda: W.q1_hex(16, seed=W.SEED_C2), 1e-8),
    ("poisson3d_40", lambda: W.poisson3d(40, seed=W.SEED_C3), 1e-10),
    ("edge_300", lambda: W.edge_diffusion(300, seed=9), 1e-8),
])
def test_cluster_parity(name, make, rtol):
    p = make()
    A, O = single(p)
    x, r = A.solve(t(p.b), rtol=rtol)
    xo, ro = oracle.pcg(O, p.b, rtol=rtol)
    assert r["status"] == ro["status"] == B.OK, (r, ro)
    assert r["solver"] == B.SOLVER_CLUSTER
    assert iters_close(r["iterations"], ro["iterations"]), (r, ro)
    tr = true_rel(O, p.b, x.cpu().numpy())
    assert tr <= 1.05 * rtol, tr
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr + 1e-15
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    x2, r2 = A.solve(t(p.b), rtol=rtol)
    assert torch.equal(x, x2) and r2 == r
    A.close()


def test_cluster_batched():
    bt = W.batch(20, seed=44, size_range=(30, 20000))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    A.set_solver(B.SOLVER_CLUSTER)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-9)
    xo, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-9)
    resid = bt.b - oracle.spmv(O, x.cpu().numpy())
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.OK, (s, rs[s], ros[s])
        assert rs[s]["solver"] == B.SOLVER_CLUSTER
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"]), (s, rs[s], ros[s])
        sl = slice(ro[s], ro[s + 1])
        assert np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl]) <= 1.05e-9
    # the stacked ensemble on one cluster
    xe, re = A.solve(t(bt.b), rtol=1e-9)
    xeo, reo = oracle.pcg(O, bt.b, rtol=1e-9)
    assert re["status"] == B.OK and iters_close(re["iterations"], reo["iterations"])
    assert true_rel(O, bt.b, xe.cpu().numpy()) <= 1.05e-9
    A.close()


def test_cluster_degenerate_paths():
    p = W.edge_diffusion(40, seed=5)
    A, O = single(p)
    # b = 0: x = 0 exactly, no iteration
    x, r = A.solve(torch.zeros(p.nrows, dtype=torch.float64, device=DEV), x=t(np.ones(p.nrows)),
                   nonzero_guess=True)
    assert r["status"] == B.OK and r["iterations"] == 0 and not torch.any(x)
    # nonzero initial guess
    x0 = np.random.default_rng(4).standard_normal(p.nrows)
    x, r = A.solve(t(p.b), x=t(x0.copy()), rtol=1e-10, nonzero_guess=True)
    xo, ro = oracle.pcg(O, p.b, rtol=1e-10, x0=x0)
    assert r["status"] == B.OK and iters_close(r["iterations"], ro["iterations"])
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    # iteration limit: same count and iterates as the oracle
    for maxit in (1, 3, 10):
        x, r = A.solve(t(p.b), rtol=1e-14, maxit=maxit)
        xo, ro = oracle.pcg(O, p.b, rtol=1e-14, maxit=maxit)
        assert r["status"] == ro["status"] == B.ERR_MAXIT and r["iterations"] == maxit
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-11 * np.linalg.norm(xo)
    # the time limit stops every CTA of the cluster at the same iteration
    x, r = A.solve(t(p.b), rtol=1e-15, maxit=100000, timeout_ns=1)
    assert r["status"] == B.ERR_TIMEOUT and r["iterations"] == 1
    x, r = A.solve(t(p.b), rtol=1e-8)
    assert r["status"] == B.OK
    # a refined solve asked for the cluster solver runs on the phase kernels
    x, r = A.solve(t(p.b), rtol=1e-8, precision=B.FP32_REFINED)
    assert r["status"] == B.OK and r["solver"] == B.SOLVER_PHASES
    A.close()
    v = p.v.copy()
    v[(p.i == 3) & (p.j == 3)] = 0.0
    A, O = single(W.Problem("zd", p.nrows, p.ncols, p.i, p.j, v, p.b))
    x, r = A.solve(t(p.b))
    assert r["status"] == B.ERR_NOT_SPD
    A.close()

