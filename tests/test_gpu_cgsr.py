"""GPU parity of the single-reduction Jacobi-PCG (Chronopoulos-Gear form: the
product fused with the iteration's one reduction, then one element-wise
update kernel with no reduction) against the oracle's orc_pcg_sr, through
ksp_solve / ksp_solve_batched / ksp_solve_cg with method GBS_KSP_CGSR.

Bars: statuses equal to the oracle's; iteration counts within max(2, 1%) of
the oracle's single-reduction count and of the textbook PCG's (same
iterates in exact arithmetic; the dot products' summation order differs),
equal under an iteration limit with iterates equal to 1e-10; the relative
true residual recomputed by the oracle from the GPU's x at most
max(1.05 rtol, 2 x the oracle's own); the GPU's closing residual within 1e-3
of the recomputation; rnorm0 to 1e-12."""
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
    return tr <= max(1.05 * rtol, 2 * ro["true_rel_residual"])


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
    ("q1hex_30", lambda: W.q1_hex(30, seed=W.SEED_C2), 1e-8),
    ("poisson3d_24", lambda: W.poisson3d(24, seed=W.SEED_C3), 1e-10),
    ("edge_32", lambda: W.edge_diffusion(32, seed=W.SEED_C4_SMALL), 1e-8),
    ("edge_300", lambda: W.edge_diffusion(300, seed=9), 1e-8),
])
def test_cgsr_parity(name, make, rtol):
    p = make()
    A, O = single(p)
    x, r = A.solve(t(p.b), rtol=rtol, method=B.KSP_CGSR)
    xo, ro = oracle.pcg_sr(O, p.b, rtol=rtol)
    _, rh = oracle.pcg(O, p.b, rtol=rtol)
    assert r["status"] == ro["status"] == B.OK, (r, ro)
    assert r["solver"] == B.SOLVER_PHASES
    assert iters_close(r["iterations"], ro["iterations"]), (r, ro)
    assert iters_close(r["iterations"], rh["iterations"]), (r, rh)
    tr = true_rel(O, p.b, x.cpu().numpy())
    assert resid_ok(tr, ro, rtol), (tr, ro)
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr + 1e-15
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    A.close()


def test_cg_entry_point_takes_the_single_reduction_form():
    """ksp_solve_cg and ksp_adjoint accept method GBS_KSP_CGSR (and refuse
    the nonsymmetric methods)."""
    p = W.edge_diffusion(50, seed=12)
    A, O = single(p)
    b = t(p.b)
    x = torch.empty_like(b)
    r = B.ksp_solve_cg(A.h, b, x, B.make_opts(rtol=1e-9, method=B.KSP_CGSR))[0]
    xo, ro = oracle.pcg_sr(O, p.b, rtol=1e-9)
    assert r["status"] == B.OK and iters_close(r["iterations"], ro["iterations"])
    g = t(np.random.default_rng(4).standard_normal(p.nrows))
    lam, _, dldv, ra = A.adjoint(x, g, rtol=1e-10, method=B.KSP_CGSR)
    assert ra[0]["status"] == B.OK
    lo, _, dvo, _ = oracle.adjoint(O, x.cpu().numpy(), g.cpu().numpy(), rtol=1e-12)
    assert np.linalg.norm(dldv.cpu().numpy() - dvo) <= 1e-7 * np.linalg.norm(dvo)
    with pytest.raises(B.GbsError):
        B.ksp_solve_cg(A.h, b, x, B.make_opts(method=B.KSP_TFQMR))
    A.close()


def test_iteration_limit_counts_and_iterates_exactly():
    p = W.edge_diffusion(40, seed=3)
    A, O = single(p)
    for maxit in (1, 2, 7, 30):
        x, r = A.solve(t(p.b), rtol=1e-14, maxit=maxit, method=B.KSP_CGSR)
        xo, ro = oracle.pcg_sr(O, p.b, rtol=1e-14, maxit=maxit)
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
    x, rs = A.solve_batched(t(bt.b), rtol=1e-9, method=B.KSP_CGSR)
    xo, ros = oracle.krylov_batched(O, bt.row_off, bt.b, oracle.PCG_SR, rtol=1e-9)
    resid = bt.b - oracle.spmv(O, x.cpu().numpy())
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.OK, (s, rs[s], ros[s])
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"]), (s, rs[s], ros[s])
        sl = slice(ro[s], ro[s + 1])
        tr = np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl])
        assert resid_ok(tr, ros[s], 1e-9), (s, tr)
    xe, re = A.solve(t(bt.b), rtol=1e-9, method=B.KSP_CGSR)
    xeo, reo = oracle.pcg_sr(O, bt.b, rtol=1e-9)
    assert re["status"] == reo["status"] == B.OK
    assert iters_close(re["iterations"], reo["iterations"])
    assert resid_ok(true_rel(O, bt.b, xe.cpu().numpy()), reo, 1e-9)
    A.close()


def test_degenerate_batch():
    """2 x 2 SPD block, empty system, 1 x 1 system, b = 0 system: 2, 0, 1, 0
    iterations, x = b / a, x = 0, as the oracle."""
    blocks = [np.array([[4.0, 1.0], [1.0, 3.0]]), np.zeros((0, 0)), np.array([[2.5]]),
              np.array([[2.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 2.0]])]
    I, J, V, nrows, ncoo = [], [], [], [], []
    for Bk in blocks:
        ii, jj = np.nonzero(Bk) if Bk.size else (np.zeros(0, int), np.zeros(0, int))
        I.append(ii.astype(np.int32)); J.append(jj.astype(np.int32)); V.append(Bk[ii, jj])
        nrows.append(Bk.shape[0]); ncoo.append(len(ii))
    A = B.Mat.from_coo_batched(np.array(nrows, np.int64), np.array(ncoo, np.int64),
                               t(np.concatenate(I)), t(np.concatenate(J)))
    A.set_values(t(np.concatenate(V)))
    b = np.array([1.0, 2.0, 5.0, 0.0, 0.0, 0.0])
    x, rs = A.solve_batched(t(b), rtol=1e-12, method=B.KSP_CGSR)
    assert [r["status"] for r in rs] == [B.OK] * 4
    assert [r["iterations"] for r in rs] == [2, 0, 1, 0]
    xh = x.cpu().numpy()
    assert not np.any(xh[3:])
    xs = np.linalg.solve(blocks[0], b[:2])
    assert np.linalg.norm(xh[:2] - xs) <= 1e-12 * np.linalg.norm(xs) * 10
    assert abs(xh[2] - 2.0) <= 4 * np.spacing(2.0)
    A.close()


def test_host_loop_matches_graph_and_reruns_are_identical():
    p = W.edge_diffusion(120, seed=6)
    A, O = single(p)
    x1, r1 = A.solve(t(p.b), rtol=1e-9, method=B.KSP_CGSR)
    x2, r2 = A.solve(t(p.b), rtol=1e-9, method=B.KSP_CGSR, host_loop=True)
    x3, r3 = A.solve(t(p.b), rtol=1e-9, method=B.KSP_CGSR)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert r1["iterations"] == r2["iterations"] == r3["iterations"]
    A.close()


def test_error_paths():
    p = W.edge_diffusion(20, seed=2)
    A, O = single(p)
    x, r = A.solve(torch.zeros(p.nrows, dtype=torch.float64, device=DEV), method=B.KSP_CGSR)
    assert r["status"] == B.OK and r["iterations"] == 0 and not torch.any(x)
    x0 = np.random.default_rng(3).standard_normal(p.nrows)
    x, r = A.solve(t(p.b), x=t(x0.copy()), rtol=1e-10, nonzero_guess=True, method=B.KSP_CGSR)
    xo, ro = oracle.pcg_sr(O, p.b, rtol=1e-10, x0=x0)
    assert r["status"] == ro["status"] == B.OK
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    assert iters_close(r["iterations"], ro["iterations"])
    bn = p.b.copy()
    bn[5] = np.nan
    x, r = A.solve(t(bn), method=B.KSP_CGSR)
    assert r["status"] == B.ERR_NAN
    x, r = A.solve(t(p.b), rtol=1e-14, maxit=0, method=B.KSP_CGSR)
    assert r["status"] == B.ERR_MAXIT and r["iterations"] == 0
    x, r = A.solve(t(p.b), rtol=1e-15, maxit=100000, timeout_ns=1, method=B.KSP_CGSR)
    assert r["status"] == B.ERR_TIMEOUT
    with pytest.raises(B.GbsError):
        A.solve(t(p.b), method=B.KSP_CGSR, precision=B.FP32_REFINED)
    A.close()
    v = p.v.copy()
    v[(p.i == 7) & (p.j == 7)] = 0.0                  # zero diagonal
    A, O = single(W.Problem("zd", p.nrows, p.ncols, p.i, p.j, v, p.b))
    x, r = A.solve(t(p.b), method=B.KSP_CGSR)
    assert r["status"] == B.ERR_NOT_SPD
    A.close()


def test_two_kernels_per_iteration():
    p = W.edge_diffusion(64, seed=4)
    A, O = single(p)
    A.solve(t(p.b), rtol=1e-9, method=B.KSP_CGSR)        # builds the graph
    n0 = B.launch_count()
    x, r = A.solve(t(p.b), rtol=1e-9, method=B.KSP_CGSR)
    n = B.launch_count() - n0
    # call arguments + setup + closing residual + two kernels per trip: one
    # trip per iteration plus the one whose tests stop it, rounded up to the
    # graph body's 8 trips
    trips = (n - 3) // 2
    assert (n - 3) % 2 == 0 and trips % 8 == 0, (n, r)
    assert r["iterations"] + 1 <= trips <= r["iterations"] + 8, (n, r)
    A.close()
