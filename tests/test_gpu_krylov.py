"""GPU parity of the nonsymmetric solvers (Sec. 7 batched TFQMR and BiCG with
diagonal preconditioning) against the FP64 oracle, through ksp_solve and
ksp_solve_batched.

Bars: statuses equal to the oracle's; iteration counts equal when the
iteration limit ends the solve (with iterates equal to 1e-10 after up to 8
iterations); for converged solves, within max(3, 5%) of the oracle's count
for TFQMR, whose quasi-residual bound decreases smoothly, and within
max(5, 25%) for BiCG, whose residual on a nonsymmetric system jumps up and
down by factors of several from one iteration to the next, so that the iteration
where it first crosses the threshold depends on rounding: on one system of
the 24-system batch below, the same BiCG in numpy stops after 120, 122,
127 or 128 iterations depending only on how its dot products are summed,
the oracle after 135;
the relative true residual recomputed by the oracle from the GPU's x at most
2 max(rtol, the oracle's own true residual) (TFQMR stops on its
quasi-residual bound and BiCG on its recursive residual; both drift from
b - A x by the rounding of the updates, which scales with ||r0||); the GPU's
closing true residual within 1e-3 of the oracle's recomputation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_08646_gb300 import binding as B
from paper_2406_08646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
METHODS = [B.KSP_BICG, B.KSP_TFQMR]
SOLVERS = [B.SOLVER_CTA, B.SOLVER_PHASES]
ORACLE = {B.KSP_BICG: oracle.bicg, B.KSP_TFQMR: oracle.tfqmr}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def iters_close(a, b, method=B.KSP_TFQMR):
    if method == B.KSP_BICG:
        return abs(a - b) <= max(5, int(np.ceil(0.25 * max(a, b))))
    return abs(a - b) <= max(3, int(np.ceil(0.05 * max(a, b))))


def resid_ok(tr, ro, rtol):
    return tr <= 2 * max(rtol, ro["true_rel_residual"])


def true_rel(O, b, x):
    bn = np.linalg.norm(b)
    return np.linalg.norm(b - oracle.spmv(O, x)) / bn if bn > 0 else np.linalg.norm(x)


def single(p):
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    A.set_values(t(p.v))
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    return A, O


def batch_of(problems):
    """A Batch from single problems (local COO indices concatenated)."""
    nrows = np.array([p.nrows for p in problems], np.int64)
    ncoo = np.array([p.i.shape[0] for p in problems], np.int64)
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return W.Batch("custom", nrows, ncoo, cat([p.i for p in problems], np.int32),
                   cat([p.j for p in problems], np.int32), cat([p.v for p in problems], np.float64),
                   cat([p.b for p in problems], np.float64))


def assemble_batch(bt):
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    return A, O


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("m,bx,by,rtol", [(40, 30.0, -10.0, 1e-10), (23, -5.0, 60.0, 1e-8),
                                          (64, 100.0, 100.0, 1e-8)])
def test_single_system_parity(method, m, bx, by, rtol, solver):
    p = W.convdiff2d(m, bx, by, seed=100 + m)
    A, O = single(p)
    A.set_solver(solver)
    x, r = A.solve(t(p.b), rtol=rtol, method=method)
    xo, ro = ORACLE[method](O, p.b, rtol=rtol)
    assert r["status"] == ro["status"] == B.OK, (r, ro)
    assert r["solver"] == solver
    assert iters_close(r["iterations"], ro["iterations"], method), (r, ro)
    tr = true_rel(O, p.b, x.cpu().numpy())
    assert resid_ok(tr, ro, rtol), (tr, ro)
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr + 1e-15
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_batched_parity(method, solver):
    bt = W.convdiff_batch(24, seed=61, size_range=(50, 3000), peclet=(1.0, 200.0))
    A, O = assemble_batch(bt)
    A.set_solver(solver)
    rtol = 1e-9
    x, rs = A.solve_batched(t(bt.b), rtol=rtol, method=method)
    xo, ros = oracle.krylov_batched(O, bt.row_off, bt.b, method, rtol=rtol)
    xg = x.cpu().numpy()
    resid = bt.b - oracle.spmv(O, xg)      # block diagonal: block s depends on x_s only
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.OK, (s, rs[s], ros[s])
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"], method), (s, rs[s], ros[s])
        sl = slice(ro[s], ro[s + 1])
        tr = np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl])
        assert resid_ok(tr, ros[s], rtol), (s, tr, ros[s])
        assert abs(rs[s]["true_rel_residual"] - tr) <= 1e-3 * tr + 1e-15
    # a second call gives the identical answer (fixed reduction order)
    x2, _ = A.solve_batched(t(bt.b), rtol=rtol, method=method)
    assert torch.equal(x, x2)
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_ragged_and_degenerate_batch(method, solver):
    """Sizes 1, 0, 4, 36 (ragged slices), 121 and 1089 rows; the empty system and
    a zero right-hand side end at once with OK and x = 0."""
    probs = [W.convdiff2d(mm, 20.0, 5.0, seed=200 + mm) for mm in (1, 2, 6, 11, 33)]
    empty = W.Problem("empty", 0, 0, np.zeros(0, np.int32), np.zeros(0, np.int32),
                      np.zeros(0), np.zeros(0))
    probs.insert(1, empty)
    probs[3].b[:] = 0.0                        # the 6 x 6 system gets b = 0
    bt = batch_of(probs)
    A, O = assemble_batch(bt)
    A.set_solver(solver)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-10, method=method)
    xo, ros = oracle.krylov_batched(O, bt.row_off, bt.b, method, rtol=1e-10)
    xg = x.cpu().numpy()
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.OK, (s, rs[s], ros[s])
        sl = slice(ro[s], ro[s + 1])
        if not np.any(bt.b[sl]):
            assert not np.any(xg[sl]) and rs[s]["iterations"] == 0
            continue
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"], method), (s, rs[s], ros[s])
        tr = np.linalg.norm(bt.b[sl] - oracle.spmv(O, xg)[sl]) / np.linalg.norm(bt.b[sl])
        assert resid_ok(tr, ros[s], 1e-10), (s, tr, ros[s])
    A.close()


def test_bicg_on_spd_matches_pcg():
    """On a symmetric matrix BiCG performs PCG's operations: same iteration
    count as the GPU's PCG and the oracle's, same solution to rounding."""
    p = W.poisson2d(48)
    A, O = single(p)
    xb, rb = A.solve(t(p.b), rtol=1e-10, method=B.KSP_BICG)
    xc, rc = A.solve(t(p.b), rtol=1e-10)
    xo, ro = oracle.pcg(O, p.b, rtol=1e-10)
    assert rb["status"] == rc["status"] == B.OK
    assert abs(rb["iterations"] - ro["iterations"]) <= 1
    assert abs(rb["iterations"] - rc["iterations"]) <= 1
    xbn = xb.cpu().numpy()
    assert np.linalg.norm(xbn - xo) <= 1e-8 * np.linalg.norm(xo)
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_iteration_limit_counts_exactly(method, solver):
    p = W.convdiff2d(30, 40.0, 10.0, seed=7)
    A, O = single(p)
    A.set_solver(solver)
    for maxit in (1, 2, 5, 8):
        x, r = A.solve(t(p.b), rtol=1e-14, maxit=maxit, method=method)
        xo, ro = ORACLE[method](O, p.b, rtol=1e-14, maxit=maxit)
        assert r["status"] == ro["status"] == B.ERR_MAXIT, (maxit, r, ro)
        assert r["iterations"] == ro["iterations"], (maxit, r, ro)
        # few steps: the iterates agree to rounding
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * max(np.linalg.norm(xo), 1e-300)
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_nonzero_guess(method, solver):
    p = W.convdiff2d(25, -15.0, 25.0, seed=3)
    A, O = single(p)
    A.set_solver(solver)
    x0 = np.random.default_rng(1).standard_normal(p.nrows)
    xg = t(x0.copy())
    x, r = A.solve(t(p.b), x=xg, rtol=1e-10, nonzero_guess=True, method=method)
    xo, ro = ORACLE[method](O, p.b, rtol=1e-10, x0=x0)
    assert r["status"] == ro["status"] == B.OK
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    assert iters_close(r["iterations"], ro["iterations"], method), (r, ro)
    assert resid_ok(true_rel(O, p.b, x.cpu().numpy()), ro, 1e-10)
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_new_values_refresh_the_transpose(method, solver):
    """mat_set_values_coo after a solve: the next solve (BiCG: its A^T copy)
    sees the new values."""
    p = W.convdiff2d(20, 10.0, 0.0, seed=5)
    q = W.convdiff2d(20, -30.0, 50.0, seed=5)     # same pattern, other values
    A, O = single(p)
    A.set_solver(solver)
    A.solve(t(p.b), rtol=1e-10, method=method)
    A.set_values(t(q.v))
    Oq = oracle.coo_symbolic(q.nrows, q.ncols, q.i, q.j)
    oracle.coo_numeric(Oq, q.v)
    x, r = A.solve(t(q.b), rtol=1e-10, method=method)
    xo, ro = ORACLE[method](Oq, q.b, rtol=1e-10)
    assert r["status"] == B.OK and iters_close(r["iterations"], ro["iterations"], method), (r, ro)
    assert resid_ok(true_rel(Oq, q.b, x.cpu().numpy()), ro, 1e-10)
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_missing_diagonal_is_reported(method, solver):
    p = W.convdiff2d(8, 5.0, 5.0, seed=2)
    v = p.v.copy()
    v[(p.i == 3) & (p.j == 3)] = -1.0            # a negative diagonal entry
    A, O = single(W.Problem("neg", p.nrows, p.ncols, p.i, p.j, v, p.b))
    A.set_solver(solver)
    x, r = A.solve(t(p.b), method=method)
    xo, ro = ORACLE[method](O, p.b)
    assert r["status"] == ro["status"] == B.ERR_NOT_SPD
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("method", METHODS)
def test_time_limit(method, solver):
    p = W.convdiff2d(90, 200.0, 150.0, seed=4)
    A, O = single(p)
    A.set_solver(solver)
    x, r = A.solve(t(p.b), rtol=1e-15, maxit=100000, timeout_ns=1, method=method)
    assert r["status"] == B.ERR_TIMEOUT and r["iterations"] >= 1
    # the handle stays usable
    x, r = A.solve(t(p.b), rtol=1e-8, method=method)
    assert r["status"] == B.OK
    A.close()


def test_option_checks():
    p = W.convdiff2d(6, 1.0, 1.0, seed=1)
    A, O = single(p)
    b = t(p.b)
    x = torch.empty_like(b)
    with pytest.raises(B.GbsError):       # the CG entry point takes CG only
        B.ksp_solve_cg(A.h, b, x, B.make_opts(method=B.KSP_TFQMR))
    with pytest.raises(B.GbsError):       # BiCG / TFQMR are FP64 only
        A.solve(b, method=B.KSP_BICG, precision=B.FP32_REFINED)
    with pytest.raises(B.GbsError):
        A.solve(b, method=7)
    A.close()


@pytest.mark.parametrize("method", METHODS)
def test_phases_host_loop_matches_graph(method):
    """The host-stepped loop runs the same kernels: identical x and counts."""
    p = W.convdiff2d(70, 50.0, -20.0, seed=8)
    A, O = single(p)
    A.set_solver(B.SOLVER_PHASES)
    x1, r1 = A.solve(t(p.b), rtol=1e-9, method=method)
    x2, r2 = A.solve(t(p.b), rtol=1e-9, method=method, host_loop=True)
    assert torch.equal(x1, x2) and r1["iterations"] == r2["iterations"]
    assert r1["status"] == B.OK
    A.close()


@pytest.mark.parametrize("method", METHODS)
def test_ensemble_is_the_stacked_system(method):
    """ksp_solve on a batched handle solves the stacked block-diagonal system
    with one global norm and one set of scalars (the Sec. 7 ensemble): the
    oracle's solver on the stacked CSR is its reference."""
    bt = W.convdiff_batch(12, seed=62, size_range=(200, 2000), peclet=(1.0, 50.0))
    A, O = assemble_batch(bt)
    A.set_solver(B.SOLVER_PHASES)
    x, r = A.solve(t(bt.b), rtol=1e-9, method=method)
    xo, ro = ORACLE[method](O, bt.b, rtol=1e-9)
    assert r["status"] == ro["status"] == B.OK
    assert iters_close(r["iterations"], ro["iterations"], method), (r, ro)
    assert resid_ok(true_rel(O, bt.b, x.cpu().numpy()), ro, 1e-9)
    A.close()


def test_launch_counts_of_the_phase_loops():
    """Per trip: BiCG 3 kernels, TFQMR 4; plus setup, closing kernels and the
    call-argument write (TFQMR closes with the pending x update as well)."""
    p = W.convdiff2d(50, 20.0, 20.0, seed=9)
    A, O = single(p)
    A.set_solver(B.SOLVER_PHASES)
    for method, per_trip, post in ((B.KSP_BICG, 3, 1), (B.KSP_TFQMR, 4, 2)):
        A.solve(t(p.b), rtol=1e-9, method=method)         # builds the graph
        n0 = B.launch_count()
        x, r = A.solve(t(p.b), rtol=1e-9, method=method)
        n = B.launch_count() - n0
        trips = r["iterations"] if method == B.KSP_BICG else (r["iterations"] + 1) // 2
        assert n >= 1 + 1 + post + per_trip * trips, (method, n, r)
        # the graph body holds 8 trips: up to 7 more after the last one needed
        assert n <= 1 + 1 + post + per_trip * (trips + 9), (method, n, r)
        assert (n - 2 - post) % (8 * per_trip) == 0, (method, n, r)
    A.close()


@pytest.mark.parametrize("method", METHODS)
def test_large_batch_two_ctas_per_sm(method):
    """A batch of at least two systems per SM runs two 1024-thread CTAs per
    SM (the 32-register build of the kernel): every system against the
    oracle."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    bt = W.convdiff_batch(2 * nsm + 9, seed=63, size_range=(16, 600), peclet=(1.0, 80.0))
    A, O = assemble_batch(bt)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-9, method=method)
    xo, ros = oracle.krylov_batched(O, bt.row_off, bt.b, method, rtol=1e-9)
    resid = bt.b - oracle.spmv(O, x.cpu().numpy())
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["solver"] == B.SOLVER_CTA
        assert rs[s]["status"] == ros[s]["status"] == B.OK, (s, rs[s], ros[s])
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"], method), (s, rs[s], ros[s])
        sl = slice(ro[s], ro[s + 1])
        tr = np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl])
        assert resid_ok(tr, ros[s], 1e-9), (s, tr, ros[s])
    A.close()
