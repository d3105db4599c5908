"""GPU parity of the single-reduction Jacobi-PCG run as ONE kernel per
iteration (GBS_CG_SINGLE_KERNEL: each CTA updates its rows, waits on flags
for the CTAs whose rows its row products read, then runs them; one
reduction) against the oracle's orc_pcg_sr and against the two-kernel form.

Bars as for the two-kernel form: statuses equal to the oracle's; iteration
counts within max(2, 1%) of the oracle's single-reduction count and of the
textbook PCG's; equal under an iteration limit with iterates equal to 1e-10;
the relative true residual recomputed by the oracle from the GPU's x at most
max(1.05 rtol, 2 x the oracle's own).  Also: the engine really runs one
kernel per trip; a plan whose grid cannot be resident at once falls back to
two kernels; CTAs holding several blocks, a wait window covering the whole
grid (a matrix with far columns) and the host-stepped loop (bit-identical to
the graph)."""
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


def single(p, form=B.CG_SINGLE_KERNEL):
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    A.set_values(t(p.v))
    A.set_cg_form(form)
    A.set_solver(B.SOLVER_PHASES)  # small systems would otherwise take the per-CTA engine
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    return A, O


def with_random_rhs(p, seed):
    p.b = np.random.default_rng(seed).standard_normal(p.nrows)
    return p


def far_columns(n, seed):
    """An SPD matrix whose rows also couple to rows about n / 2 away: a 1-D
    Laplacian plus, for each i < n / 2, the symmetric pair (i, i + n / 2)
    with weight -0.5 (diagonal raised to keep it diagonally dominant)."""
    h = n // 2
    I, J, V = [], [], []
    for i in range(n):
        I.append(i); J.append(i); V.append(3.5)
        if i > 0:
            I.append(i); J.append(i - 1); V.append(-1.0)
        if i + 1 < n:
            I.append(i); J.append(i + 1); V.append(-1.0)
        k = i + h if i < h else i - h
        if k < n and k != i:
            I.append(i); J.append(k); V.append(-0.5)
    b = np.random.default_rng(seed).standard_normal(n)
    return W.Problem("far", n, n, np.array(I, np.int32), np.array(J, np.int32),
                     np.array(V, np.float64), b)


def launches_per_solve(A, b, **kw):
    A.solve(b, **kw)                                       # builds the graph
    n0 = B.launch_count()
    x, r = A.solve(b, **kw)
    return B.launch_count() - n0, x, r


@pytest.mark.parametrize("name,make,rtol", [
    ("poisson2d_64", lambda: with_random_rhs(W.poisson2d(64), 1), 1e-8),
    ("q1hex_12", lambda: W.q1_hex(12, seed=W.SEED_C2), 1e-8),
    ("q1hex_30", lambda: W.q1_hex(30, seed=W.SEED_C2), 1e-8),
    ("poisson3d_24", lambda: W.poisson3d(24, seed=W.SEED_C3), 1e-10),
    ("edge_32", lambda: W.edge_diffusion(32, seed=W.SEED_C4_SMALL), 1e-8),
    ("edge_300", lambda: W.edge_diffusion(300, seed=9), 1e-8),
    ("far_20000", lambda: far_columns(20000, 5), 1e-9),
])
def test_single_kernel_parity(name, make, rtol):
    p = make()
    A, O = single(p)
    for method in (B.KSP_CGSR, B.KSP_CG):
        x, r = A.solve(t(p.b), rtol=rtol, method=method)
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


def test_one_kernel_per_trip_and_the_two_kernel_fallback():
    p = W.edge_diffusion(200, seed=11)               # 40,000 rows
    A, O = single(p)
    b = t(p.b)
    n, x1, r1 = launches_per_solve(A, b, rtol=1e-9, method=B.KSP_CGSR)
    # call arguments + setup + first product + closing residual + one kernel
    # per trip: one trip per iteration, rounded up to the graph body's 8
    trips = n - 4
    assert trips % 8 == 0 and r1["iterations"] <= trips <= r1["iterations"] + 8, (n, r1)
    # 1,250 blocks on 8 CTAs per SM: more CTAs than can be resident with this
    # kernel at once, so the two-kernel form runs
    A.set_plan(spmv_rows=32, ctas_per_sm=8)
    n, x2, r2 = launches_per_solve(A, b, rtol=1e-9, method=B.KSP_CGSR)
    assert (n - 3) % 2 == 0 and ((n - 3) // 2) % 8 == 0, (n, r2)
    assert iters_close(r1["iterations"], r2["iterations"])
    assert torch.linalg.norm(x1 - x2) <= 1e-7 * torch.linalg.norm(x1)
    A.close()


def test_several_blocks_per_cta_and_whole_grid_windows():
    """Blocks of 64 rows on one CTA per SM (each CTA walks about ten blocks),
    on a stencil matrix (a narrow window) and on the far-column matrix
    (every CTA waits for the whole grid)."""
    for p in (W.edge_diffusion(120, seed=8), far_columns(30000, 6)):
        A, O = single(p)
        A.set_plan(spmv_rows=64, update_rows=512, ctas_per_sm=1)
        x, r = A.solve(t(p.b), rtol=1e-9, method=B.KSP_CGSR)
        xo, ro = oracle.pcg_sr(O, p.b, rtol=1e-9)
        assert r["status"] == ro["status"] == B.OK
        assert iters_close(r["iterations"], ro["iterations"]), (r, ro)
        assert resid_ok(true_rel(O, p.b, x.cpu().numpy()), ro, 1e-9)
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


def test_host_loop_matches_graph_and_the_two_kernel_form():
    p = W.edge_diffusion(150, seed=6)
    A, O = single(p)
    b = t(p.b)
    x1, r1 = A.solve(b, rtol=1e-9, method=B.KSP_CGSR)
    x2, r2 = A.solve(b, rtol=1e-9, method=B.KSP_CGSR, host_loop=True)
    x3, r3 = A.solve(b, rtol=1e-9, method=B.KSP_CGSR)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert r1["iterations"] == r2["iterations"] == r3["iterations"]
    A.set_cg_form(B.CG_SINGLE_REDUCTION)
    x4, r4 = A.solve(b, rtol=1e-9, method=B.KSP_CGSR)
    assert iters_close(r1["iterations"], r4["iterations"])
    assert torch.linalg.norm(x1 - x4) <= 1e-7 * torch.linalg.norm(x4)
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
    A.close()
    v = p.v.copy()
    v[(p.i == 7) & (p.j == 7)] = 0.0                  # zero diagonal
    A, O = single(W.Problem("zd", p.nrows, p.ncols, p.i, p.j, v, p.b))
    x, r = A.solve(t(p.b), method=B.KSP_CGSR)
    assert r["status"] == B.ERR_NOT_SPD
    A.close()


def test_batched_handle_solved_per_system_takes_two_kernels():
    """Per-system (batched) solves keep the two-kernel form; the ensemble
    solve of the same batched handle takes the single kernel."""
    bt = W.batch(8, seed=43, size_range=(200, 5000))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    A.set_cg_form(B.CG_SINGLE_KERNEL)
    A.set_solver(B.SOLVER_PHASES)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-9, method=B.KSP_CGSR)
    xo, ros = oracle.krylov_batched(O, bt.row_off, bt.b, oracle.PCG_SR, rtol=1e-9)
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.OK
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"]), (s, rs[s], ros[s])
    xe, re = A.solve(t(bt.b), rtol=1e-9, method=B.KSP_CGSR)
    xeo, reo = oracle.pcg_sr(O, bt.b, rtol=1e-9)
    assert re["status"] == reo["status"] == B.OK
    assert iters_close(re["iterations"], reo["iterations"])
    assert resid_ok(true_rel(O, bt.b, xe.cpu().numpy()), reo, 1e-9)
    A.close()
