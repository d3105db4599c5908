"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the
same seeded inputs.

Bars: CSR structure, perm and jmap bit-exact; COO values bit-exact (both sum
duplicates left to right in increasing COO index); SpMV within
1e-12 * sum_p |a_p| |x_col p| per row; solves to the stated relative residual,
recomputed by the oracle from the GPU's x, with iteration counts within
max(2, 1%) of the oracle's (FP64) or +-1 outer step (FP32-refined); gradients
within 1e-8 relative of the oracle's."""
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


def t(a, dtype=None):
    x = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        x = x.to(dtype)
    return x.to(DEV)


def assemble_both(nrows, ncols, i, j, v):
    A = B.Mat.from_coo(nrows, ncols, t(i), t(j))
    A.set_values(t(v))
    O = oracle.coo_symbolic(nrows, ncols, i, j)
    oracle.coo_numeric(O, v)
    return A, O


def abs_bound(O, x):
    Oa = oracle.CSR(O.nrows, O.ncols, O.row_ptr, O.col, O.perm, O.jmap, O.ncoo, np.abs(O.val))
    return oracle.spmv(Oa, np.abs(x))


def random_coo(rng, n, ncoo, ncols=None, dup=0.3, neg=0.1):
    ncols = n if ncols is None else ncols
    base = max(1, int(ncoo * (1 - dup)))
    i = rng.integers(0, n, base)
    j = rng.integers(0, ncols, base)
    pick = rng.integers(0, base, ncoo - base)
    i = np.concatenate([i, i[pick]])[:ncoo]
    j = np.concatenate([j, j[pick]])[:ncoo]
    sh = rng.permutation(len(i))
    i, j = i[sh], j[sh]
    drop = rng.random(len(i)) < neg
    i = np.where(drop & (rng.random(len(i)) < 0.5), -1, i)
    j = np.where(drop & (i >= 0), -2, j)
    v = rng.standard_normal(len(i)) * 10.0 ** rng.uniform(-3, 3, len(i))
    return i.astype(np.int32), j.astype(np.int32), v


# ------------------------------------------------------------------ assembly

@pytest.mark.parametrize("n,ncoo,ncols", [(1, 1, 1), (7, 50, 7), (64, 4096, 64),
                                          (1000, 70_000, 1000), (5000, 9000, 300),
                                          (40_000, 333_333, 40_000)])
def test_assembly_bitexact(n, ncoo, ncols):
    rng = np.random.default_rng(n + ncoo)
    i, j, v = random_coo(rng, n, ncoo, ncols)
    A, O = assemble_both(n, ncols, i, j, v)
    rp, col, val = (x.cpu().numpy() for x in A.csr())
    perm, jmap = (x.cpu().numpy() for x in A.coo_maps())
    assert np.array_equal(rp, O.row_ptr)
    assert np.array_equal(col, O.col)
    assert np.array_equal(perm, O.perm)
    assert np.array_equal(jmap, O.jmap)
    assert val.tobytes() == O.val.tobytes()
    # ADD then INSERT
    A.set_values(t(2.0 * v), mode=B.ADD)
    oracle.coo_numeric(O, 2.0 * v, mode=oracle.ADD)
    assert A.csr()[2].cpu().numpy().tobytes() == O.val.tobytes()
    A.set_values(t(v), mode=B.INSERT)
    oracle.coo_numeric(O, v, mode=oracle.INSERT)
    assert A.csr()[2].cpu().numpy().tobytes() == O.val.tobytes()
    A.close()


def test_assembly_edge_cases():
    # empty input, all entries ignored, empty rows, a lone -0.0
    for (n, i, j, v) in [(5, [], [], []), (5, [-1, 2, -3], [0, -1, -2], [1.0, 2.0, 3.0]),
                         (6, [5, 0], [5, 0], [1.0, 2.0]), (3, [1], [2], [-0.0])]:
        i = np.array(i, np.int32)
        j = np.array(j, np.int32)
        v = np.array(v, np.float64)
        A = B.Mat.from_coo(n, n, t(i) if len(i) else torch.empty(0, dtype=torch.int32, device=DEV),
                           t(j) if len(j) else torch.empty(0, dtype=torch.int32, device=DEV))
        A.set_values(t(v) if len(v) else torch.empty(0, dtype=torch.float64, device=DEV))
        O = oracle.coo_symbolic(n, n, i, j)
        oracle.coo_numeric(O, v)
        rp, col, val = (x.cpu().numpy() for x in A.csr())
        assert np.array_equal(rp, O.row_ptr) and np.array_equal(col, O.col)
        assert val.tobytes() == O.val.tobytes()
        A.close()


def test_assembly_out_of_range_is_reported():
    i = t(np.array([0, 4], np.int32))
    j = t(np.array([0, 0], np.int32))
    with pytest.raises(B.GbsError) as e:
        B.Mat.from_coo(4, 4, i, j)
    assert e.value.status == B.ERR_INDEX


def test_q1_small_assembly_and_stencil():
    p = W.q1_hex(12, seed=W.SEED_C2)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    rp, col, val = (x.cpu().numpy() for x in A.csr())
    assert np.array_equal(rp, O.row_ptr) and np.array_equal(col, O.col)
    assert val.tobytes() == O.val.tobytes()
    assert A.nnz == (3 * 13 - 2) ** 3


# ------------------------------------------------------------------ SpMV

@pytest.mark.parametrize("make", [lambda: W.poisson2d(64), lambda: W.q1_hex(12, seed=3),
                                  lambda: W.poisson3d(30, seed=4),
                                  lambda: W.edge_diffusion(77, seed=5)])
def test_spmv_parity(make):
    p = make()
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(p.ncols)
    y = A.mult(t(x)).cpu().numpy()
    yo = oracle.spmv(O, x)
    assert np.all(np.abs(y - yo) <= 1e-12 * abs_bound(O, x))
    A.close()


def test_spmv_all_plans_and_irregular_rows():
    rng = np.random.default_rng(11)
    n = 3001
    # rows of very different lengths, including one long row and empty rows
    i = np.concatenate([rng.integers(0, n, 60_000), np.full(20_000, 17)]).astype(np.int32)
    j = rng.integers(0, n, i.shape[0]).astype(np.int32)
    v = rng.standard_normal(i.shape[0])
    A, O = assemble_both(n, n, i, j, v)
    x = rng.standard_normal(n)
    yo = oracle.spmv(O, x)
    bound = abs_bound(O, x)
    # (SpMV rows, update rows, row-product kernel, CTAs per SM cap); the long
    # row makes the sliced copy mostly padding, which it must skip exactly
    for plan in [(256, 512, B.SPMV_SELL, 0), (256, 512, 1, 0), (256, 512, 2, 0),
                 (256, 512, 4, 0), (256, 512, 8, 0), (256, 512, 32, 0), (32, 32, 4, 1),
                 (96, 1024, 2, 4), (64, 64, B.SPMV_SELL, 2), (256, 512, B.SPMV_AUTO, 0)]:
        A.set_plan(*plan)
        y = A.mult(t(x)).cpu().numpy()
        assert np.all(np.abs(y - yo) <= 1e-12 * bound), plan
    A.close()


# ------------------------------------------------------------------ PCG

def true_rel(O, b, x):
    return np.linalg.norm(b - oracle.spmv(O, x)) / np.linalg.norm(b)


def iters_close(a, b):
    return abs(a - b) <= max(2, int(np.ceil(0.01 * max(a, b))))


SOLVERS = [B.SOLVER_PHASES, B.SOLVER_CTA]


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("name,make,rtol", [
    ("c1_poisson2d_64", lambda: W.poisson2d(64), 1e-8),
    ("c2_q1hex_12", lambda: W.q1_hex(12, seed=W.SEED_C2), 1e-8),
    ("c3_poisson3d_24", lambda: W.poisson3d(24, seed=W.SEED_C3), 1e-10),
    ("c4_edge_32", lambda: W.edge_diffusion(32, seed=W.SEED_C4_SMALL), 1e-8),
    ("edge_300", lambda: W.edge_diffusion(300, seed=9), 1e-8),
])
def test_pcg_fp64_parity(name, make, rtol, solver):
    p = make()
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(solver)
    x, r = A.solve(t(p.b), rtol=rtol)
    assert r["solver"] == solver
    xo, ro = oracle.pcg(O, p.b, rtol=rtol)
    xg = x.cpu().numpy()
    assert r["status"] == B.OK and ro["status"] == oracle.OK
    tr = true_rel(O, p.b, xg)
    assert tr <= rtol * 1.05, tr
    # the GPU recomputes ||b - A x|| with its own rounding (FMA rows): the two
    # agree to the rounding error bound of the residual evaluation
    kmax = int(np.diff(O.row_ptr).max()) + 1
    ev = 2 * kmax * np.finfo(float).eps * np.linalg.norm(np.abs(p.b) + abs_bound(O, xg))
    assert abs(r["true_rel_residual"] - tr) <= 1e-3 * tr + ev / np.linalg.norm(p.b)
    assert iters_close(r["iterations"], ro["iterations"]), (r["iterations"], ro["iterations"])
    assert abs(r["rnorm0"] - ro["rnorm0"]) <= 1e-12 * ro["rnorm0"]
    # both solutions solve the same system to rtol: they agree to ~cond * rtol
    assert np.linalg.norm(xg - xo) <= 1e4 * rtol * np.linalg.norm(xo) + 1e-300
    # deterministic: a second solve is bit-identical
    x2, r2 = A.solve(t(p.b), rtol=rtol)
    assert torch.equal(x, x2) and r2["iterations"] == r["iterations"]
    A.close()


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_REFINED])
def test_host_loop_matches_graph(precision):
    """The host-stepped loop runs the same kernels on the same grids as the
    graph: results are bit-identical, single and batched."""
    p = W.q1_hex(9, seed=23)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(B.SOLVER_PHASES)
    x1, r1 = A.solve(t(p.b), rtol=1e-10, precision=precision)
    x2, r2 = A.solve(t(p.b), rtol=1e-10, precision=precision, host_loop=True)
    assert r1["status"] == B.OK and torch.equal(x1, x2) and r1 == r2
    A.close()
    bt, A, O = make_batch(12, 45, 100, 2000)
    A.set_solver(B.SOLVER_PHASES)
    x1, r1 = A.solve_batched(t(bt.b), rtol=1e-9, precision=precision)
    x2, r2 = A.solve_batched(t(bt.b), rtol=1e-9, precision=precision, host_loop=True)
    assert all(q["status"] == B.OK for q in r1) and torch.equal(x1, x2) and r1 == r2
    A.close()


def test_pcg_c1_closed_form():
    p = W.poisson2d(64)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    x, r = A.solve(t(p.b), rtol=1e-8)
    h = p.extra["h"]
    lam11 = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    xc = 2 * np.pi ** 2 / lam11 * p.extra["u_exact"]
    assert r["status"] == B.OK and 1 <= r["iterations"] <= 2
    assert np.max(np.abs(x.cpu().numpy() - xc)) <= 1e-12
    A.close()


@pytest.mark.parametrize("plan", [(256, 512, -1, 0), (32, 32, 2, 1), (96, 1024, 8, 0),
                                  (512, 64, 1, 2), (256, 512, 32, 0), (128, 256, 4, 1),
                                  (256, 512, 0, 0), (32, 64, 0, 1), (1024, 2048, 0, 4),
                                  (0, 0, -1, 0), (0, 0, 2, 3)])
def test_pcg_plans(plan):
    p = W.q1_hex(10, seed=21)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_plan(*plan)
    x, r = A.solve(t(p.b), rtol=1e-9)
    assert r["status"] == B.OK
    assert true_rel(O, p.b, x.cpu().numpy()) <= 1.05e-9
    A.close()


def test_pcg_nonzero_guess_and_zero_rhs():
    p = W.edge_diffusion(40, seed=2)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    xo, _ = oracle.pcg(O, p.b, rtol=1e-12)
    x0 = t(xo.copy())
    x, r = A.solve(t(p.b), x=x0, rtol=1e-8, nonzero_guess=True)
    assert r["status"] == B.OK and r["iterations"] == 0
    x1 = t(0.5 * xo)
    x, r = A.solve(t(p.b), x=x1, rtol=1e-10, nonzero_guess=True)
    assert r["status"] == B.OK and true_rel(O, p.b, x.cpu().numpy()) <= 1.05e-10
    z = torch.zeros(p.nrows, dtype=torch.float64, device=DEV)
    xz = t(np.ones(p.nrows))
    x, r = A.solve(z, x=xz, nonzero_guess=True)
    assert r["status"] == B.OK and r["iterations"] == 0 and torch.count_nonzero(x) == 0
    A.close()


def test_pcg_error_paths_return_status():
    def dense_mat(D):
        i, j = np.nonzero(D)
        return assemble_both(D.shape[0], D.shape[1], i.astype(np.int32), j.astype(np.int32),
                             D[i, j])
    A, _ = dense_mat(np.diag([2.0, 0.0, 3.0]) + 0.1 * (np.ones((3, 3)) - np.eye(3)))
    assert A.solve(t(np.ones(3)))[1]["status"] == B.ERR_NOT_SPD
    A, _ = dense_mat(np.array([[1.0, 3.0], [3.0, 1.0]]))
    assert A.solve(t(np.array([1.0, -1.0])))[1]["status"] == B.ERR_BREAKDOWN
    p = W.poisson2d(8)
    A, _ = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    b = p.b.copy()
    b[5] = np.nan
    assert A.solve(t(b))[1]["status"] == B.ERR_NAN
    x, r = A.solve(t(np.random.default_rng(1).standard_normal(64)), maxit=1)
    assert r["status"] == B.ERR_MAXIT and r["iterations"] == 1
    # the context is still healthy after every error
    x, r = A.solve(t(p.b))
    assert r["status"] == B.OK


@pytest.mark.parametrize("solver", SOLVERS)
def test_time_limit_is_reported(solver):
    """A 1 ns wall-clock limit runs out after the first iteration: the device
    ends the loop (the per-CTA solver and the host-stepped loop at once, the
    graph at the end of its 8-trip body), the solve reports GBS_ERR_TIMEOUT
    with x finite, and the next solve on the same handle is unaffected."""
    p = W.poisson3d(16, seed=3)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(solver)
    x, r = A.solve(t(p.b), timeout_ns=1)
    assert r["status"] == B.ERR_TIMEOUT
    if solver == B.SOLVER_CTA:
        assert r["iterations"] == 1
    else:
        assert 1 <= r["iterations"] <= 8
        x2, r2 = A.solve(t(p.b), timeout_ns=1, host_loop=True)
        assert r2["status"] == B.ERR_TIMEOUT and r2["iterations"] == 1
    assert torch.isfinite(x).all()
    x, r = A.solve(t(p.b))
    assert r["status"] == B.OK and r["iterations"] > 1
    A.close()


# ------------------------------------------------------------------ FP32-refined

@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("make,rtol", [(lambda: W.q1_hex(10, seed=31), 1e-10),
                                       (lambda: W.poisson3d(24, seed=W.SEED_C3), 1e-10),
                                       (lambda: W.edge_diffusion(64, seed=32), 1e-8)])
def test_refined_parity(make, rtol, solver):
    p = make()
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(solver)
    x, r = A.solve(t(p.b), rtol=rtol, precision=B.FP32_REFINED, inner_rtol=1e-4)
    xo, ro = oracle.pcg_refined(O, p.b, rtol=rtol, inner_rtol=1e-4)
    assert r["status"] == B.OK and ro["status"] == oracle.OK
    xg = x.cpu().numpy()
    assert true_rel(O, p.b, xg) <= rtol * 1.05
    assert abs(r["outer_iterations"] - ro["outer_iterations"]) <= 1
    # the inner FP32 products in all (the oracle's inner loop is pinned
    # against a float32 emulation); FMAs and the reductions' order differ
    assert iters_close(r["iterations"], ro["iterations"]), (r, ro)
    x64, _ = oracle.pcg(O, p.b, rtol=1e-13)
    err = np.linalg.norm(xg - x64) / np.linalg.norm(x64)
    assert err <= 1e4 * rtol
    A.close()


@pytest.mark.parametrize("solver", SOLVERS)
def test_refined_stagnation_and_maxit(solver):
    p = W.poisson3d(10, seed=14)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(solver)
    x, r = A.solve(t(p.b), rtol=1e-10, precision=B.FP32_REFINED, inner_rtol=0.9, inner_maxit=1)
    assert r["status"] == B.ERR_STAGNATION
    x, r = A.solve(t(p.b), rtol=1e-10, precision=B.FP32_REFINED, max_outer=1)
    assert r["status"] == B.ERR_MAXIT and r["outer_iterations"] == 1
    A.close()


# ------------------------------------------------------------------ adjoint

def test_adjoint_parity_c4_small():
    p = W.edge_diffusion(32, seed=W.SEED_C4_SMALL)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    x, r = A.solve(t(p.b), rtol=1e-12)
    g = x - t(p.extra["x_target"])
    lam, dlda, dldv, ra = A.adjoint(x, g.contiguous(), rtol=1e-12)
    assert ra[0]["status"] == B.OK
    lo, dao, dvo, _ = oracle.adjoint(O, x.cpu().numpy(), g.cpu().numpy(), rtol=1e-13)
    for got, ref in ((lam, lo), (dlda, dao), (dldv, dvo)):
        got = got.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    # dL/dkappa through the edge signs matches the closed form -(l_a - l_b)(x_a - x_b)
    ea, eb = p.extra["edges"]
    gk = (dldv.cpu().numpy().reshape(-1, 4) * W.EDGE_SIGNS).sum(axis=1)
    l_, xx = lam.cpu().numpy(), x.cpu().numpy()
    la = np.where(ea >= 0, l_[ea], 0)
    lb = np.where(eb >= 0, l_[eb], 0)
    xa = np.where(ea >= 0, xx[ea], 0)
    xb = np.where(eb >= 0, xx[eb], 0)
    # the two forms round differently where they cancel: compare against the
    # size of the terms, not of the (possibly tiny) result
    scale = (np.abs(la) + np.abs(lb)) * (np.abs(xa) + np.abs(xb))
    assert np.all(np.abs(gk - (-(la - lb) * (xa - xb))) <= 1e-13 * scale + 1e-300)
    A.close()


def test_autograd_function_matches_finite_differences():
    from paper_2406_08646_gb300 import autograd as AG
    p = W.edge_diffusion(12, seed=5)
    ea, eb = p.extra["edges"]
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    kappa = t(p.extra["kappa"]).requires_grad_(True)
    b = t(p.b).requires_grad_(True)
    xt = t(p.extra["x_target"])
    signs = t(W.EDGE_SIGNS)

    def loss(kap, bb):
        v = (kap[:, None] * signs[None, :]).reshape(-1)
        x = AG.solve(v, bb, A, rtol=1e-13)
        return 0.5 * ((x - xt) ** 2).sum()

    L = loss(kappa, b)
    L.backward()
    gk, gb = kappa.grad.detach().cpu().numpy(), b.grad.detach().cpu().numpy()
    rng = np.random.default_rng(0)
    with torch.no_grad():
        for _ in range(3):
            d = t(rng.standard_normal(kappa.shape[0])) * kappa
            eps = 1e-6
            fd = (loss(kappa + eps * d, b) - loss(kappa - eps * d, b)).item() / (2 * eps)
            assert abs(fd - gk @ d.cpu().numpy()) <= 1e-5 * abs(fd) + 1e-9
            db = t(rng.standard_normal(b.shape[0]))
            fd = (loss(kappa, b + eps * db) - loss(kappa, b - eps * db)).item() / (2 * eps)
            assert abs(fd - gb @ db.cpu().numpy()) <= 1e-5 * abs(fd) + 1e-9
    A.close()


# ------------------------------------------------------------------ batched

def make_batch(nsys, seed, lo, hi):
    bt = W.batch(nsys, seed=seed, size_range=(lo, hi))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    return bt, A, O


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("precision", [B.FP64, B.FP32_REFINED])
def test_batched_parity(precision, solver):
    bt, A, O = make_batch(24, 41, 100, 6000)
    A.set_solver(solver)
    rp, col, val = (x.cpu().numpy() for x in A.csr())
    assert np.array_equal(rp, O.row_ptr) and np.array_equal(col, O.col)
    assert val.tobytes() == O.val.tobytes()
    x, rs = A.solve_batched(t(bt.b), rtol=1e-8, precision=precision)
    xo, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-8, precision=precision)
    xg = x.cpu().numpy()
    ro = bt.row_off
    resid = bt.b - oracle.spmv(O, xg)          # block diagonal: slice s depends on x_s only
    for s in range(bt.nsys):
        assert rs[s]["status"] == B.OK, (s, rs[s])
        sl = slice(ro[s], ro[s + 1])
        rsd = np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl])
        assert rsd <= 1.05e-8, (s, rsd)
        if precision == B.FP64:
            assert iters_close(rs[s]["iterations"], ros[s]["iterations"])
        else:
            assert abs(rs[s]["outer_iterations"] - ros[s]["outer_iterations"]) <= 1
    # graph replay gives the identical answer
    x2, rs2 = A.solve_batched(t(bt.b), rtol=1e-8, precision=precision)
    assert torch.equal(x, x2)
    A.close()


def test_batched_adjoint_and_ensemble():
    bt, A, O = make_batch(10, 43, 200, 3000)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-12)
    g = (x - t(bt.extra["x_target"])).contiguous()
    lam, dlda, dldv, ra = A.adjoint(x, g, batched=True, rtol=1e-12)
    assert all(q["status"] == B.OK for q in ra)
    lo, dao, dvo, _ = oracle.adjoint(O, x.cpu().numpy(), g.cpu().numpy(), rtol=1e-13)
    assert np.linalg.norm(dldv.cpu().numpy() - dvo) <= 1e-8 * np.linalg.norm(dvo)
    # ensemble: the stacked system with one global norm (Sec. 7 comparator)
    xe, re = A.solve(t(bt.b), rtol=1e-8)
    assert re["status"] == B.OK
    assert true_rel(O, bt.b, xe.cpu().numpy()) <= 1.05e-8
    A.close()


def test_launch_counter_and_phase_timers():
    p = W.poisson3d(12, seed=4)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(B.SOLVER_PHASES)
    c0 = B.launch_count()
    x, r = A.solve(t(p.b))
    # call-argument kernel + setup + final, and three kernels per trip: one
    # trip per iteration, the graph's body holding 8 trips (the last body's
    # trips after convergence return at once)
    n = B.launch_count() - c0 - 3
    assert n % 24 == 0 and 3 * r["iterations"] <= n < 3 * (r["iterations"] + 8), (n, r)
    ph = A.phase_ns()
    assert all(v > 0 for v in ph.values()), ph
    # the per-CTA solver: the call-argument kernel and one solver kernel
    A.set_solver(B.SOLVER_CTA)
    c0 = B.launch_count()
    x2, r2 = A.solve(t(p.b))
    assert B.launch_count() == c0 + 2 and r2["solver"] == B.SOLVER_CTA
    assert iters_close(r2["iterations"], r["iterations"])
    A.close()


def test_solver_auto_choice_and_determinism():
    p = W.poisson2d(32)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    x, r = A.solve(t(p.b), rtol=1e-10)
    assert r["solver"] == B.SOLVER_CTA            # 1024 rows: the latency path
    x2, r2 = A.solve(t(p.b), rtol=1e-10)
    assert torch.equal(x, x2) and r2 == r
    A.close()
    p = W.poisson2d(64)                           # 4096 rows: the phase kernels
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    x, r = A.solve(t(p.b), rtol=1e-10)
    assert r["solver"] == B.SOLVER_PHASES
    A.close()
    p = W.q1_hex(16, seed=6)                       # 117,649 nonzeros: the phase kernels
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    x, r = A.solve(t(p.b), rtol=1e-8)
    assert r["solver"] == B.SOLVER_PHASES and r["status"] == B.OK
    assert true_rel(O, p.b, x.cpu().numpy()) <= 1.05e-8
    A.close()


@pytest.mark.parametrize("kernel", [2, B.SPMV_SELL])
def test_batched_with_capped_grid_and_frozen_systems(kernel):
    """CTAs that walk several systems (grid capped at 1 CTA per SM) flush one
    reduction per system; systems that converge early stay frozen while the
    others iterate."""
    bt, A, O = make_batch(40, 47, 50, 4000)
    A.set_plan(64, 128, kernel, 1)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-9)
    _, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-9)
    xg = x.cpu().numpy()
    ro = bt.row_off
    resid = bt.b - oracle.spmv(O, xg)
    its = [q["iterations"] for q in rs]
    assert max(its) > min(its)
    for s in range(bt.nsys):
        assert rs[s]["status"] == B.OK
        sl = slice(ro[s], ro[s + 1])
        assert np.linalg.norm(resid[sl]) <= 1.05e-9 * np.linalg.norm(bt.b[sl])
        assert iters_close(rs[s]["iterations"], ros[s]["iterations"])
    A.close()


def test_autotune_keeps_a_valid_plan_and_parity():
    p = W.q1_hex(14, seed=12)
    A, O = assemble_both(p.nrows, p.ncols, p.i, p.j, p.v)
    A.set_solver(B.SOLVER_PHASES)
    A.autotune()
    pl = A.plan()
    assert pl["kernel"] in (B.SPMV_SELL, 1, 2, 4, 8, 32) and pl["spmv_grid"] >= 1
    x, r = A.solve(t(p.b), rtol=1e-9)
    assert r["status"] == B.OK and true_rel(O, p.b, x.cpu().numpy()) <= 1.05e-9
    y = A.mult(t(p.b)).cpu().numpy()
    assert np.all(np.abs(y - oracle.spmv(O, p.b)) <= 1e-12 * abs_bound(O, p.b))
    A.close()
