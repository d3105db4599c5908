"""GPU parity of the size split of a batched solve (GBS_SOLVER_SPLIT: the
systems of at least split_rows rows on the phase kernels, the rest on the
per-CTA solver) against the oracle's batched PCG, through
ksp_solve_cg_batched / ksp_adjoint_batched.

Bars (those of the batched parity tests): every system OK with its true
residual, recomputed by the oracle from the GPU's x, within 1.05 rtol;
FP64 iteration counts within max(2, 1%) of the oracle's, refined outer
counts within 1.  Also: each system reports the engine it ran on; the
split's answer equals each engine's own answer for its systems bit for bit
(the per-CTA part) or to the tolerance (the phase-kernel part, whose
blocks are cut for the large systems alone); the extremes (every system above or
below the split) and a change of split or solver between solves (graphs
rebuilt) work; the adjoint and the refined solve split the same way."""
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


def make_batch(nsys, seed, lo, hi):
    bt = W.batch(nsys, seed=seed, size_range=(lo, hi))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    return bt, A, O


def check_against_oracle(bt, O, x, rs, ros, precision):
    resid = bt.b - oracle.spmv(O, x.cpu().numpy())
    ro = bt.row_off
    for s in range(bt.nsys):
        assert rs[s]["status"] == B.OK, (s, rs[s])
        sl = slice(ro[s], ro[s + 1])
        rsd = np.linalg.norm(resid[sl]) / np.linalg.norm(bt.b[sl])
        assert rsd <= 1.05e-8, (s, rsd)
        if precision == B.FP64:
            assert iters_close(rs[s]["iterations"], ros[s]["iterations"]), (s, rs[s], ros[s])
        else:
            assert abs(rs[s]["outer_iterations"] - ros[s]["outer_iterations"]) <= 1


@pytest.mark.parametrize("precision", [B.FP64, B.FP32_REFINED])
def test_split_parity_and_engines(precision):
    bt, A, O = make_batch(30, 61, 200, 20000)
    rows = np.sort(bt.nrows)[::-1]
    cut = int(rows[7])                              # the 8 largest on the phase kernels
    A.set_solver(B.SOLVER_SPLIT, split_rows=cut)
    x, rs = A.solve_batched(t(bt.b), rtol=1e-8, precision=precision)
    _, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-8, precision=precision)
    check_against_oracle(bt, O, x, rs, ros, precision)
    for s in range(bt.nsys):
        want = B.SOLVER_PHASES if bt.nrows[s] >= cut else B.SOLVER_CTA
        assert rs[s]["solver"] == want, (s, rs[s])
    assert sum(r["solver"] == B.SOLVER_PHASES for r in rs) == int((bt.nrows >= cut).sum())
    # the small systems equal the per-CTA solver's own batched solve bit for
    # bit (same kernel, same order); the large ones run on tables cut for
    # them alone (other blocks, so other reduction orders) and agree with
    # the phase kernels' batched solve to the tolerance
    A.set_solver(B.SOLVER_PHASES)
    xp, rp = A.solve_batched(t(bt.b), rtol=1e-8, precision=precision)
    A.set_solver(B.SOLVER_CTA)
    xc, rc = A.solve_batched(t(bt.b), rtol=1e-8, precision=precision)
    ro = bt.row_off
    for s in range(bt.nsys):
        sl = slice(ro[s], ro[s + 1])
        if bt.nrows[s] >= cut:
            assert torch.linalg.norm(x[sl] - xp[sl]) <= 1e-5 * torch.linalg.norm(xp[sl]), s
            if precision == B.FP64:
                assert iters_close(rs[s]["iterations"], rp[s]["iterations"]), s
        else:
            assert torch.equal(x[sl], xc[sl]), s
            assert rs[s]["iterations"] == rc[s]["iterations"], s
    # the split again after other solvers: the same answer
    A.set_solver(B.SOLVER_SPLIT)
    x2, rs2 = A.solve_batched(t(bt.b), rtol=1e-8, precision=precision)
    assert torch.equal(x, x2)
    A.close()


def test_split_extremes_and_changes():
    bt, A, O = make_batch(16, 62, 300, 8000)
    _, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-9)
    for cut, n_phases in ((1, bt.nsys), (int(bt.nrows.max()) + 1, 0),
                          (int(np.sort(bt.nrows)[-3]), 3)):
        A.set_solver(B.SOLVER_SPLIT, split_rows=cut)
        x, rs = A.solve_batched(t(bt.b), rtol=1e-9)
        resid = bt.b - oracle.spmv(O, x.cpu().numpy())
        for s in range(bt.nsys):
            assert rs[s]["status"] == B.OK
            assert iters_close(rs[s]["iterations"], ros[s]["iterations"])
            sl = slice(bt.row_off[s], bt.row_off[s + 1])
            assert np.linalg.norm(resid[sl]) <= 1.05e-9 * np.linalg.norm(bt.b[sl])
        assert sum(r["solver"] == B.SOLVER_PHASES for r in rs) == n_phases, cut
    assert A.tuning()["split_rows"] == int(np.sort(bt.nrows)[-3])
    with pytest.raises(B.GbsError):
        B.mat_set_split_rows(A.h, 0)
    # an ensemble solve of the same handle is not split
    xe, re = A.solve(t(bt.b), rtol=1e-8)
    assert re["status"] == B.OK and re["solver"] in (B.SOLVER_PHASES, B.SOLVER_CTA)
    A.close()


def test_split_adjoint_and_limits():
    bt, A, O = make_batch(12, 63, 200, 5000)
    A.set_solver(B.SOLVER_SPLIT, split_rows=int(np.sort(bt.nrows)[-4]))
    x, rs = A.solve_batched(t(bt.b), rtol=1e-12)
    assert all(r["status"] == B.OK for r in rs)
    g = (x - t(bt.extra["x_target"])).contiguous()
    lam, dlda, dldv, ra = A.adjoint(x, g, batched=True, rtol=1e-12)
    assert all(q["status"] == B.OK for q in ra)
    _, _, dvo, _ = oracle.adjoint(O, x.cpu().numpy(), g.cpu().numpy(), rtol=1e-13)
    assert np.linalg.norm(dldv.cpu().numpy() - dvo) <= 1e-8 * np.linalg.norm(dvo)
    # an iteration limit stops both parts with MAXIT and the oracle's counts
    x, rs = A.solve_batched(t(bt.b), rtol=1e-14, maxit=5)
    _, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-14, maxit=5)
    for s in range(bt.nsys):
        assert rs[s]["status"] == ros[s]["status"] == B.ERR_MAXIT
        assert rs[s]["iterations"] == ros[s]["iterations"] == 5
    A.close()
