"""The autotuner: its choice keeps parity with the oracle, is persisted in a
tuning file keyed by the matrix and the device, and is reloaded by a new
handle of the same matrix without timing; the CG form it can choose (the
single-reduction loop) matches the oracle's textbook and single-reduction
PCG."""
import os
import tempfile

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


def check_parity(A, O, b, rtol):
    x, r = A.solve(t(b), rtol=rtol)
    _, ro = oracle.pcg(O, b, rtol=rtol)
    assert r["status"] == B.OK and ro["status"] == oracle.OK
    assert iters_close(r["iterations"], ro["iterations"]), (r, ro)
    tr = np.linalg.norm(b - oracle.spmv(O, x.cpu().numpy())) / np.linalg.norm(b)
    assert tr <= 1.05 * rtol, tr


def test_tuning_file_roundtrip_single_system():
    p = W.q1_hex(24, seed=55)
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
        A.set_values(t(p.v))
        assert A.autotune(path) is False                 # tuned, line appended
        plan1, tun1, sl1 = A.plan(), A.tuning(), A.slices()
        assert len(open(path).read().split("|")[1].split()) == 8
        assert tun1["solver"] in (B.SOLVER_PHASES, B.SOLVER_CTA)
        assert tun1["cg_form"] in (B.CG_TEXTBOOK, B.CG_SINGLE_REDUCTION, B.CG_SINGLE_KERNEL)
        check_parity(A, O, p.b, 1e-9)
        A.close()
        lines = open(path).read().splitlines()
        assert len(lines) == 1 and "fp64" in lines[0] and "sm=" in lines[0]
        # a new handle of the same matrix takes the stored tuning
        A2 = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
        A2.set_values(t(p.v))
        assert A2.autotune(path) is True
        assert A2.plan() == plan1 and A2.tuning() == tun1
        assert A2.slices() == sl1                         # the pattern setting too
        check_parity(A2, O, p.b, 1e-9)
        A2.close()
        assert len(open(path).read().splitlines()) == 1
        # another matrix is another key
        q = W.q1_hex(20, seed=56)
        A3 = B.Mat.from_coo(q.nrows, q.ncols, t(q.i), t(q.j))
        A3.set_values(t(q.v))
        assert A3.autotune(path) is False
        assert len(open(path).read().splitlines()) == 2
        A3.close()


def test_tuning_file_roundtrip_batched():
    bt = W.batch(48, seed=61, size_range=(200, 4000))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
        A.set_values(t(bt.v))
        assert A.autotune(path) is False
        tun = A.tuning()
        x, rs = A.solve_batched(t(bt.b), rtol=1e-9)
        _, ros = oracle.pcg_batched(O, bt.row_off, bt.b, rtol=1e-9)
        resid = bt.b - oracle.spmv(O, x.cpu().numpy())
        ro = bt.row_off
        for s in range(bt.nsys):
            assert rs[s]["status"] == B.OK and rs[s]["solver"] == (
                B.SOLVER_CTA if tun["solver"] == B.SOLVER_CTA else B.SOLVER_PHASES)
            assert iters_close(rs[s]["iterations"], ros[s]["iterations"]), (s, rs[s], ros[s])
            sl = slice(ro[s], ro[s + 1])
            assert np.linalg.norm(resid[sl]) <= 1.05e-9 * np.linalg.norm(bt.b[sl])
        A.close()
        A2 = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
        A2.set_values(t(bt.v))
        assert A2.autotune(path) is True and A2.tuning() == tun
        A2.close()


@pytest.mark.parametrize("make,rtol", [(lambda: W.q1_hex(18, seed=7), 1e-9),
                                       (lambda: W.edge_diffusion(200, seed=8), 1e-8)])
def test_single_reduction_form_through_ksp_solve_cg(make, rtol):
    """mat_set_cg_form(SINGLE_REDUCTION): ksp_solve_cg runs the two-kernel
    loop (the update_p phase timer stays 0) and matches the oracle's
    single-reduction PCG; the textbook form is back after resetting."""
    p = make()
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    A.set_values(t(p.v))
    A.set_solver(B.SOLVER_PHASES)
    A.set_cg_form(B.CG_SINGLE_REDUCTION)
    b = t(p.b)
    x = torch.empty_like(b)
    r = B.ksp_solve_cg(A.h, b, x, B.make_opts(rtol=rtol))[0]
    _, ro = oracle.pcg_sr(O, p.b, rtol=rtol)
    assert r["status"] == B.OK and iters_close(r["iterations"], ro["iterations"]), (r, ro)
    assert A.phase_ns()["update_p"] == 0
    tr = np.linalg.norm(p.b - oracle.spmv(O, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert tr <= 1.05 * rtol
    A.set_cg_form(B.CG_TEXTBOOK)
    x2, r2 = A.solve(b, rtol=rtol)
    assert r2["status"] == B.OK and A.phase_ns()["update_p"] > 0
    with pytest.raises(B.GbsError):
        A.set_cg_form(7)
    A.close()
