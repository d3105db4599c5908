"""GPU parity of the sliced copy's column patterns (mat_set_slice_patterns).

With patterns a 32-row slice stores the union of its rows' offsets col - row
once and a 32-bit mask per row instead of a column index per entry; the row
products sum the same terms in the same (CSR) order, so every result must be
BIT-IDENTICAL with patterns on and off: SpMV, every solve engine and form,
the refined solve (FP32 copy), the adjoint, BiCG / TFQMR (the transpose's
copy) and batched solves.  The choice itself is integer work and is checked
exactly against a count from the oracle's CSR: patterns are taken when every
slice's union has at most 32 offsets and the unions add up to at most 1.25
times the slices' longest rows; the copy then holds 32 x (sum of unions)
entries.  SpMV also meets the oracle bar of the parity suite."""
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


def assemble(p):
    A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
    A.set_values(t(p.v))
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    return A, O


def expected_slices(O, row_off):
    """(slices, patterns taken, entries of the copy) from the CSR pattern."""
    ws, us = [], []
    for q in range(len(row_off) - 1):
        for r0 in range(int(row_off[q]), int(row_off[q + 1]), 32):
            r1 = min(r0 + 32, int(row_off[q + 1]))
            offs, w = set(), 0
            for r in range(r0, r1):
                cs = O.col[O.row_ptr[r]:O.row_ptr[r + 1]].astype(np.int64)
                w = max(w, len(cs))
                offs.update((cs - r).tolist())
            ws.append(w)
            us.append(len(offs))
    fit = len(ws) > 0 and max(us) <= 32 and 4 * sum(us) <= 5 * sum(ws)
    return len(ws), fit, 32 * sum(us if fit else ws)


def band(n, offsets, holes, seed):
    """Rows draw their columns from r + offsets (in range), each row lacking
    `holes` of the nonzero offsets (chosen by r mod 32): a slice's union is
    all of offsets while its longest row is len(offsets) - holes.  Diagonally
    dominant, so that it is SPD when the offsets are symmetric."""
    rng = np.random.default_rng(seed)
    offs = np.array(sorted(offsets), np.int64)
    nz = offs[offs != 0]
    I, J = [], []
    for r in range(n):
        k = r % 32
        lack = {int(nz[(k + 5 * h) % len(nz)]) for h in range(holes)}
        for o in offs:
            c = r + int(o)
            if 0 <= c < n and int(o) not in lack:
                I.append(r)
                J.append(c)
    I = np.array(I, np.int32)
    J = np.array(J, np.int32)
    v = np.where(I == J, 2.0 * len(offs), -rng.uniform(0.1, 1.0, len(I)))
    return W.Problem("band", n, n, I, J, v, rng.standard_normal(n))


CASES = [
    ("q1hex_12", lambda: W.q1_hex(12, seed=W.SEED_C2)),
    ("poisson3d_24", lambda: W.poisson3d(24, seed=W.SEED_C3)),
    ("poisson2d_64", lambda: W.poisson2d(64)),
    ("edge_77", lambda: W.edge_diffusion(77, seed=5)),
    ("band_32_offsets", lambda: band(5000, range(-16, 16), 6, 1)),
    ("band_33_offsets", lambda: band(5000, range(-16, 17), 7, 2)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_choice_sizes_and_bit_identical_spmv(name, make):
    p = make()
    A, O = assemble(p)
    A.set_plan(kernel=B.SPMV_SELL)
    ns, fit, entries = expected_slices(O, [0, p.nrows])
    assert fit == (name != "band_33_offsets")
    x = np.random.default_rng(7).standard_normal(p.ncols)
    y_on = A.mult(t(x))
    assert A.slices() == {"nslices": ns, "pattern_slices": ns if fit else 0, "entries": entries}
    A.set_slice_patterns(False)
    assert A.slices()["pattern_slices"] == 0
    y_off = A.mult(t(x))
    assert torch.equal(y_on, y_off)
    yo = oracle.spmv(O, x)
    Oa = oracle.CSR(O.nrows, O.ncols, O.row_ptr, O.col, O.perm, O.jmap, O.ncoo, np.abs(O.val))
    assert np.all(np.abs(y_on.cpu().numpy() - yo) <= 1e-12 * oracle.spmv(Oa, np.abs(x)))
    A.set_slice_patterns(True)
    assert A.slices()["pattern_slices"] == (ns if fit else 0)
    assert torch.equal(A.mult(t(x)), y_on)
    A.close()


def test_empty_rows_and_slices():
    """Whole slices of empty rows (width 0, empty pattern), a ragged last
    slice and a matrix with no nonzero at all."""
    n = 150
    r = np.arange(n)
    keep = (r < 32) | (r >= 96)
    i = np.concatenate([r[keep], r[keep][:-1]]).astype(np.int32)
    j = np.concatenate([r[keep], r[keep][1:]]).astype(np.int32)
    v = np.random.default_rng(3).standard_normal(i.shape[0])
    p = W.Problem("holes", n, n, i, j, v, np.ones(n))
    A, O = assemble(p)
    A.set_plan(kernel=B.SPMV_SELL)
    x = np.random.default_rng(4).standard_normal(n)
    y = A.mult(t(x))
    ns, fit, entries = expected_slices(O, [0, n])
    assert fit and A.slices() == {"nslices": ns, "pattern_slices": ns, "entries": entries}
    assert np.array_equal(y.cpu().numpy()[~keep], np.zeros((~keep).sum()))
    A.set_slice_patterns(False)
    assert torch.equal(A.mult(t(x)), y)
    A.close()
    Z = B.Mat.from_coo(64, 64, t(np.full(5, -1, np.int32)), t(np.zeros(5, np.int32)))
    Z.set_values(t(np.ones(5)))
    Z.set_plan(kernel=B.SPMV_SELL)
    assert not torch.any(Z.mult(t(np.ones(64))))
    Z.close()


def solve_both(A, fn):
    A.set_slice_patterns(True)
    a = fn()
    A.set_slice_patterns(False)
    b = fn()
    A.set_slice_patterns(True)
    return a, b


def same(a, b):
    (xa, ra), (xb, rb) = a, b
    assert torch.equal(xa, xb)
    ra = ra if isinstance(ra, list) else [ra]
    rb = rb if isinstance(rb, list) else [rb]
    for u, w in zip(ra, rb):
        assert u["status"] == w["status"] and u["iterations"] == w["iterations"], (u, w)


@pytest.mark.parametrize("make", [lambda: W.q1_hex(12, seed=W.SEED_C2),
                                  lambda: W.poisson3d(24, seed=W.SEED_C3),
                                  lambda: W.edge_diffusion(64, seed=6)])
def test_solves_bit_identical(make):
    p = make()
    A, O = assemble(p)
    assert A.mult(t(p.b)) is not None and A.slices()["pattern_slices"] > 0
    b = t(p.b)
    for solver in (B.SOLVER_PHASES, B.SOLVER_CTA):
        A.set_solver(solver)
        for form in (B.CG_TEXTBOOK, B.CG_SINGLE_REDUCTION, B.CG_SINGLE_KERNEL):
            A.set_cg_form(form)
            same(*solve_both(A, lambda: A.solve(b, rtol=1e-9)))
        same(*solve_both(A, lambda: A.solve(b, rtol=1e-9, method=B.KSP_PIPECG)))
        same(*solve_both(A, lambda: A.solve(b, rtol=1e-9, precision=B.FP32_REFINED)))
        x, r = A.solve(b, rtol=1e-10)
        g = t(np.random.default_rng(1).standard_normal(p.nrows))
        ad = solve_both(A, lambda: A.adjoint(x, g, rtol=1e-10))
        for u, w in zip(ad[0], ad[1]):
            if isinstance(u, torch.Tensor):
                assert torch.equal(u, w)
    xo, ro = oracle.pcg(O, p.b, rtol=1e-9)
    A.set_solver(B.SOLVER_PHASES)
    A.set_cg_form(B.CG_TEXTBOOK)
    x, r = A.solve(b, rtol=1e-9)
    assert r["status"] == ro["status"] == B.OK
    assert abs(r["iterations"] - ro["iterations"]) <= max(2, int(np.ceil(0.01 * ro["iterations"])))
    A.close()


@pytest.mark.parametrize("method", [B.KSP_BICG, B.KSP_TFQMR])
def test_nonsymmetric_and_transpose_bit_identical(method):
    p = W.convdiff2d(48, 0.7, -0.4, seed=W.SEED_C6)
    A, O = assemble(p)
    b = t(p.b)
    for solver in (B.SOLVER_PHASES, B.SOLVER_CTA):
        A.set_solver(solver)
        same(*solve_both(A, lambda: A.solve(b, rtol=1e-9, method=method)))
    assert A.slices()["pattern_slices"] == A.slices()["nslices"] > 0
    A.close()


def test_batched_bit_identical():
    bt = W.batch(12, seed=45, size_range=(300, 6000))
    A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
    A.set_values(t(bt.v))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    O = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(O, bt.v)
    b = t(bt.b)
    for solver in (B.SOLVER_PHASES, B.SOLVER_CTA):
        A.set_solver(solver)
        same(*solve_both(A, lambda: A.solve_batched(b, rtol=1e-9)))
        same(*solve_both(A, lambda: A.solve_batched(b, rtol=1e-9, precision=B.FP32_REFINED)))
    ns, fit, entries = expected_slices(O, bt.row_off)
    assert A.slices() == {"nslices": ns, "pattern_slices": ns if fit else 0, "entries": entries}
    A.close()


def test_argument_check():
    p = W.poisson2d(16)
    A, _ = assemble(p)
    assert B.lib().mat_set_slice_patterns(A.h, 2) == B.ERR_ARG
    A.close()
