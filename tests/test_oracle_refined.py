"""Pins of the oracle's FP32-inner / FP64-refined PCG inner loop (Sec. 2,
challenge A7: a single-precision inner solve under a double-precision outer
one), beyond the final-residual pins in test_oracle_pcg.py.

An independent emulation, written here from the reading of the method rather
than from the oracle's code, runs the same algorithm with numpy scalars and
arrays of the stated precisions -- FP64 outer residual r = b - A x and its
norm s, inner right-hand side RN32(r / s), FP32 Jacobi-PCG on RN32(A) with
RN32(1 / a_ii), FP32 products and FP32 pairwise sums, stop when
sqrt(r_in . r_in) <= max(inner_rtol, rtol ||b|| / (2 s)) times its initial
value (or inner_maxit, or sigma <= 0), x += s d in FP64 -- and must
reproduce the oracle's inner iteration count for every outer step and its x
bit for bit.  Cases cover both terms of the inner target (inner_rtol for
the early steps, the rtol term for the last correction).  Planted mistakes
(FP64 accumulation in the FP32 dot products, the target's factor 1/2 turned
to 1, no rtol term in the target, the beta term dropped, alpha from
r_in . r_in instead of r_in . z_in) are compiled into copies of the oracle,
and each must fail the emulation pin."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2406_08646_gb300 import workloads as W

f32, f64 = np.float32, np.float64


def seq_sum(v):
    """Left-to-right sum in v's own precision (each addition rounded)."""
    return np.add.accumulate(v)[-1] if v.shape[0] else v.dtype.type(0)


def pair_sum(v):
    """Pairwise sum in v's own precision: halves of more than 8 terms summed
    recursively and added, at most 8 terms left to right."""
    n = v.shape[0]
    if n <= 8:
        return seq_sum(v) if n else v.dtype.type(0)
    h = n // 2
    return pair_sum(v[:h]) + pair_sum(v[h:])


def spmv_seq(A, vals, x):
    """y_i = sum over row i in CSR order, each product and addition rounded in
    the precision of vals and x (no fused multiply-add)."""
    rp = A.row_ptr
    lens = np.diff(rp)
    y = np.zeros(A.nrows, vals.dtype)
    for k in range(int(lens.max()) if A.nrows else 0):
        live = k < lens
        idx = np.where(live, rp[:-1] + k, 0)
        prod = vals[idx] * x[A.col[idx]]
        y = np.where(live, y + prod, y)
    return y


def emulate(A, b, rtol, inner_rtol, inner_maxit, max_outer):
    """The refined solve, step by step (returns x, status, inner counts, the
    target term each step used)."""
    n = A.nrows
    a64 = A.val.astype(f64)
    diag = np.zeros(n)
    for r in range(n):
        for q in range(A.row_ptr[r], A.row_ptr[r + 1]):
            if A.col[q] == r:
                diag[r] = a64[q]
    dinv64 = f64(1.0) / diag
    dinv32 = dinv64.astype(f32)
    a32 = a64.astype(f32)
    x = np.zeros(n)
    bnorm = np.sqrt(seq_sum(b * b))
    counts, terms = [], []
    prev, stall = np.inf, 0
    while True:
        r = b - spmv_seq(A, a64, x)
        rn = np.sqrt(seq_sum(r * r))
        if rn <= rtol * bnorm:
            return x, "ok", counts, terms
        if len(counts) >= max_outer:
            return x, "maxit", counts, terms
        if counts:
            stall = stall + 1 if rn > 0.5 * prev else 0
            if stall >= 2:
                return x, "stagnation", counts, terms
        prev = rn
        s = rn
        rt = 0.5 * rtol * bnorm / s
        tgt = max(inner_rtol, rt)
        terms.append("rtol" if rt > inner_rtol else "inner_rtol")
        r32 = (r / s).astype(f32)
        d = np.zeros(n, f32)
        z = dinv32 * r32
        p = z.copy()
        rho = pair_sum(r32 * z)
        rr = pair_sum(r32 * r32)
        thr = tgt * f64(np.sqrt(rr))
        it = 0
        while f64(np.sqrt(rr)) > thr and it < inner_maxit:
            q = spmv_seq(A, a32, p)
            sigma = pair_sum(p * q)
            if not sigma > 0:
                break
            it += 1
            alpha = rho / sigma
            d = d + alpha * p
            r32 = r32 - alpha * q
            z = dinv32 * r32
            rho_new = pair_sum(r32 * z)
            rr = pair_sum(r32 * r32)
            beta = rho_new / rho
            p = z + beta * p
            rho = rho_new
        if it == 0:
            return x, "breakdown", counts, terms
        counts.append(it)
        x = x + s * d.astype(f64)


def assemble(p):
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(A, p.v)
    return A


CASES = [
    ("edge_12", lambda: W.edge_diffusion(12, seed=3), 1e-8, 1e-4),
    ("edge_12_tight_inner", lambda: W.edge_diffusion(12, seed=3), 1e-8, 1e-6),
    ("q1hex_4", lambda: W.q1_hex(4, seed=8), 1e-10, 1e-4),
    ("poisson3d_6", lambda: W.poisson3d(6, seed=5), 1e-9, 1e-3),
]

STATUS = {"ok": oracle.OK, "maxit": oracle.ERR_MAXIT, "stagnation": oracle.ERR_STAGNATION,
          "breakdown": oracle.ERR_BREAKDOWN}


def pin_matches_emulation(solve, make, rtol, inner_rtol):
    p = make()
    A = assemble(p)
    xe, st, counts, terms = emulate(A, p.b, rtol, inner_rtol, 10000, 30)
    x, r, trace = solve(A, p.b, rtol, inner_rtol)
    assert r["status"] == STATUS[st], (r, st)
    assert trace == counts, (trace, counts)
    assert r["outer_iterations"] == len(counts)
    assert r["iterations"] == sum(counts)
    assert x.tobytes() == xe.tobytes()
    return terms


def oracle_solve(A, b, rtol, inner_rtol):
    return oracle.pcg_refined(A, b, rtol=rtol, inner_rtol=inner_rtol, inner_maxit=10000,
                              max_outer=30, want_trace=True)


@pytest.mark.parametrize("name,make,rtol,inner_rtol", CASES, ids=[c[0] for c in CASES])
def test_inner_loop_matches_float32_emulation(name, make, rtol, inner_rtol):
    pin_matches_emulation(oracle_solve, make, rtol, inner_rtol)


def test_both_target_terms_are_exercised():
    """The cases above include outer steps stopped by inner_rtol and last
    corrections stopped by the rtol ||b|| / (2 s) term."""
    seen = set()
    for _, make, rtol, inner_rtol in CASES:
        p = make()
        _, st, counts, terms = emulate(assemble(p), p.b, rtol, inner_rtol, 10000, 30)
        assert st == "ok"
        seen.update(terms)
    assert seen == {"rtol", "inner_rtol"}


def test_last_correction_stops_at_the_rtol_term():
    """The last correction needs only rtol ||b|| / (2 s): with an inner target
    far tighter than needed, the last step takes fewer inner iterations than
    a full inner_rtol solve would, and the final residual still meets rtol."""
    p = W.edge_diffusion(12, seed=3)
    A = assemble(p)
    x, r, trace = oracle.pcg_refined(A, p.b, rtol=1e-8, inner_rtol=1e-7, inner_maxit=10000,
                                     want_trace=True)
    assert r["status"] == oracle.OK
    assert r["true_rel_residual"] <= 1e-8
    xe, st, counts, terms = emulate(A, p.b, 1e-8, 1e-7, 10000, 30)
    assert terms[-1] == "rtol" and trace == counts
    # a first step solved to 1e-7 takes more inner iterations than the
    # last one, which only has to close the remaining gap
    assert counts[-1] < counts[0]


# ------------------------------------------------------------ planted mistakes

MUTANTS = [
    ("FP64 accumulation in the FP32 dot products",
     "  if (n <= 8) {\n    float s = 0.0f;",
     "  {\n    double t = 0.0;\n    for (int64_t i = 0; i < n; ++i) t += (double)x[i] * (double)y[i];\n"
     "    return (float)t;\n  }\n  if (n <= 8) {\n    float s = 0.0f;"),
    ("FP32 dot products summed left to right",
     "  if (n <= 8) {\n    float s = 0.0f;", "  if (1) {\n    float s = 0.0f;"),
    ("target factor 1/2 turned to 1", "const double tgt = fmax(inner_rtol, 0.5 * rtol * bnorm / s);",
     "const double tgt = fmax(inner_rtol, 1.0 * rtol * bnorm / s);"),
    ("no rtol term in the target", "const double tgt = fmax(inner_rtol, 0.5 * rtol * bnorm / s);",
     "const double tgt = inner_rtol;"),
    ("beta term dropped", "for (int64_t i = 0; i < n; ++i) p32[i] = z32[i] + beta * p32[i];",
     "for (int64_t i = 0; i < n; ++i) p32[i] = z32[i] + 0.0f * beta * p32[i];"),
    ("alpha from r.r", "float alpha = rho / sigma;", "float alpha = rr / sigma;"),
]


def _mutant(tmpdir, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, name
    src = src.replace(old, new)
    c = os.path.join(tmpdir, "mutant.c")
    so = os.path.join(tmpdir, f"libmut{abs(hash(name))}.so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           c, "-o", so, "-lm"])
    lib = ctypes.CDLL(so)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.orc_pcg_refined.restype = ctypes.c_int
    lib.orc_pcg_refined.argtypes = [I64, P, P, P, P, P, D, D, I64, I32, ctypes.c_int, P, P]
    pp = lambda a_: a_.ctypes.data_as(ctypes.c_void_p)

    def solve(A, b, rtol, inner_rtol):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(A.nrows)
        res = oracle._Result()
        tr = np.zeros(30, np.int32)
        lib.orc_pcg_refined(A.nrows, pp(A.row_ptr), pp(A.col), pp(A.val), pp(b), pp(x), rtol,
                            inner_rtol, 10000, 30, 0, ctypes.byref(res), pp(tr))
        r = res.as_dict()
        return x, r, [int(v) for v in tr[:r["outer_iterations"]]]

    return solve


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_fail_the_emulation_pin(name, old, new):
    with tempfile.TemporaryDirectory() as d:
        solve = _mutant(d, name, old, new)
        failed = 0
        for _, make, rtol, inner_rtol in CASES:
            try:
                pin_matches_emulation(solve, make, rtol, inner_rtol)
            except AssertionError:
                failed += 1
        assert failed >= 1, f"mutant '{name}' passed every case"
