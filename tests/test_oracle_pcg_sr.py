"""Pins of the oracle's single-reduction Jacobi-PCG (Chronopoulos and Gear's
form: the two inner products of an iteration in one reduction after the
product w = A u), the form the GPU's two-kernel CG iteration follows.

What fixes it, independently of the oracle's own code:
  * PCG's iterates in exact arithmetic: after k = 1..12 iterations its x
    equals the textbook PCG's x (orc_pcg, pinned on its own) to rounding, and
    both reach the same counts and solutions at convergence;
  * the recurrences' invariants after k iterations: r = b - A x, u = M^-1 r,
    w = A u, s = A p, recomputed here with a dense matrix;
  * dense SPD solves, finite termination in three iterations for a right-hand
    side in the span of three Laplacian eigenvectors, the C1 closed form
    (one iteration), the error paths, a nonzero guess, the batched driver and
    a degenerate batch;
  * planted mistakes: the C source is recompiled with one slip at a time (a
    dropped term of the alpha denominator, beta inverted, s updated without
    beta, r updated with p instead of s, the residual norm taken of u) and
    each mutant must fail at least one of the pins above."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2406_08646_gb300 import workloads as W


def assemble(p):
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(A, p.v)
    return A


def dense(A):
    D = np.zeros((A.nrows, A.ncols))
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    D[rows, A.col] = A.val
    return D


def from_dense(D):
    i, j = np.nonzero(D)
    A = oracle.coo_symbolic(D.shape[0], D.shape[1], i.astype(np.int32), j.astype(np.int32))
    oracle.coo_numeric(A, D[i, j])
    return A


MAKERS = [lambda: W.edge_diffusion(16, seed=5), lambda: W.q1_hex(6, seed=6),
          lambda: W.poisson3d(9, seed=7), lambda: W.poisson2d(40)]


# ------------------------------------------------------------ the pins, as
# functions of the solver under test (the oracle, or a planted mutant)

def pin_same_iterates_as_pcg(solve, make):
    p = make()
    A = assemble(p)
    b = p.b if p.name != "poisson2d_40" else np.random.default_rng(3).standard_normal(p.nrows)
    x, r = solve(A, b, 1e-10, None)
    xc, rc = oracle.pcg(A, b, rtol=1e-10)
    assert r["status"] == rc["status"] == oracle.OK
    assert abs(r["iterations"] - rc["iterations"]) <= 1, (r, rc)
    assert np.linalg.norm(x - xc) <= 1e-7 * np.linalg.norm(xc)
    assert r["true_rel_residual"] <= 1e-9
    assert r["rnorm0"] == rc["rnorm0"]


def pin_iterates_after_k(solve, k):
    """x after k iterations equals PCG's x after k iterations to rounding."""
    p = W.edge_diffusion(14, seed=3)
    A = assemble(p)
    x, r = solve(A, p.b, 1e-15, k)
    xc, rc = oracle.pcg(A, p.b, rtol=1e-15, maxit=k)
    assert r["status"] == rc["status"] == oracle.ERR_MAXIT
    assert r["iterations"] == rc["iterations"] == k
    assert np.linalg.norm(x - xc) <= 1e-11 * np.linalg.norm(xc)
    assert r["rnorm"] == pytest.approx(rc["rnorm"], rel=1e-8)


def pin_invariants(solve_aux, k):
    p = W.edge_diffusion(14, seed=3)
    A = assemble(p)
    D = dense(A)
    dinv = 1.0 / np.diag(D)
    x, r, v = solve_aux(A, p.b, 1e-15, k)
    assert r["status"] == oracle.ERR_MAXIT and r["iterations"] == k
    scale = np.linalg.norm(D, 2)

    def close(lhs, rhs, ref):
        return np.linalg.norm(lhs - rhs) <= 1e-10 * max(np.linalg.norm(ref), 1e-300)

    assert close(v["r"], p.b - D @ x, scale * np.linalg.norm(x) + np.linalg.norm(p.b))
    assert close(v["u"], dinv * v["r"], dinv.max() * np.linalg.norm(v["r"]))
    assert close(v["w"], D @ v["u"], scale * np.linalg.norm(v["u"]))
    assert close(v["s"], D @ v["p"], scale * np.linalg.norm(v["p"]))


def pin_dense_spd(solve):
    rng = np.random.default_rng(4)
    n = 30
    G = rng.standard_normal((n, n))
    D = G @ G.T + n * np.eye(n)
    A = from_dense(D)
    b = rng.standard_normal(n)
    x, r = solve(A, b, 1e-12, None)
    assert r["status"] == oracle.OK
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def pin_three_eigenvectors(solve):
    m = 20
    p = W.poisson2d(m)
    A = assemble(p)
    t = np.arange(1, m + 1) * p.extra["h"]
    X, Y = np.meshgrid(t, t, indexing="xy")
    b = sum(c * np.sin(j * np.pi * X) * np.sin(k * np.pi * Y)
            for c, (j, k) in zip((1.0, 0.5, 2.0), ((1, 1), (3, 2), (7, 9)))).reshape(-1)
    x, res = solve(A, b, 1e-10, None)
    assert res["status"] == oracle.OK and res["iterations"] == 3


def oracle_solve(A, b, rtol, maxit):
    return oracle.pcg_sr(A, b, rtol=rtol, maxit=maxit)


def oracle_solve_aux(A, b, rtol, maxit):
    return oracle.pcg_sr(A, b, rtol=rtol, maxit=maxit, want_aux=True)


# ------------------------------------------------------------ the oracle

@pytest.mark.parametrize("make", MAKERS)
def test_same_iterates_as_pcg(make):
    pin_same_iterates_as_pcg(oracle_solve, make)


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_iterates_after_k_equal_pcg(k):
    pin_iterates_after_k(oracle_solve, k)


@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_recurrence_invariants(k):
    pin_invariants(oracle_solve_aux, k)


def test_first_direction_is_the_preconditioned_residual():
    p = W.edge_diffusion(14, seed=3)
    A = assemble(p)
    dinv = 1.0 / np.diag(dense(A))
    _, _, v = oracle.pcg_sr(A, p.b, rtol=1e-15, maxit=1, want_aux=True)
    u0 = dinv * p.b
    assert np.allclose(v["p"], u0, rtol=0, atol=1e-14 * np.abs(u0).max())


def test_dense_spd_solve():
    pin_dense_spd(oracle_solve)


def test_finite_termination_three_eigenvectors():
    pin_three_eigenvectors(oracle_solve)


def test_c1_closed_form_one_iteration():
    """C1's b is proportional to the eigenvector sin(pi x) sin(pi y) and the
    diagonal is constant: one iteration (two at most in floating point), and
    x = (2 pi^2 / lambda_11) u with lambda_11 = (8 / h^2) sin^2(pi h / 2)."""
    p = W.poisson2d(64)
    A = assemble(p)
    x, r = oracle.pcg_sr(A, p.b, rtol=1e-8)
    assert r["status"] == oracle.OK and r["iterations"] <= 2
    h = p.extra["h"]
    lam = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    xs = (2 * np.pi ** 2 / lam) * p.extra["u_exact"]
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_error_paths():
    p = W.poisson2d(8)
    A = assemble(p)
    x, r = oracle.pcg_sr(A, np.zeros(p.nrows))
    assert r["status"] == oracle.OK and r["iterations"] == 0 and not np.any(x)
    b = p.b.copy()
    b[3] = np.nan
    x, r = oracle.pcg_sr(A, b)
    assert r["status"] == oracle.ERR_NAN
    rb = np.random.default_rng(9).standard_normal(p.nrows)
    x, r = oracle.pcg_sr(A, rb, rtol=1e-14, maxit=4)
    assert r["status"] == oracle.ERR_MAXIT and r["iterations"] == 4
    x, r = oracle.pcg_sr(A, rb, rtol=1e-14, maxit=0)
    assert r["status"] == oracle.ERR_MAXIT and r["iterations"] == 0
    D = dense(A)
    D[5, 5] = 0.0
    x, r = oracle.pcg_sr(from_dense(D), p.b)
    assert r["status"] == oracle.ERR_NOT_SPD
    E = np.diag([2.0, 1.0, 1.0])
    E[0, 1] = E[1, 0] = 3.0
    x, r = oracle.pcg_sr(from_dense(E), np.array([1.0, -1.0, 0.5]), rtol=1e-12)
    assert r["status"] == oracle.ERR_BREAKDOWN


def test_nonzero_guess():
    p = W.edge_diffusion(10, seed=8)
    A = assemble(p)
    x0 = np.random.default_rng(5).standard_normal(p.nrows)
    x, r = oracle.pcg_sr(A, p.b, rtol=1e-11, x0=x0)
    xs = np.linalg.solve(dense(A), p.b)
    assert r["status"] == oracle.OK
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert r["rnorm0"] == pytest.approx(np.linalg.norm(p.b - dense(A) @ x0), rel=1e-12)


def test_batched_equals_one_at_a_time():
    bt = W.batch(5, seed=12, size_range=(30, 300))
    gi, gj = bt.global_coo()
    N = int(bt.nrows.sum())
    A = oracle.coo_symbolic(N, N, gi, gj)
    oracle.coo_numeric(A, bt.v)
    ro, co = bt.row_off, bt.coo_off
    x, rs = oracle.krylov_batched(A, ro, bt.b, oracle.PCG_SR, rtol=1e-9)
    for s in range(bt.nsys):
        sl = slice(int(co[s]), int(co[s + 1]))
        As = oracle.coo_symbolic(int(bt.nrows[s]), int(bt.nrows[s]), bt.i[sl], bt.j[sl])
        oracle.coo_numeric(As, bt.v[sl])
        xs, r = oracle.pcg_sr(As, bt.b[ro[s]:ro[s + 1]], rtol=1e-9)
        assert x[ro[s]:ro[s + 1]].tobytes() == xs.tobytes()
        assert rs[s]["iterations"] == r["iterations"] and r["status"] == oracle.OK


def test_batched_degenerate_systems():
    """A 2 x 2 SPD block, an empty system, a 1 x 1 system and a b = 0 system:
    2, 0, 1, 0 iterations; x = b / a for the 1 x 1 block; x = 0 for b = 0."""
    blocks = [np.array([[4.0, 1.0], [1.0, 3.0]]), np.zeros((0, 0)), np.array([[2.5]]),
              np.array([[2.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 2.0]])]
    N = sum(B_.shape[0] for B_ in blocks)
    D = np.zeros((N, N))
    off = [0]
    for B_ in blocks:
        o, n = off[-1], B_.shape[0]
        D[o:o + n, o:o + n] = B_
        off.append(o + n)
    A = from_dense(D)
    b = np.array([1.0, 2.0, 5.0, 0.0, 0.0, 0.0])
    x, rs = oracle.krylov_batched(A, np.array(off), b, oracle.PCG_SR, rtol=1e-12)
    assert [r["status"] for r in rs] == [oracle.OK] * 4
    assert [r["iterations"] for r in rs] == [2, 0, 1, 0]
    assert not np.any(x[3:])
    xs = np.linalg.solve(blocks[0], b[:2])
    assert np.linalg.norm(x[:2] - xs) <= 1e-12 * np.linalg.norm(xs) * 10
    assert abs(x[2] - 2.0) <= 4 * np.spacing(2.0)


# ------------------------------------------------------------ planted mistakes

# (description, text in oracle.c's orc_pcg_sr, its mutated replacement)
MUTANTS = [
    ("alpha denominator without the beta term",
     "den = delta - beta * gamma / alpha_prev;", "den = delta;"),
    ("beta inverted", "beta = gamma / gamma_prev;", "beta = gamma_prev / gamma;"),
    ("s updated without beta", "s[i] = w[i] + beta * s[i];", "s[i] = w[i] + s[i];"),
    ("r updated with p instead of s", "r[i] = r[i] - alpha * s[i];",
     "r[i] = r[i] - alpha * p[i];"),
    ("residual norm of u instead of r", "const double rn = sqrt(dot(n, r, r));\n      res->rnorm = rn;\n      if (!isfinite(rn) || !isfinite(gamma) || !isfinite(delta)) {\n        st = ORC_ERR_NAN;\n        break;\n      }\n      if (rn <= rtol * bnorm) break;\n      if (it >= maxit) {\n        st = ORC_ERR_MAXIT;\n        break;\n      }\n      double beta = 0.0, den = delta;",
     "const double rn = sqrt(dot(n, u, u));\n      res->rnorm = rn;\n      if (!isfinite(rn) || !isfinite(gamma) || !isfinite(delta)) {\n        st = ORC_ERR_NAN;\n        break;\n      }\n      if (rn <= rtol * bnorm) break;\n      if (it >= maxit) {\n        st = ORC_ERR_MAXIT;\n        break;\n      }\n      double beta = 0.0, den = delta;"),
]


def _mutant_solver(tmpdir, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    a = src.index("int orc_pcg_sr(")
    e = src.index("\n}\n", a)
    body = src[a:e]
    assert body.count(old) == 1, name
    src = src[:a] + body.replace(old, new) + src[e:]
    c = os.path.join(tmpdir, "mutant.c")
    so = os.path.join(tmpdir, f"libmut{abs(hash(name))}.so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           c, "-o", so, "-lm"])
    lib = ctypes.CDLL(so)
    P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.orc_pcg_sr.restype = ctypes.c_int
    lib.orc_pcg_sr.argtypes = [I64, P, P, P, P, P, D, I64, ctypes.c_int, P, P]
    pp = lambda a_: a_.ctypes.data_as(ctypes.c_void_p)

    def solve_aux(A, b, rtol, maxit):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(A.nrows)
        res = oracle._Result()
        aux = np.zeros(5 * max(A.nrows, 1))
        mi = oracle.default_maxit(A.nrows) if maxit is None else maxit
        lib.orc_pcg_sr(A.nrows, pp(A.row_ptr), pp(A.col), pp(A.val), pp(b), pp(x), rtol, mi, 0,
                       ctypes.byref(res), pp(aux))
        n = A.nrows
        return x, res.as_dict(), {k: aux[i * n:(i + 1) * n].copy()
                                  for i, k in enumerate(("r", "u", "w", "p", "s"))}

    return (lambda A, b, rtol, maxit: solve_aux(A, b, rtol, maxit)[:2]), solve_aux


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_fail_a_pin(name, old, new):
    with tempfile.TemporaryDirectory() as d:
        solve, solve_aux = _mutant_solver(d, name, old, new)
        checks = [lambda: pin_iterates_after_k(solve, 5), lambda: pin_invariants(solve_aux, 5),
                  lambda: pin_dense_spd(solve), lambda: pin_three_eigenvectors(solve),
                  lambda: pin_same_iterates_as_pcg(solve, MAKERS[0])]
        failed = 0
        for chk in checks:
            try:
                chk()
            except AssertionError:
                failed += 1
        assert failed >= 1, f"mutant '{name}' passed every pin"
