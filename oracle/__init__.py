"""FP64 CPU oracle for the sparse SPD solver path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module compiles it on first use with gcc and wraps it with ctypes and
numpy.  Each wrapper names the paper passage its C function follows.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(dense brute force, closed forms, finite differences, invariants).
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_lib_omp = None

OK, ERR_ARG, ERR_INDEX, ERR_ALLOC = 0, 1, 2, 3
ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NAN, ERR_MAXIT, ERR_STAGNATION = 5, 6, 7, 8, 9
INSERT, ADD = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, FP64, no FMA), and
    the same source with OpenMP into liboracle_omp.so (the all-cores
    baseline; same results: see ORC_PAR in oracle.c)."""
    lock_path = _LIB_PATH + ".lock"
    with open(lock_path, "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        for path, extra in ((_LIB_PATH, []), (_LIB_OMP_PATH, ["-fopenmp"])):
            stale = (not os.path.exists(path)
                     or os.path.getmtime(path) < os.path.getmtime(_SRC))
            if force or stale:
                tmp = path + f".tmp{os.getpid()}"
                subprocess.check_call([
                    "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                    *extra, "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
                os.replace(tmp, path)
    return _LIB_PATH


def threads() -> int:
    """Host cores this process may run on (the all-cores build uses them all)."""
    return len(os.sched_getaffinity(0))


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rnorm0", ctypes.c_double), ("rnorm", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


def _load(omp: bool = False):
    """The one-thread oracle, or with omp the all-cores build of the same source."""
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            build()
            _lib_omp = _signatures(ctypes.CDLL(_LIB_OMP_PATH))
        return _lib_omp
    if _lib is None:
        build()
        _lib = _signatures(ctypes.CDLL(_LIB_PATH))
    return _lib


def _signatures(lib):
    if True:
        P = ctypes.c_void_p
        I64, I32, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.orc_coo_symbolic.restype = I64
        lib.orc_coo_symbolic.argtypes = [I64, I64, I64, P, P, P, P, P, P, P]
        lib.orc_coo_numeric.restype = None
        lib.orc_coo_numeric.argtypes = [I64, P, P, P, ctypes.c_int, P]
        lib.orc_coo_scatter.restype = None
        lib.orc_coo_scatter.argtypes = [I64, I64, P, P, P, P]
        lib.orc_bicg.restype = ctypes.c_int
        lib.orc_bicg.argtypes = [I64, P, P, P, P, P, D, I64, ctypes.c_int, P]
        lib.orc_tfqmr.restype = ctypes.c_int
        lib.orc_tfqmr.argtypes = [I64, P, P, P, P, P, D, I64, ctypes.c_int, P]
        lib.orc_pipecg.restype = ctypes.c_int
        lib.orc_pipecg.argtypes = [I64, P, P, P, P, P, D, I64, ctypes.c_int, P, P]
        lib.orc_pcg_sr.restype = ctypes.c_int
        lib.orc_pcg_sr.argtypes = [I64, P, P, P, P, P, D, I64, ctypes.c_int, P, P]
        lib.orc_krylov_batched.restype = ctypes.c_int
        lib.orc_krylov_batched.argtypes = [I32, P, P, P, P, P, P, D, I64, ctypes.c_int, P]
        lib.orc_vec_set_values_coo.restype = I64
        lib.orc_vec_set_values_coo.argtypes = [I64, I64, P, P, ctypes.c_int, P]
        lib.orc_spmv.restype = None
        lib.orc_spmv.argtypes = [I64, P, P, P, P, P]
        lib.orc_pcg.restype = ctypes.c_int
        lib.orc_pcg.argtypes = [I64, P, P, P, P, P, D, I64, ctypes.c_int, P]
        lib.orc_pcg_refined.restype = ctypes.c_int
        lib.orc_pcg_refined.argtypes = [I64, P, P, P, P, P, D, D, I64, I32,
                                        ctypes.c_int, P, P]
        lib.orc_csr_is_symmetric.restype = ctypes.c_int
        lib.orc_csr_is_symmetric.argtypes = [I64, P, P, P]
        lib.orc_adjoint.restype = ctypes.c_int
        lib.orc_adjoint.argtypes = [I64, P, P, P, P, P, P, P, D, I64, P]
        lib.orc_pcg_batched.restype = ctypes.c_int
        lib.orc_pcg_batched.argtypes = [I32, P, P, P, P, P, P, D, I64,
                                        ctypes.c_int, D, I64, I32, P]
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


@dataclass
class CSR:
    """CSR structure plus the COO maps of the symbolic stage."""
    nrows: int
    ncols: int
    row_ptr: np.ndarray  # int32[nrows+1]
    col: np.ndarray      # int32[nnz]
    perm: np.ndarray     # int32[nkept]   sorted position -> original COO index
    jmap: np.ndarray     # int32[nnz+1]   segment offsets into perm
    ncoo: int
    val: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def nkept(self) -> int:
        return int(self.perm.shape[0])


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


def default_maxit(n: int) -> int:
    """maxit default when unset: 10 n, capped at 100,000 (a reading; the paper is silent)."""
    return int(min(10 * max(n, 1), 100_000))


def coo_symbolic(nrows: int, ncols: int, i, j) -> CSR:
    """Sec. 5 preallocation: pattern of the kept COO entries (negatives ignored)."""
    lib = _load()
    i = _c(i, np.int32)
    j = _c(j, np.int32)
    ncoo = int(i.shape[0])
    assert j.shape[0] == ncoo
    row_ptr = np.zeros(nrows + 1, np.int32)
    col = np.zeros(max(ncoo, 1), np.int32)
    perm = np.zeros(max(ncoo, 1), np.int32)
    jmap = np.zeros(ncoo + 1, np.int32)
    nkept = ctypes.c_int64(0)
    nnz = lib.orc_coo_symbolic(nrows, ncols, ncoo, _p(i), _p(j), _p(row_ptr), _p(col),
                               _p(perm), _p(jmap), ctypes.byref(nkept))
    if nnz < 0:
        raise OracleError(int(-nnz), "coo_symbolic")
    return CSR(nrows, ncols, row_ptr, col[:nnz].copy(), perm[:nkept.value].copy(),
               jmap[:nnz + 1].copy(), ncoo)


def coo_numeric(A: CSR, v, mode: int = INSERT, omp: bool = False) -> np.ndarray:
    """Sec. 5 MatSetValuesCOO: in-order duplicate sum; INSERT replaces, ADD adds.
    omp: the all-cores build (same results)."""
    lib = _load(omp)
    v = _c(v, np.float64)
    assert v.shape[0] == A.ncoo
    if A.val is None or mode == INSERT:
        val = np.zeros(A.nnz, np.float64) if A.val is None else A.val.copy()
    else:
        val = A.val.copy()
    lib.orc_coo_numeric(A.nnz, _p(A.jmap), _p(A.perm), _p(v), mode, _p(val))
    A.val = val
    return val


def coo_scatter(A: CSR, dlda) -> np.ndarray:
    """Transpose of the numeric stage: dL/dv_k = dL/da_{p(k)}, 0 for ignored k."""
    lib = _load()
    dlda = _c(dlda, np.float64)
    out = np.zeros(A.ncoo, np.float64)
    lib.orc_coo_scatter(A.nnz, A.ncoo, _p(A.jmap), _p(A.perm), _p(dlda), _p(out))
    return out


BICG, TFQMR, PIPECG, PCG_SR = 1, 2, 3, 4


def _nonsym(fn, A: CSR, b, rtol, maxit, x0):
    lib = _load()
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64) if x0 is None else _c(x0, np.float64).copy()
    res = _Result()
    maxit = default_maxit(A.nrows) if maxit is None else maxit
    getattr(lib, fn)(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x), rtol,
                     maxit, 0 if x0 is None else 1, ctypes.byref(res))
    return x, res.as_dict()


def bicg(A: CSR, b, rtol: float = 1e-8, maxit: int | None = None, x0=None):
    """BiCG with the diagonal preconditioner (Sec. 7 batched solvers), rt_0 = r_0."""
    return _nonsym("orc_bicg", A, b, rtol, maxit, x0)


def tfqmr(A: CSR, b, rtol: float = 1e-8, maxit: int | None = None, x0=None):
    """TFQMR, right-preconditioned with the diagonal (Sec. 7 batched solvers)."""
    return _nonsym("orc_tfqmr", A, b, rtol, maxit, x0)


def pipecg(A: CSR, b, rtol: float = 1e-8, maxit: int | None = None, x0=None,
           want_aux: bool = False):
    """Pipelined Jacobi-PCG (one reduction per iteration; Ghysels-Vanroose).
    With want_aux, also returns the final r, u, w, p, s, q, z (dict)."""
    lib = _load()
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64) if x0 is None else _c(x0, np.float64).copy()
    res = _Result()
    maxit = default_maxit(A.nrows) if maxit is None else maxit
    aux = np.zeros(7 * A.nrows, np.float64) if want_aux else None
    lib.orc_pipecg(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x), rtol, maxit,
                   0 if x0 is None else 1, ctypes.byref(res),
                   _p(aux) if want_aux else None)
    if not want_aux:
        return x, res.as_dict()
    n = A.nrows
    names = ("r", "u", "w", "p", "s", "q", "z")
    return x, res.as_dict(), {k: aux[i * n:(i + 1) * n].copy() for i, k in enumerate(names)}


def pcg_sr(A: CSR, b, rtol: float = 1e-8, maxit: int | None = None, x0=None,
           want_aux: bool = False):
    """Jacobi-PCG in Chronopoulos and Gear's single-reduction form (one
    reduction per iteration, taken after the product w = A u; PCG's iterates
    in exact arithmetic).  With want_aux, also returns the final r, u, w, p,
    s (dict)."""
    lib = _load()
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64) if x0 is None else _c(x0, np.float64).copy()
    res = _Result()
    maxit = default_maxit(A.nrows) if maxit is None else maxit
    aux = np.zeros(5 * A.nrows, np.float64) if want_aux else None
    lib.orc_pcg_sr(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x), rtol, maxit,
                   0 if x0 is None else 1, ctypes.byref(res),
                   _p(aux) if want_aux else None)
    if not want_aux:
        return x, res.as_dict()
    n = A.nrows
    names = ("r", "u", "w", "p", "s")
    return x, res.as_dict(), {k: aux[i * n:(i + 1) * n].copy() for i, k in enumerate(names)}


def krylov_batched(A: CSR, row_off, b, method: int, rtol: float = 1e-8,
                   maxit: int | None = None):
    """Batched BiCG (method 1), TFQMR (method 2), pipelined CG (method 3) or
    single-reduction CG (method 4): each diagonal block alone."""
    lib = _load()
    row_off = _c(row_off, np.int64)
    nsys = int(row_off.shape[0] - 1)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64)
    res = (_Result * max(nsys, 1))()
    mx = int(np.diff(row_off).max()) if nsys else 1
    maxit = default_maxit(mx) if maxit is None else maxit
    lib.orc_krylov_batched(nsys, _p(row_off), _p(A.row_ptr), _p(A.col), _p(A.val), _p(b),
                           _p(x), rtol, maxit, method, ctypes.cast(res, ctypes.c_void_p))
    return x, [res[s].as_dict() for s in range(nsys)]


def vec_set_values_coo(n: int, i, v, mode: int = INSERT, y=None) -> np.ndarray:
    """Sec. 5 COO interface for vectors: y_r = in-order sum of v[k] with
    i[k] = r (INSERT), or y_r + that sum (ADD); other entries of y unchanged."""
    lib = _load()
    i = _c(i, np.int32)
    v = _c(v, np.float64)
    assert v.shape[0] == i.shape[0]
    y = np.zeros(n, np.float64) if y is None else _c(y, np.float64).copy()
    st = lib.orc_vec_set_values_coo(n, i.shape[0], _p(i), _p(v), mode, _p(y))
    if st < 0:
        raise OracleError(int(-st), "vec_set_values_coo")
    return y


def spmv(A: CSR, x, omp: bool = False) -> np.ndarray:
    """MatMult (Sec. 6.1): y_i = sum_p a_p x_{col p}, CSR order, FP64.
    omp: the all-cores build (same results)."""
    lib = _load(omp)
    x = _c(x, np.float64)
    y = np.zeros(A.nrows, np.float64)
    lib.orc_spmv(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(x), _p(y))
    return y


def pcg(A: CSR, b, rtol: float = 1e-8, maxit: int | None = None, x0=None,
        omp: bool = False):
    """Jacobi-PCG (Sec. 6.1 CG, Sec. 7 diagonal preconditioning). Returns (x, result).
    omp: the all-cores build (same results)."""
    lib = _load(omp)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64) if x0 is None else _c(x0, np.float64).copy()
    res = _Result()
    maxit = default_maxit(A.nrows) if maxit is None else maxit
    lib.orc_pcg(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x), rtol,
                maxit, 0 if x0 is None else 1, ctypes.byref(res))
    return x, res.as_dict()


def pcg_refined(A: CSR, b, rtol: float = 1e-8, inner_rtol: float = 1e-4,
                inner_maxit: int | None = None, max_outer: int = 30, x0=None,
                want_trace: bool = False):
    """FP32-inner PCG inside FP64 iterative refinement (Sec. 2, multiprecision).
    With want_trace, also returns each outer step's inner iteration count."""
    lib = _load()
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64) if x0 is None else _c(x0, np.float64).copy()
    res = _Result()
    inner_maxit = default_maxit(A.nrows) if inner_maxit is None else inner_maxit
    trace = np.zeros(max(max_outer, 1), np.int32)
    lib.orc_pcg_refined(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x),
                        rtol, inner_rtol, inner_maxit, max_outer,
                        0 if x0 is None else 1, ctypes.byref(res), _p(trace))
    if not want_trace:
        return x, res.as_dict()
    r = res.as_dict()
    return x, r, [int(v) for v in trace[:r["outer_iterations"]]]


def is_symmetric(A: CSR) -> bool:
    lib = _load()
    return bool(lib.orc_csr_is_symmetric(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val)))


def adjoint(A: CSR, x, g, rtol: float = 1e-10, maxit: int | None = None):
    """Linear-solve adjoint (Sec. 1 adjoint capability): lambda = A^-T g,
    dL/da_p = -lambda_row x_col, dL/dv by the COO scatter.  Returns
    (lambda, dlda, dldv, result)."""
    lib = _load()
    x = _c(x, np.float64)
    g = _c(g, np.float64)
    lam = np.zeros(A.nrows, np.float64)
    dlda = np.zeros(A.nnz, np.float64)
    res = _Result()
    maxit = default_maxit(A.nrows) if maxit is None else maxit
    lib.orc_adjoint(A.nrows, _p(A.row_ptr), _p(A.col), _p(A.val), _p(x), _p(g), _p(lam),
                    _p(dlda), rtol, maxit, ctypes.byref(res))
    dldv = coo_scatter(A, dlda)
    return lam, dlda, dldv, res.as_dict()


def pcg_batched(A: CSR, row_off, b, rtol: float = 1e-8, maxit: int | None = None,
                precision: int = 0, inner_rtol: float = 1e-4,
                inner_maxit: int | None = None, max_outer: int = 30):
    """Sec. 7 batched solve: each diagonal block solved on its own.
    Returns (x, list of per-system results)."""
    lib = _load()
    row_off = _c(row_off, np.int64)
    nsys = int(row_off.shape[0] - 1)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows, np.float64)
    res = (_Result * max(nsys, 1))()
    sizes = np.diff(row_off)
    mx = int(sizes.max()) if nsys else 1
    maxit = default_maxit(mx) if maxit is None else maxit
    inner_maxit = default_maxit(mx) if inner_maxit is None else inner_maxit
    lib.orc_pcg_batched(nsys, _p(row_off), _p(A.row_ptr), _p(A.col), _p(A.val), _p(b),
                        _p(x), rtol, maxit, precision, inner_rtol, inner_maxit,
                        max_outer, ctypes.cast(res, ctypes.c_void_p))
    return x, [res[s].as_dict() for s in range(nsys)]
