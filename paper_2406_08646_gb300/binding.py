"""Thin ctypes binding of libgbs.so (C-ABI in include/gbs.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Tensors supply device memory; the stream is torch's current stream
unless one is given.  The functions keep the C names (mat_create_coo,
mat_set_values_coo, mat_mult, ksp_solve_cg, ksp_adjoint, ...); :class:`Mat` is
a small convenience wrapper over them.

Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbs.so")

OK, ERR_ARG, ERR_INDEX, ERR_ALLOC, ERR_CUDA = 0, 1, 2, 3, 4
ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NAN, ERR_MAXIT = 5, 6, 7, 8
ERR_STAGNATION, ERR_TIMEOUT, ERR_LAUNCH = 9, 10, 11
INSERT, ADD = 0, 1
FP64, FP32_REFINED = 0, 1
SPMV_AUTO, SPMV_SELL = -1, 0  # plan kernels; 1, 2, 4, 8, 32 = CSR-vector lanes per row
SOLVER_AUTO, SOLVER_PHASES, SOLVER_CTA, SOLVER_SPLIT = 0, 1, 2, 3
KSP_CG, KSP_BICG, KSP_TFQMR, KSP_PIPECG, KSP_CGSR = 0, 1, 2, 3, 4
CG_TEXTBOOK, CG_SINGLE_REDUCTION, CG_SINGLE_KERNEL = 0, 1, 2

EXPORTED = ["ksp_opts_default", "mat_create_coo", "mat_create_coo_batched",
            "mat_set_values_coo", "mat_mult", "ksp_solve_cg", "ksp_solve_cg_batched",
            "ksp_adjoint", "ksp_adjoint_batched", "ksp_get_result", "mat_get_info",
            "mat_get_csr", "mat_get_coo_maps", "mat_set_plan", "mat_get_plan",
            "mat_autotune", "mat_destroy", "gbs_launch_count", "gbs_last_error",
            "ksp_solve_cg_noalloc", "ksp_get_phase_ns", "mat_set_solver",
            "vec_create_coo", "vec_set_values_coo", "vec_get_info", "vec_destroy",
            "ksp_solve", "ksp_solve_batched", "q1_hex_element_coo", "q1_hex_element_values",
            "edge_coo_values", "mat_autotune_file", "mat_set_cg_form", "mat_get_tuning",
            "mat_set_split_rows", "mat_set_slice_patterns", "mat_get_slices"]


class KspOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("inner_rtol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("inner_maxit", ctypes.c_int32),
                ("timeout_ns", ctypes.c_int64), ("nonzero_guess", ctypes.c_int32),
                ("host_loop", ctypes.c_int32), ("method", ctypes.c_int32)]


class KspResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("outer_iterations", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("rnorm0", ctypes.c_double), ("rnorm", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class GbsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libgbs status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libgbs.so (built by __graft_entry__.build() or _build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "ksp_opts_default": (None, [P]),
        "mat_create_coo": (ctypes.c_int, [I64, I64, I64, P, P, P, PP]),
        "mat_create_coo_batched": (ctypes.c_int, [I32, P, P, P, P, P, PP]),
        "mat_set_values_coo": (ctypes.c_int, [P, P, ctypes.c_int, P]),
        "mat_mult": (ctypes.c_int, [P, P, P, P]),
        "ksp_solve_cg": (ctypes.c_int, [P, P, P, P, P, P]),
        "ksp_solve_cg_batched": (ctypes.c_int, [P, P, P, P, P, P]),
        "ksp_solve": (ctypes.c_int, [P, P, P, P, P, P]),
        "ksp_solve_batched": (ctypes.c_int, [P, P, P, P, P, P]),
        "ksp_adjoint": (ctypes.c_int, [P, P, P, P, P, P, P, P, P]),
        "ksp_adjoint_batched": (ctypes.c_int, [P, P, P, P, P, P, P, P, P]),
        "ksp_get_result": (ctypes.c_int, [P, P, I32, P]),
        "mat_get_info": (ctypes.c_int, [P, P, P, P, P, P]),
        "mat_get_csr": (ctypes.c_int, [P, PP, PP, PP, P]),
        "mat_get_coo_maps": (ctypes.c_int, [P, PP, PP, P]),
        "mat_set_plan": (ctypes.c_int, [P, I32, I32, I32, I32]),
        "mat_get_plan": (ctypes.c_int, [P, P, P, P, P, P]),
        "mat_autotune": (ctypes.c_int, [P, P]),
        "mat_destroy": (ctypes.c_int, [P]),
        "gbs_launch_count": (I64, []),
        "gbs_last_error": (ctypes.c_char_p, []),
        "ksp_solve_cg_noalloc": (ctypes.c_int, [I64, P, P, P, P, P, P, P, P]),
        "ksp_get_phase_ns": (ctypes.c_int, [P, P, P]),
        "mat_set_solver": (ctypes.c_int, [P, I32]),
        "vec_create_coo": (ctypes.c_int, [I64, I64, P, P, PP]),
        "vec_set_values_coo": (ctypes.c_int, [P, P, ctypes.c_int, P, P]),
        "vec_get_info": (ctypes.c_int, [P, P, P, P]),
        "vec_destroy": (ctypes.c_int, [P]),
        "q1_hex_element_coo": (ctypes.c_int, [I32, P, P, P]),
        "q1_hex_element_values": (ctypes.c_int, [I32, P, P, P]),
        "edge_coo_values": (ctypes.c_int, [I64, P, P, P]),
        "mat_autotune_file": (ctypes.c_int, [P, ctypes.c_char_p, P, P]),
        "mat_set_cg_form": (ctypes.c_int, [P, I32]),
        "mat_get_tuning": (ctypes.c_int, [P, P, P, P]),
        "mat_set_split_rows": (ctypes.c_int, [P, I64]),
        "mat_set_slice_patterns": (ctypes.c_int, [P, I32]),
        "mat_get_slices": (ctypes.c_int, [P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return lib().gbs_last_error().decode()


def launch_count() -> int:
    return int(lib().gbs_launch_count())


def _check(status: int):
    if status != OK:
        raise GbsError(status, last_error())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t: torch.Tensor | None, dtype, n: int | None = None, name: str = "tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def make_opts(rtol=1e-8, maxit=-1, precision=FP64, inner_rtol=1e-4, max_outer=30,
              inner_maxit=-1, timeout_ns=0, nonzero_guess=False,
              host_loop=False, method=KSP_CG) -> KspOpts:
    o = KspOpts()
    lib().ksp_opts_default(ctypes.byref(o))
    o.rtol, o.maxit, o.precision = float(rtol), int(maxit), int(precision)
    o.inner_rtol, o.max_outer, o.inner_maxit = float(inner_rtol), int(max_outer), int(inner_maxit)
    o.timeout_ns, o.nonzero_guess = int(timeout_ns), int(bool(nonzero_guess))
    o.host_loop = int(bool(host_loop))
    o.method = int(method)
    return o


# --------------------------------------------------------------- C-named calls

def mat_create_coo(nrows: int, ncols: int, i: torch.Tensor, j: torch.Tensor, stream=None):
    n = i.numel()
    h = ctypes.c_void_p()
    _check(lib().mat_create_coo(nrows, ncols, n, _dev(i, torch.int32, None, "i"),
                                _dev(j, torch.int32, n, "j"), _stream(stream), ctypes.byref(h)))
    return h


def mat_create_coo_batched(nrows, ncoo, i: torch.Tensor, j: torch.Tensor, stream=None):
    import numpy as np
    nr = np.ascontiguousarray(nrows, dtype=np.int64)
    nc = np.ascontiguousarray(ncoo, dtype=np.int64)
    if nr.shape != nc.shape:
        raise ValueError("nrows and ncoo must have one entry per system")
    h = ctypes.c_void_p()
    tot = int(nc.sum())
    _check(lib().mat_create_coo_batched(int(nr.shape[0]), nr.ctypes.data_as(ctypes.c_void_p),
                                        nc.ctypes.data_as(ctypes.c_void_p),
                                        _dev(i, torch.int32, tot, "i"),
                                        _dev(j, torch.int32, tot, "j"), _stream(stream),
                                        ctypes.byref(h)))
    return h


def mat_set_values_coo(A, v: torch.Tensor, mode: int = INSERT, stream=None):
    _check(lib().mat_set_values_coo(A, _dev(v, torch.float64, None, "v"), mode, _stream(stream)))


def mat_mult(A, x: torch.Tensor, y: torch.Tensor, stream=None):
    _check(lib().mat_mult(A, _dev(x, torch.float64, None, "x"), _dev(y, torch.float64, None, "y"),
                          _stream(stream)))


def ksp_solve_cg(A, b, x, opts: KspOpts | None = None, want_result=True, stream=None):
    res = KspResult()
    st = lib().ksp_solve_cg(A, _dev(b, torch.float64, None, "b"), _dev(x, torch.float64, None, "x"),
                            ctypes.byref(opts) if opts is not None else None,
                            ctypes.byref(res) if want_result else None, _stream(stream))
    return _solve_status(st, [res] if want_result else None)


def ksp_solve_cg_batched(A, b, x, nsys: int, opts: KspOpts | None = None, want_result=True,
                         stream=None):
    res = (KspResult * nsys)()
    st = lib().ksp_solve_cg_batched(A, _dev(b, torch.float64, None, "b"),
                                    _dev(x, torch.float64, None, "x"),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.cast(res, ctypes.c_void_p) if want_result else None,
                                    _stream(stream))
    return _solve_status(st, list(res) if want_result else None)


def ksp_solve(A, b, x, opts: KspOpts | None = None, want_result=True, stream=None):
    res = KspResult()
    st = lib().ksp_solve(A, _dev(b, torch.float64, None, "b"), _dev(x, torch.float64, None, "x"),
                         ctypes.byref(opts) if opts is not None else None,
                         ctypes.byref(res) if want_result else None, _stream(stream))
    return _solve_status(st, [res] if want_result else None)


def ksp_solve_batched(A, b, x, nsys: int, opts: KspOpts | None = None, want_result=True,
                      stream=None):
    res = (KspResult * nsys)()
    st = lib().ksp_solve_batched(A, _dev(b, torch.float64, None, "b"),
                                 _dev(x, torch.float64, None, "x"),
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.cast(res, ctypes.c_void_p) if want_result else None,
                                 _stream(stream))
    return _solve_status(st, list(res) if want_result else None)


def ksp_adjoint(A, x, dldx, lam, dlda=None, dldv=None, opts: KspOpts | None = None,
                want_result=True, stream=None, nsys: int | None = None):
    batched = nsys is not None
    res = (KspResult * (nsys if batched else 1))()
    fn = lib().ksp_adjoint_batched if batched else lib().ksp_adjoint
    st = fn(A, _dev(x, torch.float64, None, "x"), _dev(dldx, torch.float64, None, "dLdx"),
            _dev(lam, torch.float64, None, "lambda"), _dev(dlda, torch.float64, None, "dLda"),
            _dev(dldv, torch.float64, None, "dLdv"),
            ctypes.byref(opts) if opts is not None else None,
            ctypes.cast(res, ctypes.c_void_p) if want_result else None, _stream(stream))
    return _solve_status(st, list(res) if want_result else None)


def _solve_status(st, res):
    """Solver statuses (MAXIT, BREAKDOWN, ...) come back in the results; only
    argument / CUDA failures raise."""
    if res is None:
        _check(st)
        return None
    out = [r.as_dict() for r in res]
    if st in (ERR_ARG, ERR_ALLOC, ERR_CUDA, ERR_LAUNCH):
        raise GbsError(st, last_error())
    return out


def ksp_get_result(A, count: int = 1, stream=None):
    res = (KspResult * count)()
    lib().ksp_get_result(A, ctypes.cast(res, ctypes.c_void_p), count, _stream(stream))
    return [r.as_dict() for r in res]


def ksp_get_phase_ns(A, stream=None) -> dict:
    """Per-phase time (ns) of the last solve, summed over iterations (each
    phase from its kernel's start to the next phase kernel's start)."""
    arr = (ctypes.c_int64 * 5)()
    _check(lib().ksp_get_phase_ns(A, ctypes.cast(arr, ctypes.c_void_p), _stream(stream)))
    return dict(zip(["setup", "spmv", "update_xr", "update_p", "true_residual"], list(arr)))


def mat_get_info(A) -> dict:
    nr, nc, nnz, ncoo = (ctypes.c_int64() for _ in range(4))
    nsys = ctypes.c_int32()
    _check(lib().mat_get_info(A, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz),
                              ctypes.byref(ncoo), ctypes.byref(nsys)))
    return {"nrows": nr.value, "ncols": nc.value, "nnz": nnz.value, "ncoo": ncoo.value,
            "nsys": nsys.value}


class _CudaArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3,
                                         "strides": None}


def _view(ptr, n, dtype):
    typestr = {torch.int32: "<i4", torch.float64: "<f8"}[dtype]
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaArray(int(ptr), int(n), typestr), device="cuda")


def mat_get_csr(A):
    """Borrowed device views (row_ptr, col, val) of the CSR arrays."""
    info = mat_get_info(A)
    rp, col, val = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    nnz = ctypes.c_int64()
    _check(lib().mat_get_csr(A, ctypes.byref(rp), ctypes.byref(col), ctypes.byref(val),
                             ctypes.byref(nnz)))
    return (_view(rp.value, info["nrows"] + 1, torch.int32),
            _view(col.value, nnz.value, torch.int32), _view(val.value, nnz.value, torch.float64))


def mat_get_coo_maps(A):
    """Borrowed device views (perm, jmap)."""
    info = mat_get_info(A)
    perm, jmap = ctypes.c_void_p(), ctypes.c_void_p()
    nkept = ctypes.c_int64()
    _check(lib().mat_get_coo_maps(A, ctypes.byref(perm), ctypes.byref(jmap), ctypes.byref(nkept)))
    return (_view(perm.value, nkept.value, torch.int32),
            _view(jmap.value, info["nnz"] + 1, torch.int32))


def mat_set_plan(A, spmv_rows: int, update_rows: int, kernel: int = SPMV_AUTO,
                 ctas_per_sm: int = 0):
    _check(lib().mat_set_plan(A, spmv_rows, update_rows, kernel, ctas_per_sm))


def mat_get_plan(A) -> dict:
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().mat_get_plan(A, *[ctypes.byref(t) for t in v]))
    return dict(zip(["spmv_rows", "update_rows", "kernel", "ctas_per_sm", "spmv_grid"],
                    [t.value for t in v]))


def mat_set_solver(A, solver: int):
    _check(lib().mat_set_solver(A, solver))


def mat_autotune_file(A, path: str, stream=None) -> bool:
    """Tune A, or apply the tuning stored for its key in the file at path;
    returns True when it came from the file."""
    hit = ctypes.c_int32(0)
    _check(lib().mat_autotune_file(A, os.fsencode(path), ctypes.byref(hit), _stream(stream)))
    return bool(hit.value)


def mat_set_cg_form(A, form: int):
    _check(lib().mat_set_cg_form(A, int(form)))


def mat_get_tuning(A) -> dict:
    sv, cf, sr = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    _check(lib().mat_get_tuning(A, ctypes.byref(sv), ctypes.byref(cf), ctypes.byref(sr)))
    return {"solver": sv.value, "cg_form": cf.value, "split_rows": sr.value}


def mat_set_split_rows(A, min_rows: int):
    _check(lib().mat_set_split_rows(A, int(min_rows)))


def mat_set_slice_patterns(A, on: bool):
    _check(lib().mat_set_slice_patterns(A, 1 if on else 0))


def mat_get_slices(A) -> dict:
    v = [ctypes.c_int64(0) for _ in range(3)]
    _check(lib().mat_get_slices(A, *[ctypes.byref(t) for t in v]))
    return dict(zip(["nslices", "pattern_slices", "entries"], [t.value for t in v]))


def mat_autotune(A, stream=None):
    _check(lib().mat_autotune(A, _stream(stream)))


def mat_destroy(A):
    if A:
        lib().mat_destroy(A)


def vec_create_coo(n: int, i: torch.Tensor, stream=None):
    h = ctypes.c_void_p()
    _check(lib().vec_create_coo(n, i.numel(), _dev(i, torch.int32, None, "i"), _stream(stream),
                                ctypes.byref(h)))
    return h


def vec_set_values_coo(V, v: torch.Tensor, y: torch.Tensor, mode: int = INSERT, stream=None):
    _check(lib().vec_set_values_coo(V, _dev(v, torch.float64, None, "v"), mode,
                                    _dev(y, torch.float64, None, "y"), _stream(stream)))


def q1_hex_element_coo(ne: int, i: torch.Tensor, j: torch.Tensor, stream=None):
    """COO indices of the ne^3 Q1 element blocks (int32[64 ne^3] each)."""
    n = 64 * ne ** 3
    _check(lib().q1_hex_element_coo(int(ne), _dev(i, torch.int32, n, "i"),
                                    _dev(j, torch.int32, n, "j"), _stream(stream)))


def q1_hex_element_values(ne: int, kappa: torch.Tensor, v: torch.Tensor, stream=None):
    """COO values (kappa_e h) K_ref of the ne^3 Q1 element blocks with the
    Dirichlet edits (float64[64 ne^3]) from kappa (float64[ne^3])."""
    _check(lib().q1_hex_element_values(int(ne), _dev(kappa, torch.float64, ne ** 3, "kappa"),
                                       _dev(v, torch.float64, 64 * ne ** 3, "v"),
                                       _stream(stream)))


def edge_coo_values(kappa: torch.Tensor, v: torch.Tensor, stream=None):
    """COO values (+k, +k, -k, -k) of every edge (float64[4 nedges])."""
    m = kappa.numel()
    _check(lib().edge_coo_values(m, _dev(kappa, torch.float64, m, "kappa"),
                                 _dev(v, torch.float64, 4 * m, "v"), _stream(stream)))


def vec_get_info(V) -> dict:
    n, ne, nc = (ctypes.c_int64() for _ in range(3))
    _check(lib().vec_get_info(V, ctypes.byref(n), ctypes.byref(ne), ctypes.byref(nc)))
    return {"n": n.value, "nentries": ne.value, "ncoo": nc.value}


class Vec:
    """Owning wrapper of a gbs_vec handle (vector COO assembly)."""

    def __init__(self, n, i, stream=None):
        self.h = vec_create_coo(n, i, stream)
        self.info = vec_get_info(self.h)

    def set_values(self, v, y=None, mode=INSERT, stream=None):
        if y is None:
            y = torch.zeros(self.info["n"], dtype=torch.float64, device=v.device)
        vec_set_values_coo(self.h, v, y, mode, stream)
        return y

    def close(self):
        if self.h:
            lib().vec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- wrapper

class Mat:
    """Owning wrapper of a gbs_mat handle."""

    def __init__(self, handle, batched_rows=None):
        self.h = handle
        self.info = mat_get_info(handle)
        self.batched_rows = batched_rows

    @classmethod
    def from_coo(cls, nrows, ncols, i, j, stream=None) -> "Mat":
        return cls(mat_create_coo(nrows, ncols, i, j, stream))

    @classmethod
    def from_coo_batched(cls, nrows, ncoo, i, j, stream=None) -> "Mat":
        return cls(mat_create_coo_batched(nrows, ncoo, i, j, stream), list(nrows))

    @property
    def nrows(self) -> int:
        return self.info["nrows"]

    @property
    def nnz(self) -> int:
        return self.info["nnz"]

    @property
    def nsys(self) -> int:
        return self.info["nsys"]

    def set_values(self, v, mode=INSERT, stream=None):
        mat_set_values_coo(self.h, v, mode, stream)

    def mult(self, x, y=None, stream=None):
        if y is None:
            y = torch.empty(self.nrows, dtype=torch.float64, device=x.device)
        mat_mult(self.h, x, y, stream)
        return y

    def solve(self, b, x=None, stream=None, want_result=True, **kw):
        if x is None:
            x = torch.empty_like(b)
        r = ksp_solve(self.h, b, x, make_opts(**kw), want_result, stream)
        return x, (r[0] if r else None)

    def solve_batched(self, b, x=None, stream=None, want_result=True, **kw):
        if x is None:
            x = torch.empty_like(b)
        r = ksp_solve_batched(self.h, b, x, self.nsys, make_opts(**kw), want_result, stream)
        return x, r

    def adjoint(self, x, dldx, dlda=True, dldv=True, stream=None, want_result=True,
                batched=False, **kw):
        lam = torch.empty_like(dldx)
        ga = torch.empty(self.nnz, dtype=torch.float64, device=x.device) if dlda else None
        gv = torch.empty(self.info["ncoo"], dtype=torch.float64, device=x.device) if dldv else None
        r = ksp_adjoint(self.h, x, dldx, lam, ga, gv, make_opts(**kw), want_result, stream,
                        nsys=self.nsys if batched else None)
        return lam, ga, gv, r

    def csr(self):
        return mat_get_csr(self.h)

    def coo_maps(self):
        return mat_get_coo_maps(self.h)

    def set_plan(self, spmv_rows=0, update_rows=0, kernel=SPMV_AUTO, ctas_per_sm=0):
        mat_set_plan(self.h, spmv_rows, update_rows, kernel, ctas_per_sm)

    def plan(self) -> dict:
        return mat_get_plan(self.h)

    def set_slice_patterns(self, on: bool):
        """Column patterns of the sliced copy on (default) or off; results
        are bit-identical either way."""
        mat_set_slice_patterns(self.h, on)

    def slices(self) -> dict:
        return mat_get_slices(self.h)

    def set_solver(self, solver: int, split_rows=None):
        """The engine (SOLVER_*); with SOLVER_SPLIT, split_rows is the row
        count from which a batch's systems run on the phase kernels."""
        if split_rows is not None:
            mat_set_split_rows(self.h, split_rows)
        mat_set_solver(self.h, solver)

    def phase_ns(self) -> dict:
        return ksp_get_phase_ns(self.h)

    def autotune(self, path=None, stream=None):
        """Tune the solve (persisted in the file at path when given; returns
        whether the tuning came from that file)."""
        if path is None:
            mat_autotune(self.h, stream)
            return False
        return mat_autotune_file(self.h, path, stream)

    def set_cg_form(self, form: int):
        mat_set_cg_form(self.h, form)

    def tuning(self) -> dict:
        return mat_get_tuning(self.h)

    def close(self):
        if self.h:
            mat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
