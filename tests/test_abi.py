"""Host-side checks (no GPU): the C-ABI library builds for sm_103a, loads, and
exports every function include/gbs.h declares; the binding's struct layouts
match the header's."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_08646_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mat_create_coo", "mat_set_values_coo", "mat_mult", "ksp_solve_cg",
                 "ksp_adjoint", "ksp_solve_cg_batched", "mat_create_coo_batched",
                 "mat_destroy", "gbs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2406_08646_gb300 import binding
    assert sorted(binding.EXPORTED) == declared_functions()


def test_struct_sizes_match_header():
    """Compile a tiny C program against gbs.h and compare sizeof/offsetof with
    the ctypes mirrors."""
    import subprocess
    import tempfile
    from paper_2406_08646_gb300 import binding as B
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "gbs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ksp_opts), sizeof(ksp_result),
         offsetof(ksp_opts, timeout_ns), offsetof(ksp_opts, host_loop),
         offsetof(ksp_opts, method), offsetof(ksp_result, true_rel_residual));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    got = [int(v) for v in out]
    assert got == [ctypes.sizeof(B.KspOpts), ctypes.sizeof(B.KspResult),
                   B.KspOpts.timeout_ns.offset, B.KspOpts.host_loop.offset,
                   B.KspOpts.method.offset, B.KspResult.true_rel_residual.offset]


def test_opts_defaults_and_errors_without_gpu(lib):
    from paper_2406_08646_gb300 import binding as B
    o = B.make_opts()
    assert o.rtol == 1e-8 and o.maxit == -1 and o.precision == 0 and o.max_outer == 30
    # host-side argument checks return before any device work
    L = B.lib()
    h = ctypes.c_void_p()
    assert L.mat_create_coo(-1, 4, 0, None, None, None, ctypes.byref(h)) == B.ERR_ARG
    assert "sizes" in B.last_error()
    assert L.mat_mult(None, None, None, None) == B.ERR_ARG
    assert L.ksp_solve_cg(None, None, None, None, None, None) == B.ERR_ARG
    assert L.mat_destroy(None) == B.OK


def test_product_path_has_no_cpu_fallback():
    """The binding and the package never import the oracle."""
    pkg = os.path.join(ROOT, "paper_2406_08646_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn


P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
HANDLE_CALLS = {  # every entry point taking a matrix / vector handle: its argument types
    "mat_set_values_coo": [P, P, I32, P],
    "mat_mult": [P, P, P, P],
    "ksp_solve_cg": [P, P, P, P, P, P],
    "ksp_solve_cg_batched": [P, P, P, P, P, P],
    "ksp_solve": [P, P, P, P, P, P],
    "ksp_solve_batched": [P, P, P, P, P, P],
    "ksp_adjoint": [P, P, P, P, P, P, P, P, P],
    "ksp_adjoint_batched": [P, P, P, P, P, P, P, P, P],
    "ksp_get_result": [P, P, I32, P],
    "ksp_get_phase_ns": [P, P, P],
    "mat_get_info": [P, P, P, P, P, P],
    "mat_get_csr": [P, P, P, P, P],
    "mat_get_coo_maps": [P, P, P, P],
    "mat_set_plan": [P, I32, I32, I32, I32],
    "mat_get_plan": [P, P, P, P, P, P],
    "mat_set_solver": [P, I32],
    "mat_autotune": [P, P],
    "mat_autotune_file": [P, P, P, P],
    "mat_set_cg_form": [P, I32],
    "mat_get_tuning": [P, P, P, P],
    "mat_set_split_rows": [P, I64],
    "mat_set_slice_patterns": [P, I32],
    "mat_get_slices": [P, P, P, P],
    "vec_set_values_coo": [P, P, I32, P, P],
    "vec_get_info": [P, P, P, P],
}


def test_every_handle_entry_point_rejects_a_null_handle_without_gpu(lib):
    """A null handle is an argument error (GBS_ERR_ARG with a message), found
    before any device call; destroying a null handle is a no-op."""
    from paper_2406_08646_gb300 import binding as B
    assert set(HANDLE_CALLS) | {"mat_destroy", "vec_destroy"} == {
        n for n in declared_functions()
        if n.startswith(("mat_", "ksp_", "vec_")) and n not in (
            "mat_create_coo", "mat_create_coo_batched", "vec_create_coo",
            "ksp_opts_default", "ksp_solve_cg_noalloc")}
    for name, types in HANDLE_CALLS.items():
        f = getattr(lib, name)
        f.argtypes = types
        f.restype = ctypes.c_int
        args = [None if t is P else 0 for t in types]
        assert f(*args) == B.ERR_ARG, name
        assert B.last_error(), name
    for name in ("mat_destroy", "vec_destroy"):
        f = getattr(lib, name)
        f.argtypes = [P]
        f.restype = ctypes.c_int
        assert f(None) == B.OK, name


def test_create_size_checks_without_gpu(lib):
    """Sizes and counts are checked on the host before any device call."""
    from paper_2406_08646_gb300 import binding as B
    h = ctypes.c_void_p()
    f = lib.mat_create_coo
    f.argtypes = [I64, I64, I64, P, P, P, P]
    f.restype = ctypes.c_int
    assert f(4, -1, 0, None, None, None, ctypes.byref(h)) == B.ERR_ARG
    assert f(4, 4, -5, None, None, None, ctypes.byref(h)) == B.ERR_ARG
    assert f(1 << 31, 4, 0, None, None, None, ctypes.byref(h)) == B.ERR_ARG  # int32 indices
    g = lib.mat_create_coo_batched
    g.argtypes = [I32, P, P, P, P, P, P]
    g.restype = ctypes.c_int
    assert g(0, None, None, None, None, None, ctypes.byref(h)) == B.ERR_ARG
    v = lib.vec_create_coo
    v.argtypes = [I64, I64, P, P, P]
    v.restype = ctypes.c_int
    assert v(-1, 0, None, None, ctypes.byref(h)) == B.ERR_ARG
    n = lib.ksp_solve_cg_noalloc
    n.argtypes = [I64, P, P, P, P, P, P, P, P]
    n.restype = ctypes.c_int
    assert n(-1, None, None, None, None, None, None, None, None) == B.ERR_ARG


def test_binding_rejects_host_tensors_and_fills_options_without_gpu():
    """The binding passes only CUDA tensors to the library (a host tensor is
    refused before any call: there is no CPU path), and make_opts fills the
    header's struct field by field."""
    import torch
    from paper_2406_08646_gb300 import binding as B
    with pytest.raises(ValueError):
        B._dev(torch.zeros(3, dtype=torch.float64), torch.float64, 3, "b")
    assert B._dev(None, torch.float64) is None
    o = B.make_opts(rtol=1e-10, maxit=77, precision=B.FP32_REFINED, inner_rtol=1e-3,
                    max_outer=5, inner_maxit=9, timeout_ns=123, nonzero_guess=True,
                    host_loop=True, method=B.KSP_TFQMR)
    assert (o.rtol, o.maxit, o.precision, o.inner_rtol, o.max_outer, o.inner_maxit,
            o.timeout_ns, o.nonzero_guess, o.host_loop, o.method) == (
        1e-10, 77, B.FP32_REFINED, 1e-3, 5, 9, 123, 1, 1, B.KSP_TFQMR)


def test_generation_entry_points_check_arguments_without_gpu(lib):
    """The device-side COO generators refuse bad sizes and null pointers on
    the host, before any device call."""
    from paper_2406_08646_gb300 import binding as B
    lib.q1_hex_element_coo.argtypes = [I32, P, P, P]
    lib.q1_hex_element_values.argtypes = [I32, P, P, P]
    lib.edge_coo_values.argtypes = [I64, P, P, P]
    for f in (lib.q1_hex_element_coo, lib.q1_hex_element_values, lib.edge_coo_values):
        f.restype = ctypes.c_int
    assert lib.q1_hex_element_coo(0, None, None, None) == B.ERR_ARG
    assert lib.q1_hex_element_coo(400, None, None, None) == B.ERR_ARG
    assert lib.q1_hex_element_coo(4, None, None, None) == B.ERR_ARG
    assert lib.q1_hex_element_values(4, None, None, None) == B.ERR_ARG
    assert lib.edge_coo_values(-1, None, None, None) == B.ERR_ARG
    assert lib.edge_coo_values(1 << 29, None, None, None) == B.ERR_ARG
    assert lib.edge_coo_values(0, None, None, None) == B.OK
