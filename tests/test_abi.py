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
