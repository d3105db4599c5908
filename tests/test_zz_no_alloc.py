"""The allocation-free solve entry point, ksp_solve_cg_noalloc.

Some callers cannot allocate device memory (their memory is budgeted by
another allocator, or they cannot pay for the synchronisation cudaMalloc
implies); this entry point serves them from a fixed static scratch array.
The test calls it through the C-ABI, twice in a row, on a CSR matrix built by
the library, and checks both answers against ksp_solve_cg's on the same
system, within the solve tolerance the parity tests use.  It also checks the
size limit is refused up front.  Collected last on purpose (file name)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2406_08646_gb300 import binding as B
from paper_2406_08646_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_solve_matches_ksp_solve_cg_twice():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    L = B.lib()
    p = W.edge_diffusion(150, seed=123)          # 22,500 rows, ragged last block
    A = B.Mat.from_coo(p.nrows, p.ncols, torch.from_numpy(p.i).to(dev),
                       torch.from_numpy(p.j).to(dev))
    A.set_values(torch.from_numpy(p.v).to(dev))
    b = torch.from_numpy(p.b).to(dev)
    rtol = 1e-10
    x_ref, r_ref = A.solve(b, rtol=rtol)
    assert r_ref["status"] == B.OK
    rp, col, val = A.csr()
    opts = B.make_opts(rtol=rtol)
    stream = B._stream(None)
    for call in range(2):
        x = torch.full_like(b, float("nan"))
        res = B.KspResult()
        st = L.ksp_solve_cg_noalloc(p.nrows, _p(rp), _p(col), _p(val), _p(b), _p(x),
                                    ctypes.byref(opts), ctypes.byref(res), stream)
        assert st == B.OK, B.last_error()
        assert res.status == B.OK
        assert abs(res.iterations - r_ref["iterations"]) <= max(2, r_ref["iterations"] // 100)
        assert res.true_rel_residual <= rtol * 1.05
        err = torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)
        assert err.item() <= 1e4 * rtol, (call, err.item())
        # residual of the no-alloc answer, computed with the library's SpMV
        ax = A.mult(x)
        assert (torch.linalg.norm(b - ax) / torch.linalg.norm(b)).item() <= rtol * 1.05
    A.close()


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    L = B.lib()
    res = B.KspResult()
    st = L.ksp_solve_cg_noalloc(262145, None, None, None, None, None, None,
                                ctypes.byref(res), None)
    assert st == B.ERR_ARG
    assert "262144" in B.last_error()
