"""The allocation-free solve entry point, ksp_solve_cg_noalloc.

Some callers cannot allocate device memory (their memory is budgeted by
another allocator, or they cannot pay for the synchronisation cudaMalloc
implies); this entry point serves them from a fixed static scratch array.
The tests call it through the C-ABI:
  * twice in a row on a CSR matrix built by the library, checking both
    answers against ksp_solve_cg's on the same system and against the
    oracle (true residual recomputed by the oracle's SpMV on a host copy of
    the CSR, iteration count against the oracle's PCG);
  * at exactly the array's row limit (a 512 x 512 5-point Laplacian,
    262,144 rows);
  * on a matrix with a zero and one with a missing diagonal entry
    (GBS_ERR_NOT_SPD, also with a NULL result pointer);
  * with arguments it must refuse up front (too many rows, another method).
Collected last on purpose (file name)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2406_08646_gb300 import binding as B
from paper_2406_08646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NOALLOC_MAX_ROWS = 262144


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(n, rp, col, val, b, x, opts, res=True):
    L = B.lib()
    r = B.KspResult() if res else None
    st = L.ksp_solve_cg_noalloc(n, _p(rp), _p(col), _p(val), _p(b), _p(x),
                                ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(r) if res else None, B._stream(None))
    return st, r


def _host_csr(n, rp, col, val):
    return oracle.CSR(n, n, rp.cpu().numpy(), col.cpu().numpy(),
                      np.zeros(0, np.int32), np.zeros(1, np.int32), 0, val.cpu().numpy())


def _oracle_true_rel(O, b, x):
    bh = b.cpu().numpy()
    return np.linalg.norm(bh - oracle.spmv(O, x.cpu().numpy())) / np.linalg.norm(bh)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_noalloc_solve_matches_ksp_solve_cg_and_the_oracle_twice():
    dev = torch.device("cuda:0")
    p = W.edge_diffusion(150, seed=123)          # 22,500 rows, ragged last block
    A = B.Mat.from_coo(p.nrows, p.ncols, torch.from_numpy(p.i).to(dev),
                       torch.from_numpy(p.j).to(dev))
    A.set_values(torch.from_numpy(p.v).to(dev))
    b = torch.from_numpy(p.b).to(dev)
    rtol = 1e-10
    x_ref, r_ref = A.solve(b, rtol=rtol)
    assert r_ref["status"] == B.OK
    rp, col, val = A.csr()
    O = _host_csr(p.nrows, rp, col, val)
    _, ro = oracle.pcg(O, p.b, rtol=rtol)
    assert ro["status"] == oracle.OK
    opts = B.make_opts(rtol=rtol)
    for call in range(2):
        x = torch.full_like(b, float("nan"))
        st, res = _noalloc(p.nrows, rp, col, val, b, x, opts)
        assert st == B.OK, B.last_error()
        assert res.status == B.OK
        assert abs(res.iterations - r_ref["iterations"]) <= max(2, r_ref["iterations"] // 100)
        assert abs(res.iterations - ro["iterations"]) <= max(2, ro["iterations"] // 100)
        assert res.true_rel_residual <= rtol * 1.05
        err = torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)
        assert err.item() <= 1e4 * rtol, (call, err.item())
        # the answer's residual recomputed by the oracle on the host CSR
        assert _oracle_true_rel(O, b, x) <= rtol * 1.05
    A.close()


def test_noalloc_at_exactly_the_row_limit():
    dev = torch.device("cuda:0")
    m = 512
    p = W.poisson2d(m)                            # 262,144 rows: the whole array
    assert p.nrows == NOALLOC_MAX_ROWS
    b_h = np.random.default_rng(2024).standard_normal(p.nrows)
    A = B.Mat.from_coo(p.nrows, p.ncols, torch.from_numpy(p.i).to(dev),
                       torch.from_numpy(p.j).to(dev))
    A.set_values(torch.from_numpy(p.v).to(dev))
    b = torch.from_numpy(b_h).to(dev)
    rp, col, val = A.csr()
    O = _host_csr(p.nrows, rp, col, val)
    rtol = 1e-8
    _, ro = oracle.pcg(O, b_h, rtol=rtol)
    x = torch.full_like(b, float("nan"))
    st, res = _noalloc(p.nrows, rp, col, val, b, x, B.make_opts(rtol=rtol))
    assert st == B.OK, B.last_error()
    assert abs(res.iterations - ro["iterations"]) <= max(2, ro["iterations"] // 100)
    assert _oracle_true_rel(O, b, x) <= rtol * 1.05
    A.close()


def test_noalloc_reports_a_bad_diagonal_with_or_without_a_result():
    dev = torch.device("cuda:0")
    p = W.edge_diffusion(40, seed=5)
    A = B.Mat.from_coo(p.nrows, p.ncols, torch.from_numpy(p.i).to(dev),
                       torch.from_numpy(p.j).to(dev))
    A.set_values(torch.from_numpy(p.v).to(dev))
    rp, col, val = (t.clone() for t in A.csr())
    A.close()
    rph, colh = rp.cpu().numpy(), col.cpu().numpy()
    r = 777                                       # zero this row's diagonal entry
    q = rph[r] + int(np.nonzero(colh[rph[r]:rph[r + 1]] == r)[0][0])
    val[q] = 0.0
    b = torch.from_numpy(p.b).to(dev)
    x = torch.empty_like(b)
    st, res = _noalloc(p.nrows, rp, col, val, b, x, B.make_opts())
    assert st == B.ERR_NOT_SPD and res.status == B.ERR_NOT_SPD
    st, _ = _noalloc(p.nrows, rp, col, val, b, x, B.make_opts(), res=False)
    assert st == B.ERR_NOT_SPD
    # a missing diagonal: [[0 1] [1 2]] stored without its (0, 0) entry
    rp2 = torch.tensor([0, 1, 3], dtype=torch.int32, device=dev)
    col2 = torch.tensor([1, 0, 1], dtype=torch.int32, device=dev)
    val2 = torch.tensor([1.0, 1.0, 2.0], dtype=torch.float64, device=dev)
    b2 = torch.ones(2, dtype=torch.float64, device=dev)
    x2 = torch.empty_like(b2)
    st, res = _noalloc(2, rp2, col2, val2, b2, x2, None)
    assert st == B.ERR_NOT_SPD and res.status == B.ERR_NOT_SPD
    # and a good solve right after still works on the shared array
    val[q] = float(np.abs(p.v).max()) * 4.0
    st, res = _noalloc(p.nrows, rp, col, val, b, x, B.make_opts(rtol=1e-8))
    assert st == B.OK and res.status == B.OK


def test_noalloc_rejects_sizes_beyond_the_static_scratch_and_other_methods():
    L = B.lib()
    res = B.KspResult()
    st = L.ksp_solve_cg_noalloc(NOALLOC_MAX_ROWS + 1, None, None, None, None, None, None,
                                ctypes.byref(res), None)
    assert st == B.ERR_ARG
    assert str(NOALLOC_MAX_ROWS) in B.last_error()
    dev = torch.device("cuda:0")
    z = torch.zeros(8, dtype=torch.float64, device=dev)
    zi = torch.zeros(8, dtype=torch.int32, device=dev)
    for method in (B.KSP_BICG, B.KSP_TFQMR, B.KSP_PIPECG):
        st, _ = _noalloc(4, zi, zi, z, z, z, B.make_opts(method=method))
        assert st == B.ERR_ARG and "method" in B.last_error()
