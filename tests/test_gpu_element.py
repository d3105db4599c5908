"""Device-side COO generation (the user Jacobian kernel of Sec. 3 filling v on
the GPU, with Sec. 5's per-element offsets) against the seeded host
generator: the Q1 element blocks (indices and values with the Dirichlet
edits) and the edge values, bit for bit (compared as 64-bit patterns, so
that +0.0 / -0.0 count), from one element up to the full 96^3 mesh; then the
matrix assembled from the device-generated triples against the oracle's
assembly of the host triples."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2406_08646_gb300 import binding as B
from paper_2406_08646_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def dev():
    return torch.device("cuda:0")


def bits(t):
    return t.contiguous().view(torch.int64)


@pytest.mark.parametrize("ne", [1, 2, 3, 5, 12, 31])
def test_q1_element_blocks_bitexact(ne):
    p = W.q1_hex(ne, seed=1000 + ne)
    n = 64 * ne ** 3
    i = torch.empty(n, dtype=torch.int32, device=dev())
    j = torch.empty(n, dtype=torch.int32, device=dev())
    v = torch.full((n,), float("nan"), dtype=torch.float64, device=dev())
    kappa = torch.from_numpy(p.extra["kappa"]).to(dev())
    B.q1_hex_element_coo(ne, i, j)
    B.q1_hex_element_values(ne, kappa, v)
    torch.cuda.synchronize()
    assert np.array_equal(i.cpu().numpy(), p.i)
    assert np.array_equal(j.cpu().numpy(), p.j)
    assert np.array_equal(bits(v).cpu().numpy(), p.v.view(np.int64))


def test_q1_element_blocks_full_size_and_assembly():
    ne = 96
    p = W.q1_hex(ne, seed=W.SEED_C2)
    n = 64 * ne ** 3
    i = torch.empty(n, dtype=torch.int32, device=dev())
    j = torch.empty(n, dtype=torch.int32, device=dev())
    v = torch.empty(n, dtype=torch.float64, device=dev())
    B.q1_hex_element_coo(ne, i, j)
    B.q1_hex_element_values(ne, torch.from_numpy(p.extra["kappa"]).to(dev()), v)
    assert torch.equal(i, torch.from_numpy(p.i).to(dev()))
    assert torch.equal(j, torch.from_numpy(p.j).to(dev()))
    assert torch.equal(bits(v), bits(torch.from_numpy(p.v).to(dev())))
    del i, j, v
    torch.cuda.empty_cache()


def test_assembly_from_device_generated_triples_matches_the_oracle():
    ne = 14
    p = W.q1_hex(ne, seed=77)
    n = 64 * ne ** 3
    i = torch.empty(n, dtype=torch.int32, device=dev())
    j = torch.empty(n, dtype=torch.int32, device=dev())
    v = torch.empty(n, dtype=torch.float64, device=dev())
    B.q1_hex_element_coo(ne, i, j)
    B.q1_hex_element_values(ne, torch.from_numpy(p.extra["kappa"]).to(dev()), v)
    A = B.Mat.from_coo(p.nrows, p.ncols, i, j)
    A.set_values(v)
    O = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(O, p.v)
    rp, col, val = (t.cpu().numpy() for t in A.csr())
    assert np.array_equal(rp, O.row_ptr) and np.array_equal(col, O.col)
    assert np.array_equal(val.view(np.int64), O.val.view(np.int64))
    x, r = A.solve(torch.from_numpy(p.b).to(dev()), rtol=1e-9)
    assert r["status"] == B.OK
    res = np.linalg.norm(p.b - oracle.spmv(O, x.cpu().numpy())) / np.linalg.norm(p.b)
    assert res <= 1e-9 * 1.05
    A.close()


@pytest.mark.parametrize("make", [lambda: W.edge_diffusion(37, seed=3),
                                  lambda: W.edge_diffusion(1024, seed=W.SEED_C4)])
def test_edge_values_bitexact(make):
    p = make()
    kappa = torch.from_numpy(p.extra["kappa"]).to(dev())
    v = torch.full((4 * kappa.numel(),), float("nan"), dtype=torch.float64, device=dev())
    B.edge_coo_values(kappa, v)
    assert torch.equal(bits(v), bits(torch.from_numpy(p.v).to(dev())))


def test_edge_values_of_a_batch_bitexact():
    bt = W.batch(24, seed=5, size_range=(100, 3000))
    kappa = torch.from_numpy(np.concatenate(bt.extra["kappa"])).to(dev())
    v = torch.empty(4 * kappa.numel(), dtype=torch.float64, device=dev())
    B.edge_coo_values(kappa, v)
    assert torch.equal(bits(v), bits(torch.from_numpy(bt.v).to(dev())))


def test_generation_argument_errors():
    L = B.lib()
    z = torch.zeros(64, dtype=torch.float64, device=dev())
    zi = torch.zeros(64, dtype=torch.int32, device=dev())
    p = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)
    s = B._stream(None)
    assert L.q1_hex_element_coo(0, p(zi), p(zi), s) == B.ERR_ARG
    assert L.q1_hex_element_coo(400, p(zi), p(zi), s) == B.ERR_ARG     # 64 ne^3 >= 2^31
    assert L.q1_hex_element_coo(1, p(zi, 4), p(zi), s) == B.ERR_ARG    # not 16-byte aligned
    assert L.q1_hex_element_values(1, p(z), p(z, 8), s) == B.ERR_ARG
    assert L.q1_hex_element_values(1, None, p(z), s) == B.ERR_ARG
    assert L.edge_coo_values(-1, p(z), p(z), s) == B.ERR_ARG
    assert L.edge_coo_values(0, None, None, s) == B.OK
    assert L.edge_coo_values(2, p(z), p(z, 8), s) == B.ERR_ARG
