"""GPU parity of the vector COO assembly (Sec. 5's COO interface for vectors)
against the oracle: bit-exact values, INSERT and ADD, untouched entries,
ignored and out-of-range indices."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_08646_gb300 import binding as B

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("n,ncoo", [(1, 1), (13, 200), (1000, 30000), (70001, 500000)])
def test_vec_assembly_bitexact(n, ncoo):
    rng = np.random.default_rng(n)
    i = rng.integers(0, n, ncoo).astype(np.int32)
    i[rng.random(ncoo) < 0.1] = -1
    v = rng.standard_normal(ncoo) * 10.0 ** rng.uniform(-3, 3, ncoo)
    y0 = rng.standard_normal(n)
    V = B.Vec(n, t(i))
    assert V.info["nentries"] == len(np.unique(i[i >= 0]))
    for mode in (B.INSERT, B.ADD):
        y = V.set_values(t(v), t(y0), mode).cpu().numpy()
        exp = oracle.vec_set_values_coo(n, i, v, mode, y0)
        assert y.tobytes() == exp.tobytes(), mode
    V.close()


def test_vec_element_load_vector():
    """Q1-style load vector: 8 contributions per element into its nodes."""
    m = 24
    ex, ey, ez = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    base = (ex + (m + 1) * (ey + (m + 1) * ez)).reshape(-1)
    offs = np.array([a + (m + 1) * (b + (m + 1) * c) for c in (0, 1) for b in (0, 1)
                     for a in (0, 1)])
    i = (base[:, None] + offs[None, :]).reshape(-1).astype(np.int32)
    v = np.random.default_rng(3).uniform(0.1, 10.0, i.shape[0])
    n = (m + 1) ** 3
    V = B.Vec(n, t(i))
    y = V.set_values(t(v)).cpu().numpy()
    assert y.tobytes() == oracle.vec_set_values_coo(n, i, v).tobytes()
    V.close()


def test_vec_errors():
    with pytest.raises(B.GbsError) as e:
        B.Vec(4, t(np.array([0, 4], np.int32)))
    assert e.value.status == B.ERR_INDEX
    V = B.Vec(5, t(np.array([-1, -2], np.int32)))     # nothing kept: y untouched
    y0 = torch.arange(5, dtype=torch.float64, device=DEV)
    y = V.set_values(t(np.array([1.0, 2.0])), y0.clone())
    assert torch.equal(y, y0) and V.info["nentries"] == 0
    V.close()
