"""Pins of the oracle's COO -> CSR assembly (Sec. 5: the assembled matrix is the
sum of the contributions v[k] to a_{i[k],j[k]}; negative indices are ignored;
preallocation fixes the pattern, set-values fills it with INSERT or ADD).

The oracle sorts; these pins use other routes: a Python dict fold, a dense
np.add.at accumulate, a hand-worked example, and invariants."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_coo(rng, n, ncoo, dup=0.3, neg=0.1, integer=False, ncols=None):
    ncols = n if ncols is None else ncols
    base = max(1, int(ncoo * (1 - dup)))
    i = rng.integers(0, n, base)
    j = rng.integers(0, ncols, base)
    pick = rng.integers(0, base, ncoo - base)
    i = np.concatenate([i, i[pick]])
    j = np.concatenate([j, j[pick]])
    sh = rng.permutation(ncoo)
    i, j = i[sh], j[sh]
    drop = rng.random(ncoo) < neg
    which = rng.random(ncoo) < 0.5
    i = np.where(drop & which, -1 - rng.integers(0, 3, ncoo), i)
    j = np.where(drop & ~which, -1 - rng.integers(0, 3, ncoo), j)
    if integer:
        v = rng.integers(-8, 9, ncoo).astype(np.float64)
    else:
        v = rng.standard_normal(ncoo) * 10.0 ** rng.uniform(-3, 3, ncoo)
    return i.astype(np.int32), j.astype(np.int32), v


def dict_fold(i, j, v):
    """Brute force: per (row, col), left fold over k ascending."""
    acc = {}
    for k in range(len(i)):
        if i[k] < 0 or j[k] < 0:
            continue
        key = (int(i[k]), int(j[k]))
        acc[key] = v[k] if key not in acc else acc[key] + v[k]
    return acc


def csr_entries(A):
    out = {}
    for r in range(A.nrows):
        for p in range(A.row_ptr[r], A.row_ptr[r + 1]):
            out[(r, int(A.col[p]))] = A.val[p] if A.val is not None else None
    return out


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_dict_fold_bitexact(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    ncoo = int(rng.integers(0, 4097))
    i, j, v = random_coo(rng, n, ncoo)
    A = oracle.coo_symbolic(n, n, i, j)
    oracle.coo_numeric(A, v)
    ref = dict_fold(i, j, v)
    got = csr_entries(A)
    assert set(got) == set(ref)
    for key, val in ref.items():
        assert np.float64(got[key]).tobytes() == np.float64(val).tobytes(), key
    # CSR invariants: rows ascending, columns strictly ascending in a row
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz
    assert np.all(np.diff(A.row_ptr) >= 0)
    for r in range(n):
        c = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    assert A.nkept == int(np.sum((i >= 0) & (j >= 0)))


@pytest.mark.parametrize("seed", range(4))
def test_dense_add_at_integer_values(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = int(rng.integers(1, 50)), int(rng.integers(1, 50))
    i, j, v = random_coo(rng, n, 3000, integer=True, ncols=m)
    A = oracle.coo_symbolic(n, m, i, j)
    oracle.coo_numeric(A, v)
    D = np.zeros((n, m))
    keep = (i >= 0) & (j >= 0)
    np.add.at(D, (i[keep], j[keep]), v[keep])
    R = np.zeros((n, m))
    for r in range(n):
        for p in range(A.row_ptr[r], A.row_ptr[r + 1]):
            R[r, A.col[p]] = A.val[p]
    assert np.array_equal(D, R)
    # the sum over all nonzeros equals the sum over the kept entries, exactly
    assert A.val.sum() == v[keep].sum()


def test_maps_are_consistent():
    rng = np.random.default_rng(7)
    i, j, v = random_coo(rng, 40, 2000)
    A = oracle.coo_symbolic(40, 40, i, j)
    rows = np.repeat(np.arange(40), np.diff(A.row_ptr))
    assert A.jmap[0] == 0 and A.jmap[-1] == A.nkept
    for p in range(A.nnz):
        seg = A.perm[A.jmap[p]:A.jmap[p + 1]]
        assert len(seg) >= 1 and np.all(np.diff(seg) > 0)   # increasing k
        assert np.all(i[seg] == rows[p]) and np.all(j[seg] == A.col[p])
    assert sorted(A.perm.tolist()) == np.flatnonzero((i >= 0) & (j >= 0)).tolist()


def test_structure_invariant_under_permutation():
    rng = np.random.default_rng(8)
    i, j, v = random_coo(rng, 30, 1500, integer=True)
    A = oracle.coo_symbolic(30, 30, i, j)
    oracle.coo_numeric(A, v)
    sh = rng.permutation(len(i))
    B = oracle.coo_symbolic(30, 30, i[sh], j[sh])
    oracle.coo_numeric(B, v[sh])
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col)
    assert np.array_equal(A.val, B.val)          # integers: any order is exact


def test_add_mode_and_insert_mode():
    rng = np.random.default_rng(9)
    i, j, v = random_coo(rng, 20, 500, integer=True)
    A = oracle.coo_symbolic(20, 20, i, j)
    a1 = oracle.coo_numeric(A, v).copy()
    a2 = oracle.coo_numeric(A, 2 * v, mode=oracle.ADD).copy()
    assert np.array_equal(a2, 3 * a1)
    a3 = oracle.coo_numeric(A, v, mode=oracle.INSERT)
    assert np.array_equal(a3, a1)


def test_negative_zero_kept_and_empty_cases():
    A = oracle.coo_symbolic(3, 3, np.array([1], np.int32), np.array([2], np.int32))
    oracle.coo_numeric(A, np.array([-0.0]))
    assert np.signbit(A.val[0])
    E = oracle.coo_symbolic(5, 5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert E.nnz == 0 and np.all(E.row_ptr == 0)
    N = oracle.coo_symbolic(5, 5, np.array([-1, 2, -3], np.int32),
                            np.array([0, -1, -2], np.int32))
    assert N.nnz == 0 and N.nkept == 0
    R = oracle.coo_symbolic(6, 6, np.array([5, 0], np.int32), np.array([5, 0], np.int32))
    assert R.row_ptr.tolist() == [0, 1, 1, 1, 1, 1, 2]     # empty rows repeat


def test_out_of_range_is_an_error():
    with pytest.raises(oracle.OracleError) as e:
        oracle.coo_symbolic(4, 4, np.array([0, 4], np.int32), np.array([0, 0], np.int32))
    assert e.value.status == oracle.ERR_INDEX
    with pytest.raises(oracle.OracleError):
        oracle.coo_symbolic(4, 3, np.array([0], np.int32), np.array([3], np.int32))


def test_scatter_is_the_transpose_of_numeric():
    rng = np.random.default_rng(10)
    i, j, v = random_coo(rng, 25, 800, integer=True)
    A = oracle.coo_symbolic(25, 25, i, j)
    a = oracle.coo_numeric(A, v)
    w = rng.integers(-5, 6, A.nnz).astype(np.float64)
    g = oracle.coo_scatter(A, w)
    assert float(w @ a) == float(g @ v)               # <w, S v> = <S^T w, v>
    assert np.all(g[(i < 0) | (j < 0)] == 0.0)


def test_hand_worked_example():
    with open(os.path.join(GOLDEN, "coo_worked_example.json")) as f:
        ex = json.load(f)
    A = oracle.coo_symbolic(ex["nrows"], ex["ncols"], np.array(ex["i"], np.int32),
                            np.array(ex["j"], np.int32))
    oracle.coo_numeric(A, np.array(ex["v"], np.float64))
    assert A.row_ptr.tolist() == ex["row_ptr"]
    assert A.col.tolist() == ex["col"]
    assert A.val.tolist() == ex["val"]
    assert A.perm.tolist() == ex["perm"]
    assert A.jmap.tolist() == ex["jmap"]


# ------------------------------------------------------------------ vectors

@pytest.mark.parametrize("seed", range(4))
def test_vec_coo_equals_matrix_route_and_dense_sum(seed):
    """Vector COO assembly (Sec. 5 for vectors) pinned two other ways: the
    matrix assembly of the same entries as an n x 1 matrix (sort route), and,
    for integer values, a dense np.add.at accumulate; ADD adds to y, indices
    that do not appear keep y."""
    rng = np.random.default_rng(100 + seed)
    n, ncoo = 97, 2000
    i, _, v = random_coo(rng, n, ncoo)
    y0 = rng.standard_normal(n)
    A = oracle.coo_symbolic(n, 1, i, np.zeros_like(i))
    a = oracle.coo_numeric(A, v)
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    yi = oracle.vec_set_values_coo(n, i, v, oracle.INSERT, y0)
    exp = y0.copy()
    exp[rows] = a
    assert yi.tobytes() == exp.tobytes()
    ya = oracle.vec_set_values_coo(n, i, v, oracle.ADD, y0)
    exp = y0.copy()
    exp[rows] = y0[rows] + a
    assert ya.tobytes() == exp.tobytes()
    iv = rng.integers(-8, 9, ncoo).astype(np.float64)
    dense = np.zeros(n)
    keep = i >= 0
    np.add.at(dense, i[keep], iv[keep])
    got = oracle.vec_set_values_coo(n, i, iv, oracle.ADD, np.zeros(n))
    assert np.array_equal(got, dense)


def test_vec_coo_order_and_errors():
    # the fold starts from the first term: a lone -0.0 stays -0.0, and the
    # order is increasing COO index (1e16 + 1 - 1e16 = 0, but 1e16 - 1e16 + 1 = 1)
    y = oracle.vec_set_values_coo(3, np.array([2, 0, 0, 0], np.int32),
                                  np.array([-0.0, 1e16, 1.0, -1e16]), oracle.INSERT,
                                  np.array([5.0, 6.0, 7.0]))
    assert np.signbit(y[2]) and y[2] == 0.0 and y[1] == 6.0 and y[0] == 0.0
    y = oracle.vec_set_values_coo(2, np.array([0, 0, 0], np.int32),
                                  np.array([1e16, -1e16, 1.0]), oracle.INSERT)
    assert y[0] == 1.0
    with pytest.raises(oracle.OracleError):
        oracle.vec_set_values_coo(2, np.array([2], np.int32), np.array([1.0]))
