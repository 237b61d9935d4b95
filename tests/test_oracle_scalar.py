"""Oracle pins for scalar (1x1-block) CSR systems: the paper's CSR inputs.

The oracle's functions take the block dimension from the data; with bs = 1
each one must reduce to its textbook scalar form. The pins check it against
facts the mathematics fixes: ILU0's pattern property and its scalar IKJ
definition on a dense copy, exact LU on a path, Jacobi for one-row
subdomains, the SpMV as a dense product, the fixed dot order on crafted
values, and BiCGSTAB iterates against SciPy's.
"""
import numpy as np
import pytest

import oracle
import synth
from _dense import dense_scalar_ilu0

sp = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")


def _dense(row_ptr, col, val, n):
    D = np.zeros((n, n))
    for i in range(n):
        for q in range(row_ptr[i], row_ptr[i + 1]):
            D[i, col[q]] = np.asarray(val).reshape(-1)[q]
    return D


def _mask(row_ptr, col, n):
    M = np.zeros((n, n), bool)
    for i in range(n):
        M[i, col[row_ptr[i]:row_ptr[i + 1]]] = True
    return M


def _lu_dense(LU, n):
    L, U = np.eye(n), np.zeros((n, n))
    v = LU.val.reshape(-1)
    for i in range(n):
        for q in range(LU.row_ptr[i], LU.row_ptr[i + 1]):
            (L if LU.col[q] < i else U)[i, LU.col[q]] = v[q]
    return L, U


@pytest.mark.parametrize("grid,sub,model", [((6, 5, 4), (3, 3, 2), synth.MODEL_LAPLACE),
                                            ((8, 8, 4), (8, 8, 4), synth.MODEL_LAYERED)])
def test_scalar_ilu0_pattern_property_and_textbook_form(grid, sub, model):
    s = synth.system(*grid, 5, model=model, bs=1)
    d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
    assert d.LU.bs == 1 and d.status == 0
    n = s.n
    L, U = _lu_dense(d.LU, n)
    Add = _dense(d.Add.row_ptr, d.Add.col, d.Add.val, n)
    mask = _mask(d.Add.row_ptr, d.Add.col, n)
    assert np.abs((L @ U - Add)[mask]).max() <= 1e-13 * np.abs(Add).max()
    Lt, Ut = dense_scalar_ilu0(Add, mask)
    assert np.abs(L - Lt).max() <= 1e-13 and np.abs(U - Ut).max() <= 1e-13 * np.abs(Ut).max()


def test_scalar_chain_is_exact_lu():
    """A path (n x 1 x 1, one subdomain) has no fill: the apply solves A z = r."""
    s = synth.system(40, 1, 1, 9, bs=1)
    d = oracle.decompose(s.row_ptr, s.col, s.val, (40, 1, 1), (40, 1, 1))
    r = np.random.default_rng(1).uniform(-1, 1, 40)
    z = oracle.apply(d.LU, r)
    A = _dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, 40)
    assert np.abs(z - np.linalg.solve(A, r)).max() <= 1e-13 * np.abs(z).max()


def test_scalar_one_row_subdomains_are_jacobi():
    s = synth.system(4, 3, 2, 11, bs=1)
    d = oracle.decompose(s.row_ptr, s.col, s.val, (4, 3, 2), (1, 1, 1))
    r = np.random.default_rng(2).uniform(-1, 1, s.n)
    diag = np.array([d.Ap.val.reshape(-1)[q] for i in range(s.n)
                     for q in range(d.Ap.row_ptr[i], d.Ap.row_ptr[i + 1]) if d.Ap.col[q] == i])
    assert np.array_equal(oracle.apply(d.LU, r), r / diag)


def test_scalar_spmv_is_dense_product():
    s = synth.system(5, 4, 3, 13, bs=1)
    A = oracle.BSR(s.row_ptr, s.col, s.val)
    x = np.random.default_rng(3).uniform(-1, 1, s.n)
    assert np.abs(oracle.spmv(A, x) - _dense(s.row_ptr, s.col, s.val, s.n) @ x).max() <= 1e-14
    assert np.abs(oracle.spmv(A, s.xstar) - s.b).max() == 0.0  # the generator's b, same order


def test_scalar_dot_order():
    """Rows of one entry: q_i = x_i y_i, halving sums in 256-row tiles, then over
    tiles. 2^53 at row 0 and 1.0 at rows 1 and 129 (the pair (1, 129) meets at
    the h = 128 level, then joins 2^53 last): 2^53 + 2 exactly; a left-to-right
    sum would give 2^53."""
    x = np.zeros(512)
    x[0], x[1], x[129] = 2.0 ** 53, 1.0, 1.0
    assert oracle.dot(x, np.ones(512), bs=1) == 2.0 ** 53 + 2.0
    assert sum(x) == 2.0 ** 53


def test_scalar_bicgstab_matches_scipy_iterates():
    grid, sub = (8, 8, 8), (4, 4, 4)
    s = synth.system(*grid, 17, model=synth.MODEL_LAYERED, bs=1)
    d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
    b = s.b[d.perm]
    A = sp.csr_matrix(_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, s.n))
    M = spla.LinearOperator((s.n, s.n), matvec=lambda v: oracle.apply(d.LU, np.ravel(v)))
    for k in (1, 2, 4):
        ours = oracle.bicgstab(d.Ap, d.LU, b, maxit=k, rtol=1e-30)
        ref, _ = spla.bicgstab(A, b, x0=np.zeros(s.n), rtol=1e-30, atol=0.0, maxiter=k, M=M)
        assert ours.iterations == k
        assert np.linalg.norm(ours.x - ref) <= 1e-9 * np.linalg.norm(ref)
    full = oracle.bicgstab(d.Ap, d.LU, b)
    assert full.status == 0 and full.rel_res_true < 1e-8


def test_block_size_from_flat_values():
    """Flat value arrays carry bs*bs entries per block: the oracle reads the
    block size from their length (a scalar matrix is never read as 3x3)."""
    s1 = synth.system(4, 3, 2, 3, bs=1)
    s3 = synth.system(4, 3, 2, 3)
    assert oracle.BSR(s1.row_ptr, s1.col, np.ravel(s1.val)).bs == 1
    assert oracle.BSR(s3.row_ptr, s3.col, np.ravel(s3.val)).bs == 3
    assert oracle.BSR(s3.row_ptr, s3.col, np.asarray(s3.val).reshape(-1, 3, 3)).bs == 3
    assert oracle.BSR(s1.row_ptr, s1.col, None, block=1).bs == 1
