"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test names the passage it pins and what a plausible mistake would break.
All of these run on the CPU (no GPU marker).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth
from _dense import (block_mask, blocks_dense, bsr_to_dense, dense_block_ilu0, dense_scalar_ilu0,
                    local_coords, lu_to_dense)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _system(grid, seed=11, model=synth.MODEL_LAPLACE):
    return synth.system(*grid, seed, model=model)


def _dec(grid, sub, seed=11, model=synth.MODEL_LAPLACE):
    s = _system(grid, seed, model)
    return s, oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)


def _perm_vec(v, perm):
    return np.ascontiguousarray(np.asarray(v).reshape(-1, 3)[perm].reshape(-1))


# ---------------------------------------------------------------- Table 5 -----

def _table5_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table5_partition_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows.append((t[0], *map(int, t[1:11]), float(t[11])))
    return rows


@pytest.mark.parametrize("row", _table5_rows(), ids=lambda r: r[0])
def test_table5_partition_counts(row):
    """Table 5 (Section 5.3): nnz before/after the drop of Section 3.2, exactly.

    Pins Algorithm 2 (labels), Algorithm 3 (reorder keeps every block) and the
    drop rule; a wrong cut index or a drop of same-subdomain blocks changes the
    printed integers.
    """
    name, nx, ny, nz, sx, sy, sz, rows_per_sub, nsub, nnz, nnz_after, pct = row
    rp, col = synth.pattern(nx, ny, nz)
    d = oracle.decompose(rp, col, None, (nx, ny, nz), (sx, sy, sz), factor=False)
    assert oracle.nparts((nx, ny, nz), (sx, sy, sz)) == nsub
    assert np.all(np.diff(d.part_ptr) == rows_per_sub)
    assert 9 * d.Ap.nnzb == nnz
    assert 9 * d.Add.nnzb == nnz_after
    assert round(100.0 * (nnz - nnz_after) / nnz, 2) == pct
    # Table 2 prints the scalar row counts rounded to 0.1M
    assert {"laplacian1": 6.3, "laplacian2": 12.6}[name] == round(3 * nx * ny * nz / 1e6, 1)


# ---------------------------------------------------------- Algorithm 2 ------

@pytest.mark.parametrize("grid,sub", [((8, 6, 4), (4, 3, 2)), ((7, 5, 3), (4, 2, 2)), ((5, 1, 1), (2, 1, 1))])
def test_partition_boxes(grid, sub):
    """Algorithm 2: every label is an axis-aligned box of at most sx*sy*sz cells, labels
    enumerate boxes x-fastest, and edge boxes shrink on ragged grids (ceil-division)."""
    nx, ny, nz = grid
    part = oracle.partition(grid, sub)
    npart = oracle.nparts(grid, sub)
    assert part.min() == 0 and part.max() == npart - 1
    g = np.arange(nx * ny * nz)
    ii, jj, kk = g % nx, (g // nx) % ny, g // (nx * ny)
    bx, by = -(-nx // sub[0]), -(-ny // sub[1])
    for p in range(npart):
        cells = part == p
        ci, cj, ck = ii[cells], jj[cells], kk[cells]
        ext = (ci.max() - ci.min() + 1, cj.max() - cj.min() + 1, ck.max() - ck.min() + 1)
        assert cells.sum() == ext[0] * ext[1] * ext[2]  # a full box
        assert all(e <= s for e, s in zip(ext, sub))
        # box position enumerates x fastest, then y, then z
        assert (ci.min() // sub[0], cj.min() // sub[1], ck.min() // sub[2]) == (p % bx, (p // bx) % by, p // (bx * by))


# ---------------------------------------------------------- Algorithm 3 ------

def test_reorder_is_PAPt_and_groups_subdomains():
    """Algorithm 3 / Section 3.1: A_p = P A P^T, label groups contiguous, and
    ascending original order inside a group (the stable reading)."""
    grid, sub = (6, 5, 4), (3, 2, 2)
    s, d = _dec(grid, sub)
    n = s.n
    assert sorted(d.perm.tolist()) == list(range(n))
    assert np.array_equal(d.iperm[d.perm], np.arange(n))
    label = d.part_id[d.perm]
    for p in range(len(d.part_ptr) - 1):
        seg = slice(d.part_ptr[p], d.part_ptr[p + 1])
        assert np.all(label[seg] == p)
        assert np.all(np.diff(d.perm[seg]) > 0)
    A = bsr_to_dense(s.row_ptr, s.col, s.val, n)
    Ap = bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n)
    sperm = (3 * d.perm[:, None] + np.arange(3)).reshape(-1)
    assert np.array_equal(Ap, A[np.ix_(sperm, sperm)])
    for i in range(n):
        assert np.all(np.diff(d.Ap.col[d.Ap.row_ptr[i]:d.Ap.row_ptr[i + 1]]) > 0)


def test_drop_keeps_exactly_same_subdomain_blocks():
    """Section 3.2: A_dd = A_p masked to blocks whose row and column share a label;
    the kept count follows kept = N + 2 (faces - cut faces)."""
    grid, sub = (6, 5, 4), (3, 2, 2)
    s, d = _dec(grid, sub)
    n = s.n
    label = d.part_id[d.perm]
    Ap = bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n)
    Add = bsr_to_dense(d.Add.row_ptr, d.Add.col, d.Add.val, n)
    same = np.kron(label[:, None] == label[None, :], np.ones((3, 3), bool))
    assert np.array_equal(Add, np.where(same, Ap, 0.0))
    nx, ny, nz = grid
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    cut = ((-(-nx // sub[0]) - 1) * ny * nz + (-(-ny // sub[1]) - 1) * nx * nz
           + (-(-nz // sub[2]) - 1) * nx * ny)
    assert d.Add.nnzb == n + 2 * (faces - cut)


# ---------------------------------------------------------- Algorithm 7 ------

@pytest.mark.parametrize("grid,sub,model", [((6, 5, 4), (3, 5, 2), synth.MODEL_LAPLACE),
                                            ((5, 4, 4), (5, 2, 4), synth.MODEL_LAYERED)])
def test_ilu0_reproduces_A_on_pattern(grid, sub, model):
    """ILU0 defining property (Algorithm 7; Saad ch. 10): (L U)_ij = A_dd,ij for every
    block in the pattern of A_dd.  Any dropped or mis-signed update term breaks it."""
    s, d = _dec(grid, sub, model=model)
    n = s.n
    assert d.status == 0
    L, U = lu_to_dense(d.LU.row_ptr, d.LU.col, d.LU.val, n)
    Add = bsr_to_dense(d.Add.row_ptr, d.Add.col, d.Add.val, n)
    mask = np.kron(block_mask(d.Add.row_ptr, d.Add.col, n), np.ones((3, 3), bool))
    P = L @ U
    scale = np.abs(Add).max()
    assert np.abs((P - Add)[mask]).max() <= 1e-13 * scale


def test_one_subdomain_equals_global_block_ilu0():
    """One subdomain covering the grid is global ILU0: compare with a brute-force
    dense-block IKJ (textbook form) on a 4x4x4 grid."""
    grid = (4, 4, 4)
    s, d = _dec(grid, grid, model=synth.MODEL_LAYERED)
    n = s.n
    assert np.array_equal(d.perm, np.arange(n))
    W = dense_block_ilu0(blocks_dense(s.row_ptr, s.col, s.val, n), block_mask(s.row_ptr, s.col, n))
    got = blocks_dense(d.LU.row_ptr, d.LU.col, d.LU.val, n)
    mask = block_mask(s.row_ptr, s.col, n)
    scale = np.abs(W[mask]).max()
    assert np.abs((got - W)[mask]).max() <= 1e-13 * scale


def test_block_ilu0_equals_scalar_ilu0_action():
    """A 3x3-block ILU0 with dense blocks acts like scalar ILU0 on the expanded pattern
    (the two factorizations are equal in exact arithmetic)."""
    grid = (3, 3, 2)
    s, d = _dec(grid, grid)
    n = s.n
    A = bsr_to_dense(s.row_ptr, s.col, s.val, n)
    mask = np.kron(block_mask(s.row_ptr, s.col, n), np.ones((3, 3), bool))
    Ls, Us = dense_scalar_ilu0(A, mask)
    r = np.random.default_rng(0).uniform(-1, 1, 3 * n)
    z_scalar = np.linalg.solve(Us, np.linalg.solve(Ls, r))
    z = oracle.apply(d.LU, r)
    assert np.abs(z - z_scalar).max() <= 1e-12 * np.abs(z_scalar).max()


def test_chain_is_exact_lu():
    """A 1D chain (n x 1 x 1) in one subdomain has no fill: ILU0 is the exact LU, so
    M^-1 b equals the dense solve, and BiCGSTAB stops after one iteration."""
    grid = (40, 1, 1)
    s, d = _dec(grid, grid)
    n = s.n
    A = bsr_to_dense(s.row_ptr, s.col, s.val, n)
    z = oracle.apply(d.LU, s.b)
    ref = np.linalg.solve(A, s.b)
    assert np.abs(z - ref).max() <= 1e-13 * np.abs(ref).max()
    res = oracle.bicgstab(d.Ap, d.LU, s.b)
    assert res.status == oracle.OK and res.iterations == 1
    assert np.abs(res.x - s.xstar).max() <= 1e-12


def test_one_cell_subdomains_are_block_jacobi():
    """1x1x1 subdomains drop every coupling: M^-1 r = D_A^-1 r (block Jacobi) and every
    row sits on level 0 of both DAGs."""
    grid = (4, 3, 2)
    s, d = _dec(grid, (1, 1, 1))
    n = s.n
    assert d.Add.nnzb == n
    r = np.random.default_rng(1).uniform(-1, 1, 3 * n)
    z = oracle.apply(d.LU, r)
    for i in range(n):
        blk = d.Ap.val[d.Ap.row_ptr[i]:d.Ap.row_ptr[i + 1]][d.Ap.col[d.Ap.row_ptr[i]:d.Ap.row_ptr[i + 1]] == i][0]
        ref = np.linalg.solve(blk, r[3 * i:3 * i + 3])
        assert np.abs(z[3 * i:3 * i + 3] - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())
    assert oracle.levels_lower(d.Add)[1] == 1 and oracle.levels_upper(d.Add)[1] == 1


# ---------------------------------------------------------- Algorithm 5 ------

def _alg5_fixed_point(rp, col, lo, hi):
    """Algorithm 5 as an iteration (levels raised until nothing changes), for one subdomain."""
    nrows = hi - lo
    hmap = np.full(nrows, nrows + 1)
    for i in range(lo, hi):
        if not any(c < i for c in col[rp[i]:rp[i + 1]]):
            hmap[i - lo] = 0
    level = 0
    while True:
        marked = []
        for i in range(lo, hi):
            if hmap[i - lo] > level and all(hmap[c - lo] <= level for c in col[rp[i]:rp[i + 1]] if c < i):
                marked.append(i)
        for i in marked:
            hmap[i - lo] = level + 1
        if not marked:
            break
        level += 1
    return hmap


@pytest.mark.parametrize("grid,sub", [((8, 8, 4), (4, 4, 2)), ((6, 6, 6), (3, 2, 6))])
def test_levels_closed_form_and_alg5(grid, sub):
    """Level sets (Algorithm 5 and its reverse for U): in a box subdomain in natural
    order the L level of local cell (a,b,c) is a+b+c and the U level is
    (sx-1-a)+(sy-1-b)+(sz-1-c); there are sx+sy+sz-2 levels; Algorithm 5's iteration
    reaches the same levels."""
    s, d = _dec(grid, sub)
    a, b, c = local_coords(grid, sub, d.perm, d.part_ptr)
    lo, nl = oracle.levels_lower(d.Add)
    up, nu = oracle.levels_upper(d.Add)
    assert np.array_equal(lo, a + b + c)
    assert np.array_equal(up, (sub[0] - 1 - a) + (sub[1] - 1 - b) + (sub[2] - 1 - c))
    assert nl == nu == sum(sub) - 2
    p0, p1 = d.part_ptr[0], d.part_ptr[1]
    assert np.array_equal(_alg5_fixed_point(d.Add.row_ptr, d.Add.col, p0, p1), lo[p0:p1])


# ---------------------------------------------------------- apply ------------

def test_apply_inverts_LU_and_stays_in_subdomain():
    """M^-1 (L U z) = z, and r supported on one subdomain maps to z supported on
    that subdomain only (no inter-subdomain coupling survives the drop)."""
    grid, sub = (6, 6, 4), (3, 3, 2)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    n = s.n
    L, U = lu_to_dense(d.LU.row_ptr, d.LU.col, d.LU.val, n)
    z = np.random.default_rng(2).uniform(-1, 1, 3 * n)
    w = L @ (U @ z)
    assert np.abs(oracle.apply(d.LU, w) - z).max() <= 1e-11
    r = np.zeros(3 * n)
    p = 2
    r[3 * d.part_ptr[p]:3 * d.part_ptr[p + 1]] = 1.0
    zz = oracle.apply(d.LU, r)
    outside = np.ones(3 * n, bool)
    outside[3 * d.part_ptr[p]:3 * d.part_ptr[p + 1]] = False
    assert np.all(zz[outside] == 0.0) and np.abs(zz[~outside]).max() > 0


# ---------------------------------------------------------- SpMV, dot ---------

def test_spmv_dense_and_generator():
    """y = A x against a dense matvec; on the natural-order matrix the oracle's
    fixed per-row order reproduces the generator's b = A x* bit for bit."""
    grid, sub = (5, 4, 3), (2, 2, 3)
    s, d = _dec(grid, sub)
    n = s.n
    A = bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n)
    x = np.random.default_rng(3).uniform(-1, 1, 3 * n)
    assert np.abs(oracle.spmv(d.Ap, x) - A @ x).max() <= 1e-14 * np.abs(A).sum(1).max()
    An = oracle.BSR(s.row_ptr, s.col, s.val)
    assert np.array_equal(oracle.spmv(An, s.xstar), s.b)


def test_dot_order_pins():
    """The fixed dot order: per-row FMA, halving sum within 256-row tiles, halving
    sum over tiles.  Crafted values where only that order gives 2^53 + 2."""
    n = 512
    x = np.zeros(3 * n)
    y = np.ones(3 * n)
    x[0] = 2.0 ** 53          # row 0 of tile 0
    x[3 * 1] = 1.0            # row 1
    x[3 * 129] = 1.0          # row 129 pairs with row 1 at the first halving step
    assert oracle.dot(x, y) == 2.0 ** 53 + 2.0
    # sequential or recursive-pairwise summation would lose both ones:
    assert math.fsum([2.0 ** 53, 1.0]) + 1.0 == 2.0 ** 53
    # tiles combine by halving too: tiles 0 and 2 pair first when there are 4 tiles
    x = np.zeros(3 * 1024)
    x[0] = 2.0 ** 53
    x[3 * 256] = 1.0          # tile 1
    x[3 * 768] = 1.0          # tile 3 pairs with tile 1
    assert oracle.dot(x, np.ones_like(x)) == 2.0 ** 53 + 2.0


@pytest.mark.parametrize("n", [1, 255, 256, 257, 1000, 4096 + 7])
def test_dot_accuracy(n):
    """Against an exactly rounded sum (math.fsum of exact products is not available, so
    compare with fsum of the rounded products within the pairwise error bound) and
    exactly on small integers."""
    rng = np.random.default_rng(n)
    x = rng.uniform(-1, 1, 3 * n)
    y = rng.uniform(-1, 1, 3 * n)
    ref = math.fsum((x * y).tolist())
    bound = (2 + math.log2(max(2, n)) + 9) * 2.0 ** -53 * float(np.abs(x * y).sum()) + 1e-300
    assert abs(oracle.dot(x, y) - ref) <= bound
    xi = rng.integers(-1000, 1000, 3 * n).astype(float)
    yi = rng.integers(-1000, 1000, 3 * n).astype(float)
    assert oracle.dot(xi, yi) == float(np.dot(xi.astype(np.int64), yi.astype(np.int64)))


# ---------------------------------------------------------- Algorithm 1 ------

def test_bicgstab_matches_scipy_iterates():
    """Algorithm 1 with M = LU, x0 = 0: the first k iterates equal SciPy's preconditioned
    BiCGSTAB (same method, independent code) up to rounding."""
    grid, sub = (8, 8, 8), (4, 4, 4)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    n = s.n
    b = _perm_vec(s.b, d.perm)
    A = sp.csr_matrix(bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n))
    M = spla.LinearOperator((3 * n, 3 * n), matvec=lambda v: oracle.apply(d.LU, np.ravel(v)))
    for k in (1, 2, 4):
        ours = oracle.bicgstab(d.Ap, d.LU, b, maxit=k, rtol=1e-30)
        ref, _ = spla.bicgstab(A, b, x0=np.zeros(3 * n), rtol=1e-30, atol=0.0, maxiter=k, M=M)
        assert ours.iterations == k
        assert np.linalg.norm(ours.x - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("grid,sub,model", [((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),
                                            ((16, 16, 16), (16, 16, 8), synth.MODEL_LAYERED)])
def test_bicgstab_converges(grid, sub, model):
    """Algorithm 1 reaches ||b - A x|| / ||b|| < 1e-8, the recurrence residual tracks
    the true one, and x approaches x* as far as the conditioning allows."""
    s, d = _dec(grid, sub, seed=1, model=model)
    b = _perm_vec(s.b, d.perm)
    res = oracle.bicgstab(d.Ap, d.LU, b)
    assert res.status == oracle.OK and res.restarts == 0
    assert res.rel_res_true < 1e-8 and res.rel_res_recurrence < 1e-8
    assert abs(res.rel_res_true - res.rel_res_recurrence) <= 1e-3 * res.rel_res_recurrence + 1e-15
    x = _perm_vec(res.x, d.iperm)
    tol = 1e-6 if model == synth.MODEL_LAPLACE else 1e-3
    assert np.linalg.norm(x - s.xstar) <= tol * np.linalg.norm(s.xstar)
    assert len(res.history) == res.iterations + 1 and res.history[0] == 1.0


def test_bicgstab_breakdown_and_zero_rhs():
    """b = 0 returns x = 0 at once; maxit exhaustion reports NOT_CONVERGED."""
    grid, sub = (4, 4, 4), (2, 2, 2)
    s, d = _dec(grid, sub)
    res = oracle.bicgstab(d.Ap, d.LU, np.zeros(3 * s.n))
    assert res.status == oracle.OK and res.iterations == 0 and not res.x.any()
    res = oracle.bicgstab(d.Ap, d.LU, _perm_vec(s.b, d.perm), maxit=2, rtol=1e-30)
    assert res.status == oracle.NOT_CONVERGED and res.iterations == 2


def test_zero_pivot_detected():
    """A singular diagonal block stops ILU0 with the failing row."""
    grid, sub = (3, 2, 1), (3, 2, 1)
    s = _system(grid)
    val = s.val.copy()
    diag_q = [q for q in range(s.row_ptr[0], s.row_ptr[1]) if s.col[q] == 0][0]
    val[diag_q] = 0.0
    d = oracle.decompose(s.row_ptr, s.col, val, grid, sub)
    assert d.status == -1
