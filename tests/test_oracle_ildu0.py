"""Pins of the oracle's ILDU0 form, its restart branch, its initial guess and
its OpenMP build, against facts fixed by the paper and by mathematics.

The ILDU0 form (Algorithm 7 with the post-processing of Section 4.3) is the
arithmetic the fused apply performs: L, the explicitly stored inverses
inv_D = U_ii^-1 and U~ = inv_D U. It is pinned here against the ILU0 form
(pinned on its own in test_oracle_pins.py), against dense linear algebra,
against exact inverses and against SciPy's BiCGSTAB. CPU only.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth
from _dense import block_mask, bsr_to_dense, lu_to_dense


def _dec(grid, sub, seed=11, model=synth.MODEL_LAPLACE):
    s = synth.system(*grid, seed, model=model)
    return s, oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)


def _perm_vec(v, perm):
    return np.ascontiguousarray(np.asarray(v).reshape(-1, 3)[perm].reshape(-1))


def _ildu_dense(M: oracle.ILDU, n):
    """Dense L (unit diagonal), D (= inv(inv_D), via numpy) and U~ (unit diagonal)."""
    bs = M.F.bs
    L = np.eye(bs * n)
    Ut = np.eye(bs * n)
    for i in range(n):
        for q in range(M.F.row_ptr[i], M.F.row_ptr[i + 1]):
            j = M.F.col[q]
            tgt = L if j < i else (Ut if j > i else None)
            if tgt is not None:
                tgt[bs * i:bs * i + bs, bs * j:bs * j + bs] = M.F.val[q]
    D = np.zeros((bs * n, bs * n))
    for i in range(n):
        D[bs * i:bs * i + bs, bs * i:bs * i + bs] = np.linalg.inv(M.inv_d[i])
    return L, D, Ut


# ---------------------------------------------------------------- inverse ----

def test_inverse_exact_on_representable_cases():
    """Gauss-Jordan with partial pivoting returns the exact inverse wherever every
    step is exact: a permutation (pivoting needed: zero leading entries), scaled
    permutations by powers of two, and a triangular matrix with power-of-two
    pivots and binary-fraction entries."""
    P = np.array([[0.0, 1, 0], [0, 0, 1], [1, 0, 0]])
    assert np.array_equal(oracle.inverse(P), P.T)
    S = np.array([[0.0, 2, 0], [0, 0, 0.25], [8, 0, 0]])
    assert np.array_equal(oracle.inverse(S), np.array([[0, 0, 0.125], [0.5, 0, 0], [0, 4, 0]]))
    U = np.array([[2.0, 1, 0], [0, 4, 2], [0, 0, 8]])
    assert np.array_equal(oracle.inverse(U), np.array([[0.5, -0.125, 0.03125], [0, 0.25, -0.0625], [0, 0, 0.125]]))
    assert np.array_equal(oracle.inverse(np.array([[4.0]])), np.array([[0.25]]))


def test_inverse_against_numpy_and_failures():
    """Random well-conditioned 3x3 blocks: within a few ulps of LAPACK's inverse (via
    numpy), M X = I; singular, zero-column and non-finite blocks are refused."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        M = rng.uniform(-1, 1, (3, 3)) + 3 * np.eye(3) * rng.choice([-1, 1])
        X = oracle.inverse(M)
        ref = np.linalg.inv(M)
        assert np.abs(X - ref).max() <= 1e-14 * np.abs(ref).max()
        assert np.abs(M @ X - np.eye(3)).max() <= 1e-14
    assert oracle.inverse(np.array([[1.0, 2, 3], [2, 4, 6], [1, 0, 1]])) is None
    assert oracle.inverse(np.array([[0.0, 1, 2], [0, 3, 4], [0, 5, 6]])) is None
    assert oracle.inverse(np.array([[np.nan, 0, 0], [0, 1, 0], [0, 0, 1]])) is None
    assert oracle.inverse(np.array([[0.0]])) is None


# ---------------------------------------------------------------- factors ----

@pytest.mark.parametrize("grid,sub,model", [((6, 5, 4), (3, 5, 2), synth.MODEL_LAPLACE),
                                            ((5, 4, 4), (5, 2, 4), synth.MODEL_LAYERED)])
def test_ildu0_is_ilu0_rescaled(grid, sub, model):
    """Section 4.3: the ILDU0 factors are the ILU0 factors with the diagonal taken
    out of U: same L, inv_D_i U_ii = I, U~_ik = inv_D_i U_ik, and L D U~ reproduces
    A_dd on its pattern (the ILU0 property).  Scaling the lower blocks instead,
    multiplying by inv_D from the right, or dropping an update term breaks one."""
    s, d = _dec(grid, sub, model=model)
    n = s.n
    M = d.ildu()
    Lo, Uo = lu_to_dense(d.LU.row_ptr, d.LU.col, d.LU.val, n)
    L, D, Ut = _ildu_dense(M, n)
    scale_l = np.abs(Lo).max()
    assert np.abs(L - Lo).max() <= 1e-13 * scale_l
    for i in range(n):
        Uii = Uo[3 * i:3 * i + 3, 3 * i:3 * i + 3]
        assert np.abs(M.inv_d[i] @ Uii - np.eye(3)).max() <= 1e-13
    Ut_ref = np.zeros_like(Uo)
    for i in range(n):
        Ut_ref[3 * i:3 * i + 3] = M.inv_d[i] @ Uo[3 * i:3 * i + 3]
    off = ~np.kron(np.eye(n, dtype=bool), np.ones((3, 3), bool))
    assert np.abs((Ut - Ut_ref)[off]).max() <= 1e-13 * np.abs(Ut_ref[off]).max()
    Add = bsr_to_dense(d.Add.row_ptr, d.Add.col, d.Add.val, n)
    mask = np.kron(block_mask(d.Add.row_ptr, d.Add.col, n), np.ones((3, 3), bool))
    P = L @ D @ Ut
    assert np.abs((P - Add)[mask]).max() <= 1e-13 * np.abs(Add).max()
    # the diagonal positions of F hold zeros (the unit diagonal is implied)
    for i in range(n):
        q = [q for q in range(M.F.row_ptr[i], M.F.row_ptr[i + 1]) if M.F.col[q] == i][0]
        assert not M.F.val[q].any()


def test_ildu0_scalar_blocks():
    """bs = 1 (scalar CSR): inv_D_i = 1 / U_ii (a 1x1 Gauss-Jordan step is the
    reciprocal: exact against 1 / A_ii on rows without lower entries, where
    U_ii = A_ii) and U~_ik = inv_D_i U_ik, as Algorithm 7's post-processing writes
    it; elsewhere within rounding of the ILU0 form's U."""
    grid, sub = (6, 5, 4), (3, 5, 2)
    s = synth.system(*grid, 3, model=synth.MODEL_LAYERED, bs=1)
    d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
    M = d.ildu()
    n = s.n
    exact_rows = 0
    for i in range(n):
        lo, hi = d.LU.row_ptr[i], d.LU.row_ptr[i + 1]
        cols = d.LU.col[lo:hi]
        uii = d.LU.val[lo:hi][cols == i][0, 0, 0]
        if not np.any(cols < i):
            aii = d.Add.val[lo:hi][cols == i][0, 0, 0]
            assert M.inv_d[i, 0, 0] == 1.0 / aii
            exact_rows += 1
            for q in range(lo, hi):
                if cols[q - lo] > i:
                    assert M.F.val[q, 0, 0] == M.inv_d[i, 0, 0] * d.Add.val[q, 0, 0]
        assert abs(M.inv_d[i, 0, 0] - 1.0 / uii) <= 1e-14 * abs(1.0 / uii)
        for q in range(lo, hi):
            if cols[q - lo] > i:
                want = d.LU.val[q, 0, 0] / uii
                assert abs(M.F.val[q, 0, 0] - want) <= 1e-13 * abs(want)
    assert exact_rows == len(d.part_ptr) - 1  # one corner row per box subdomain


def test_ildu0_zero_pivot():
    """A singular diagonal block stops the factorization with the failing row."""
    grid, sub = (3, 2, 1), (3, 2, 1)
    s = synth.system(*grid, 11)
    val = s.val.copy()
    dq = [q for q in range(s.row_ptr[0], s.row_ptr[1]) if s.col[q] == 0][0]
    val[dq] = 0.0
    d = oracle.decompose(s.row_ptr, s.col, val, grid, sub, factor=False)
    _, st = oracle.ildu0(d.Add, d.part_ptr)
    assert st == -1


# ---------------------------------------------------------------- apply ------

@pytest.mark.parametrize("grid,sub,model", [((8, 8, 6), (4, 4, 3), synth.MODEL_LAYERED),
                                            ((7, 5, 3), (4, 2, 2), synth.MODEL_LAPLACE)])
def test_apply_ildu0_equals_ilu0_form(grid, sub, model):
    """Both forms compute M^-1 r of the same M (Section 4.3): equal to rounding, and
    the ILDU0 apply inverts L D U~ (a dense product)."""
    s, d = _dec(grid, sub, model=model)
    n = s.n
    M = d.ildu()
    r = np.random.default_rng(4).uniform(-1, 1, 3 * n)
    z = oracle.apply_ildu0(M, r)
    ref = oracle.apply(d.LU, r)
    assert np.abs(z - ref).max() <= 1e-13 * np.abs(ref).max()
    L, D, Ut = _ildu_dense(M, n)
    w = L @ (D @ (Ut @ r))
    assert np.abs(oracle.apply_ildu0(M, w) - r).max() <= 1e-11


def test_apply_ildu0_chain_block_jacobi_and_locality():
    """1D chain in one subdomain: exact LU, so the apply is the dense solve.  One-cell
    subdomains: block Jacobi.  r on one subdomain: z on that subdomain only."""
    grid = (40, 1, 1)
    s, d = _dec(grid, grid)
    A = bsr_to_dense(s.row_ptr, s.col, s.val, s.n)
    ref = np.linalg.solve(A, s.b)
    assert np.abs(oracle.apply_ildu0(d.ildu(), s.b) - ref).max() <= 1e-13 * np.abs(ref).max()
    grid = (4, 3, 2)
    s, d = _dec(grid, (1, 1, 1))
    r = np.random.default_rng(1).uniform(-1, 1, 3 * s.n)
    z = oracle.apply_ildu0(d.ildu(), r)
    for i in range(s.n):
        lo, hi = d.Ap.row_ptr[i], d.Ap.row_ptr[i + 1]
        blk = d.Ap.val[lo:hi][d.Ap.col[lo:hi] == i][0]
        want = np.linalg.solve(blk, r[3 * i:3 * i + 3])
        assert np.abs(z[3 * i:3 * i + 3] - want).max() <= 1e-14 * max(1.0, np.abs(want).max())
    grid, sub = (6, 6, 4), (3, 3, 2)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    r = np.zeros(3 * s.n)
    p = 2
    seg = slice(3 * d.part_ptr[p], 3 * d.part_ptr[p + 1])
    r[seg] = 1.0
    z = oracle.apply_ildu0(d.ildu(), r)
    outside = np.ones(3 * s.n, bool)
    outside[seg] = False
    assert np.all(z[outside] == 0.0) and np.abs(z[seg]).max() > 0


# ---------------------------------------------------------------- Algorithm 1

def test_bicgstab_ildu0_matches_scipy_iterates():
    """Algorithm 1 with the ILDU0-form M: the first k iterates equal SciPy's
    preconditioned BiCGSTAB with the same operator (independent code)."""
    grid, sub = (8, 8, 8), (4, 4, 4)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    n = s.n
    b = _perm_vec(s.b, d.perm)
    M = d.ildu()
    A = sp.csr_matrix(bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n))
    op = spla.LinearOperator((3 * n, 3 * n), matvec=lambda v: oracle.apply_ildu0(M, np.ravel(v)))
    for k in (1, 2, 5):
        ours = oracle.bicgstab(d.Ap, M, b, maxit=k, rtol=1e-30)
        ref, _ = spla.bicgstab(A, b, x0=np.zeros(3 * n), rtol=1e-30, atol=0.0, maxiter=k, M=op)
        assert ours.iterations == k
        assert np.linalg.norm(ours.x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_bicgstab_initial_guess_matches_scipy():
    """Algorithm 1 takes x0: r0 = b - A x0, r^ = r0, p = r0.  The oracle's iterates
    from a nonzero x0 equal SciPy's from the same x0, and hist[0] = ||r0|| / ||b||."""
    grid, sub = (8, 8, 4), (4, 4, 4)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    n = s.n
    b = _perm_vec(s.b, d.perm)
    M = d.ildu()
    A = sp.csr_matrix(bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n))
    op = spla.LinearOperator((3 * n, 3 * n), matvec=lambda v: oracle.apply_ildu0(M, np.ravel(v)))
    x0 = np.random.default_rng(9).uniform(-2, 2, 3 * n)
    for k in (1, 3, 6):
        ours = oracle.bicgstab(d.Ap, M, b, maxit=k, rtol=1e-30, x0=x0)
        ref, _ = spla.bicgstab(A, b, x0=x0.copy(), rtol=1e-30, atol=0.0, maxiter=k, M=op)
        assert np.linalg.norm(ours.x - ref) <= 1e-9 * np.linalg.norm(ref)
    res = oracle.bicgstab(d.Ap, M, b, maxit=1, rtol=1e-30, x0=x0)
    r0 = b - A @ x0
    assert abs(res.history[0] - np.linalg.norm(r0) / np.linalg.norm(b)) <= 1e-13 * res.history[0]


def test_restart_branch():
    """The true-residual restart (Algorithm 1 plus the restart reading): from an
    initial guess 1e8 times the solution's size the recurrence reaches rtol while
    b - A x (rounding floor about eps ||A|| ||x0||) still misses it, so the solve
    restarts once from the true residual (r = r^ = p = b - A x, rho = r^ . r) and
    the iteration count carries on.  Checked three ways: the run after the restart
    is bit for bit a fresh run started at the restart point; the count is the sum
    of the two legs (no iteration counted twice); and the continued iterates equal
    SciPy's BiCGSTAB started at the restart point (independent code)."""
    grid, sub = (8, 8, 8), (4, 4, 4)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    n = s.n
    b = _perm_vec(s.b, d.perm)
    M = d.ildu()
    rtol = 1e-8
    x0 = np.random.default_rng(5).uniform(-1, 1, 3 * n) * 1e8
    full = oracle.bicgstab(d.Ap, M, b, rtol=rtol, x0=x0)
    assert full.status == oracle.OK and full.restarts == 1 and full.rel_res_true < rtol
    # the first leg ends at the first recurrence residual below rtol
    j1 = int(np.argmax(full.history < rtol))
    assert 0 < j1 < full.iterations
    leg1 = oracle.bicgstab(d.Ap, M, b, rtol=rtol, x0=x0, maxit=j1)
    assert leg1.iterations == j1 and leg1.status == oracle.NOT_CONVERGED and leg1.restarts == 1
    assert leg1.rel_res_true >= rtol  # the true residual missed rtol there
    assert np.array_equal(leg1.history, full.history[:j1 + 1])
    # second leg: a fresh solve from the restart point gives the same bits
    leg2 = oracle.bicgstab(d.Ap, M, b, rtol=rtol, x0=leg1.x)
    assert leg2.restarts == 0 and leg2.status == oracle.OK
    assert full.iterations == j1 + leg2.iterations
    assert np.array_equal(full.x, leg2.x)
    assert np.array_equal(full.history[j1 + 1:], leg2.history[1:])
    # and SciPy, started at the restart point, follows the same iterates
    A = sp.csr_matrix(bsr_to_dense(d.Ap.row_ptr, d.Ap.col, d.Ap.val, n))
    op = spla.LinearOperator((3 * n, 3 * n), matvec=lambda v: oracle.apply_ildu0(M, np.ravel(v)))
    for k in (1, 3):
        ours = oracle.bicgstab(d.Ap, M, b, rtol=1e-30, x0=leg1.x, maxit=k)
        ref, _ = spla.bicgstab(A, b, x0=leg1.x.copy(), rtol=1e-30, atol=0.0, maxiter=k, M=op)
        assert np.linalg.norm(ours.x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_restart_that_still_misses_reports_not_converged():
    """One restart at most: with rtol below the true residual's rounding floor
    (1e-16 here), the recurrence converges twice, the true residual misses both
    times, and the solve reports NOT_CONVERGED with one restart."""
    grid, sub = (6, 6, 6), (3, 3, 3)
    s, d = _dec(grid, sub, model=synth.MODEL_LAYERED)
    b = _perm_vec(s.b, d.perm)
    res = oracle.bicgstab(d.Ap, d.ildu(), b, rtol=1e-16, maxit=3000)
    assert res.restarts == 1 and res.status == oracle.NOT_CONVERGED
    assert res.rel_res_recurrence < 1e-16 <= res.rel_res_true
    assert res.iterations < 3000


# ---------------------------------------------------------------- OpenMP -----

def test_openmp_build_is_bit_identical():
    """The OpenMP build (threads over subdomains, rows and dot tiles) gives the
    single-thread build's bits: factors, applies, SpMV, dots and whole solves
    in both preconditioner forms."""
    grid, sub = (16, 16, 12), (8, 8, 4)
    s = synth.system(*grid, 3, model=synth.MODEL_LAYERED)
    rng = np.random.default_rng(2)
    r = rng.uniform(-1, 1, 3 * s.n)
    out = {}
    try:
        for k in (1, 4):
            oracle.set_threads(k)
            d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
            M = d.ildu()
            b = _perm_vec(s.b, d.perm)
            out[k] = (M.F.val.copy(), M.inv_d.copy(), oracle.apply_ildu0(M, r), oracle.apply(d.LU, r),
                      oracle.spmv(d.Ap, r), np.array([oracle.dot(r, b)]),
                      oracle.bicgstab(d.Ap, M, b).x, oracle.bicgstab(d.Ap, d.LU, b).history)
    finally:
        oracle.set_threads(1)
    for a, c in zip(out[1], out[4]):
        assert np.array_equal(a, c)
