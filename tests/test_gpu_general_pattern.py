"""Rows with more blocks than the descriptor carries slot counts for.

The 7-point stencil gives at most three strictly-lower and three strictly-upper
blocks per row, which the piece descriptor covers; wider patterns take the
apply's general path (slots beyond the third read their counts from the
record). A 27-point block stencil (up to 13 blocks on each side of the
diagonal) exercises it: decomposition, levels, apply and BiCGSTAB against the
oracle, in every factor precision.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402


def stencil27(nx, ny, nz, seed):
    """Seeded 27-point 3x3-block system: off-diagonal blocks -0.05 I + U(-0.02, 0.02),
    diagonal blocks 6.5 I + U(-0.1, 0.1) (block diagonally dominant), b = A x*."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    rp, cols, vals = [0], [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = []
                for dk in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        for di in (-1, 0, 1):
                            a, b_, c = i + di, j + dj, k + dk
                            if 0 <= a < nx and 0 <= b_ < ny and 0 <= c < nz:
                                row.append(a + nx * (b_ + ny * c))
                for col in sorted(row):
                    if col == i + nx * (j + ny * k):
                        blk = 6.5 * np.eye(3) + rng.uniform(-0.1, 0.1, (3, 3))
                    else:
                        blk = -0.05 * np.eye(3) + rng.uniform(-0.02, 0.02, (3, 3))
                    cols.append(col)
                    vals.append(blk)
                rp.append(len(cols))
    rp = np.array(rp, np.int32)
    col = np.array(cols, np.int32)
    val = np.array(vals, np.float64)
    xs = rng.uniform(-1, 1, 3 * n)
    b = oracle.spmv(oracle.BSR(rp, col, val), xs)
    return rp, col, val, b, n


def nrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = [((6, 5, 4), (3, 3, 2)), ((8, 8, 8), (4, 4, 4)), ((9, 7, 5), (9, 7, 5))]


@pytest.mark.parametrize("grid,sub", CASES)
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("df64", 1e-12), ("f32", 1e-5), ("bf16", 5e-2)])
def test_wide_rows_apply_and_levels(grid, sub, prec, tol):
    rp, col, val, b, n = stencil27(*grid, seed=11)
    d = oracle.decompose(rp, col, val, grid, sub)
    rows = np.repeat(np.arange(n), np.diff(d.Add.row_ptr))
    assert (np.bincount(rows[d.Add.col < rows], minlength=n).max()) > 3  # the general path is taken
    ctx = g.Ilu0DD(rp, col, val, grid, sub, factor_prec=prec)
    try:
        assert np.array_equal(ctx.export(B.X_LEVEL_L), oracle.levels_lower(d.Add)[0])
        assert np.array_equal(ctx.export(B.X_LEVEL_U), oracle.levels_upper(d.Add)[0])
        r = np.random.default_rng(3).uniform(-1, 1, 3 * n)
        z = ctx.apply(torch.from_numpy(r).cuda()).cpu().numpy()
        assert nrel(z, oracle.apply(d.LU, r)) <= tol
    finally:
        ctx.close()


@pytest.mark.parametrize("grid,sub", CASES)
def test_wide_rows_bicgstab(grid, sub):
    rp, col, val, b, n = stencil27(*grid, seed=12)
    d = oracle.decompose(rp, col, val, grid, sub)
    ctx = g.Ilu0DD(rp, col, val, grid, sub)
    try:
        x, info = ctx.solve(torch.from_numpy(b).cuda())
        bp = b.reshape(-1, 3)[d.perm].reshape(-1)
        ref = oracle.bicgstab(d.Ap, d.LU, bp)
        assert info["status"] == 0 and info["iterations"] == ref.iterations
        xo = ref.x.reshape(-1, 3)[d.iperm].reshape(-1)
        assert nrel(x.cpu().numpy(), xo) <= 1e-12
    finally:
        ctx.close()


def test_wide_rows_batched_equals_single():
    """27-point systems (rows beyond the descriptor's slot counts): the batched
    solve gives the single-system solve's bits."""
    systems = [stencil27(8, 8, 8, seed=31), stencil27(9, 7, 5, seed=32)]
    grids = [((8, 8, 8), (4, 4, 4)), ((9, 7, 5), (9, 7, 5))]
    ctxs = [g.Ilu0DD(rp, col, val, grid, sub) for (rp, col, val, b, n), (grid, sub) in zip(systems, grids)]
    bs = [torch.from_numpy(b).cuda() for (rp, col, val, b, n) in systems]
    try:
        singles = [c.solve(b) for c, b in zip(ctxs, bs)]
        batch = g.Batch(ctxs)
        xs, infos = batch.solve(bs)
        for (x1, i1), x2, i2 in zip(singles, xs, infos):
            assert i1["iterations"] == i2["iterations"] and torch.equal(x1, x2)
        batch.close()
    finally:
        for c in ctxs:
            c.close()
