"""The vendor baseline (cuSPARSE global block ILU0) against the oracle.

With one subdomain covering the whole grid, Algorithm 3's permutation is the
identity and Section 3.2 drops nothing, so the oracle's block ILU0 (Algorithm
7) is the global ILU0 that cuSPARSE's bsrilu02 computes on the same pattern.
The two store the factors differently (cuSPARSE runs scalar ILU0 on the
expanded pattern), so their products and their triangular solves must agree
to rounding. This checks the oracle against a library routine and the vendor
baseline's setup at once.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import context  # noqa: E402


def _vendor_dense_factors(s, f):
    """cuSPARSE's bsrilu02 is scalar ILU0 on the expanded block pattern: the
    diagonal block holds its own packed unit-lower / upper LU, blocks left of it
    belong to L and blocks right of it to U (all row-major)."""
    n = s.n
    L, U = np.eye(3 * n), np.zeros((3 * n, 3 * n))
    f = f.reshape(-1, 3, 3)
    for i in range(n):
        for q in range(s.row_ptr[i], s.row_ptr[i + 1]):
            j = s.col[q]
            bi, bj = slice(3 * i, 3 * i + 3), slice(3 * j, 3 * j + 3)
            if j < i:
                L[bi, bj] = f[q]
            elif j > i:
                U[bi, bj] = f[q]
            else:
                L[bi, bj] = np.tril(f[q], -1) + np.eye(3)
                U[bi, bj] = np.triu(f[q])
    return L, U


@pytest.mark.parametrize("model", [synth.MODEL_LAPLACE, synth.MODEL_LAYERED])
def test_vendor_global_ilu0_product_matches_oracle(model):
    """L U of the vendor factors equals L U of the oracle's block factors (one
    subdomain = the whole grid), entry by entry, fill positions included."""
    grid = (6, 5, 4)
    s = synth.system(*grid, 41, model=model)
    d = oracle.decompose(s.row_ptr, s.col, s.val, grid, grid)
    assert np.array_equal(d.perm, np.arange(s.n))
    assert np.array_equal(d.LU.col, s.col) and np.array_equal(d.LU.row_ptr, s.row_ptr)
    v = context.VendorIlu0(s.row_ptr, s.col, s.val)
    try:
        Lv, Uv = _vendor_dense_factors(s, v.factors())
    finally:
        v.close()
    Lo, Uo = np.eye(3 * s.n), np.zeros((3 * s.n, 3 * s.n))
    for i in range(s.n):
        for q in range(d.LU.row_ptr[i], d.LU.row_ptr[i + 1]):
            j = d.LU.col[q]
            (Lo if j < i else Uo)[3 * i:3 * i + 3, 3 * j:3 * j + 3] = d.LU.val[q]
    Mo = Lo @ Uo
    assert np.abs(Lv @ Uv - Mo).max() <= 1e-12 * np.abs(Mo).max()


@pytest.mark.parametrize("grid,model", [((12, 10, 9), synth.MODEL_LAPLACE), ((16, 16, 8), synth.MODEL_LAYERED)])
def test_vendor_apply_and_spmv_match_oracle(grid, model):
    s = synth.system(*grid, 41, model=model)
    d = oracle.decompose(s.row_ptr, s.col, s.val, grid, grid)
    v = context.VendorIlu0(s.row_ptr, s.col, s.val)
    try:
        r = np.random.default_rng(7).uniform(-1, 1, 3 * s.n)
        rd = torch.from_numpy(r).cuda()
        z = torch.empty_like(rd)
        v.apply(rd, z)
        zo = oracle.apply(d.LU, r)
        assert np.abs(z.cpu().numpy() - zo).max() <= 1e-12 * np.abs(zo).max()
        y = torch.empty_like(rd)
        v.spmv(rd, y)
        yo = oracle.spmv(oracle.BSR(s.row_ptr, s.col, s.val), r)
        assert np.abs(y.cpu().numpy() - yo).max() <= 1e-14 * np.abs(yo).max()
    finally:
        v.close()


def test_fp64_fma_rate_is_sane():
    g = context.fp64_fma_gflops(256)
    assert 10.0 < g < 1e5
