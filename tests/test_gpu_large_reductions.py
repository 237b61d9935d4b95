"""Fixed-order reductions at sizes where the final fold over tile partials has
16 or more partials per thread of the finishing block (over 1M block rows),
which runs the depth-first evaluation of the halving sum. They must still
match the oracle bit for bit: dot products through the allocation-free entry
point and through a context, and a full BiCGSTAB at 1M rows, whose every
iteration reduces two dots in the SpMV and two in the update that way.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402


@pytest.mark.parametrize("rows", [600_000, 1_048_576, 2_100_000, 4_194_304])
def test_large_noalloc_dot_matches_oracle(rows):
    lib = g.load()
    rng = np.random.default_rng(rows)
    x = rng.normal(size=3 * rows)
    y = rng.normal(size=3 * rows) * 1e3
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.ilu0dd_dot_noalloc(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), ctypes.c_int64(rows),
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert out.item() == oracle.dot(x, y)


def test_large_context_dot_matches_oracle():
    """160^3 system: 16,000 tiles padded to 16,384, 64 partials per thread."""
    s = synth.system(160, 160, 160, 3, model=synth.MODEL_LAYERED)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, (160, 160, 160), (16, 16, 8))
    try:
        rng = np.random.default_rng(9)
        x, y = rng.normal(size=3 * s.n), rng.normal(size=3 * s.n)
        assert ctx.dot(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).item() == oracle.dot(x, y)
    finally:
        ctx.close()


def test_bicgstab_million_rows_matches_oracle():
    grid, sub = (100, 100, 100), (16, 16, 8)
    s = synth.system(*grid, 2)
    d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub)
    try:
        x, info = ctx.solve(torch.from_numpy(s.b).cuda())
        ref = oracle.bicgstab(d.Ap, d.LU, s.b.reshape(-1, 3)[d.perm].reshape(-1))
        assert info["status"] == 0 and info["iterations"] == ref.iterations
        hist = ctx.history(info["iterations"] + 1)
        assert np.allclose(hist, ref.history, rtol=1e-6, atol=1e-13)
        xo = ref.x.reshape(-1, 3)[d.iperm].reshape(-1)
        assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * np.abs(xo).max()
    finally:
        ctx.close()
