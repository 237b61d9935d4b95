"""Empty input: a matrix with no rows (a graph partition of nothing) sets up,
applies, multiplies and solves without launching work, alone and inside a
batch beside a non-empty system, and reports what bicgstab_solve reports for
it: status OK, no iteration, residual 0."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402


def empty_ctx(prec):
    rp = np.zeros(1, np.int32)
    col = np.zeros(0, np.int32)
    val = np.zeros((0, 3, 3))
    return g.Ilu0DD(rp, col, val, part_id=np.zeros(0, np.int32), nparts=0, factor_prec=prec)


@pytest.mark.parametrize("prec", ["f64", "f32", "df64", "bf16"])
def test_empty_system(prec):
    ctx = empty_ctx(prec)
    try:
        assert ctx.query("n") == 0 and ctx.query("nsub") == 0 and ctx.query("kept") == 0
        v = torch.empty(0, dtype=torch.float64, device="cuda")
        assert ctx.apply(v).numel() == 0
        assert ctx.spmv(v).numel() == 0
        out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
        ctx.dot(v, v.clone(), out)
        assert out.item() == 0.0
        x, info = ctx.solve(v)
        assert x.numel() == 0 and info["status"] == 0 and info["iterations"] == 0
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_empty_system_in_a_batch():
    grid, sub = (8, 8, 8), (4, 4, 4)
    s = synth.system(*grid, 21)
    full = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub)
    empty = empty_ctx("f64")
    try:
        b = torch.from_numpy(s.b).cuda()
        x1, i1 = full.solve(b)
        batch = g.Batch([empty, full, empty])
        v = torch.empty(0, dtype=torch.float64, device="cuda")
        xs, infos = batch.solve([v, b, v])
        assert [i["status"] for i in infos] == [0, 0, 0]
        assert infos[0]["iterations"] == infos[2]["iterations"] == 0
        assert infos[1]["iterations"] == i1["iterations"] and torch.equal(xs[1], x1)
        assert xs[0].numel() == 0 and xs[2].numel() == 0
        batch.close()
    finally:
        full.close()
        empty.close()


def test_empty_system_takes_null_vectors_through_the_abi():
    """Null vector pointers are accepted for a system with no rows (there is
    nothing to read or write), as the header states for n_brows = 0."""
    ctx = empty_ctx("f64")
    try:
        lib = g.binding.load()
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert lib.ilu0_dd_apply(ctx._ctx, None, None, s) == 0
        assert lib.ilu0_dd_spmv(ctx._ctx, None, None, s) == 0
        assert lib.ilu0_dd_permute(ctx._ctx, None, None, 0, s) == 0
        torch.cuda.synchronize()
    finally:
        ctx.close()
