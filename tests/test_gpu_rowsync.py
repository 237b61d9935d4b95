"""The apply with Algorithm 4's synchronization (one completion flag per row,
each row waiting for exactly the rows it reads) against the level-ordered
apply and the oracle.

Both run the same per-row arithmetic in the same order on the same packed
stream; only when a row may start differs. So the results are bit-identical
in every factor precision and block dimension, on 7-point, 27-point and
unsymmetric patterns (where the U sweep would overwrite L results that rows
of the L sweep still read, without the barrier between the sweeps). The FP64
apply with its subdomain vector in global memory instead of shared memory
(the shared-memory ablation) gives the same bits as well.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from test_gpu_general_pattern import stencil27  # noqa: E402

GEOMS = [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED),
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE),     # no L pieces at all
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE),
    ((64, 64, 64), (16, 16, 8), synth.MODEL_LAYERED),
]
IDS = [f"{a[0]}x{a[1]}x{a[2]}-sub{b[0]}x{b[1]}x{b[2]}-m{m}" for a, b, m in GEOMS]


def nrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("bs", [3, 1])
@pytest.mark.parametrize("prec", ["f64", "f32", "bf16", "df64"])
@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_rowsync_equals_level_apply(grid, sub, model, prec, bs):
    s = synth.system(*grid, 21, model=model, bs=bs)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec)
    try:
        r = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, ctx.size)).cuda()
        assert torch.equal(ctx.apply_rowsync(r), ctx.apply(r))
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_rowsync_27_point_matches_oracle():
    grid, sub = (9, 7, 5), (9, 7, 5)
    rp, col, val, b, n = stencil27(*grid, seed=13)
    d = oracle.decompose(rp, col, val, grid, sub)
    ctx = g.Ilu0DD(rp, col, val, grid, sub)
    try:
        r = np.random.default_rng(4).uniform(-1, 1, 3 * n)
        z = ctx.apply_rowsync(torch.from_numpy(r).cuda())
        assert torch.equal(z, ctx.apply(torch.from_numpy(r).cuda()))
        assert nrel(z.cpu().numpy(), oracle.apply(d.LU, r)) <= 1e-12
    finally:
        ctx.close()


def unsymmetric(nx, ny, nz, seed):
    """The 7-point system with the +x and +y upper blocks of every third row
    removed (the pattern loses its symmetry; ILU0 works on any pattern with
    the diagonal)."""
    s = synth.system(nx, ny, nz, seed)
    rp, cols, vals = [0], [], []
    v = s.val.reshape(-1, 3, 3)
    for i in range(s.n):
        for q in range(s.row_ptr[i], s.row_ptr[i + 1]):
            j = s.col[q]
            if i % 3 == 0 and j in (i + 1, i + nx):
                continue
            cols.append(j)
            vals.append(v[q])
        rp.append(len(cols))
    return np.array(rp, np.int32), np.array(cols, np.int32), np.array(vals), s.n


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rowsync_unsymmetric_pattern(prec):
    grid, sub = (16, 16, 8), (16, 16, 8)
    rp, col, val, n = unsymmetric(*grid, 17)
    d = oracle.decompose(rp, col, val, grid, sub)
    ctx = g.Ilu0DD(rp, col, val, grid, sub, factor_prec=prec)
    try:
        r = np.random.default_rng(6).uniform(-1, 1, 3 * n)
        z = ctx.apply(torch.from_numpy(r).cuda())
        assert torch.equal(ctx.apply_rowsync(torch.from_numpy(r).cuda()), z)
        assert nrel(z.cpu().numpy(), oracle.apply(d.LU, r)) <= (1e-12 if prec == "f64" else 1e-5)
    finally:
        ctx.close()


def test_rowsync_refuses_boxes_without_room_for_the_flags():
    """16x16x37 cells (9,472 rows, 222 KiB of FP64 vector) fit the level
    apply but not one more byte per row."""
    grid = (16, 16, 37)
    s = synth.system(*grid, 3)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, grid)
    try:
        r = torch.zeros(ctx.size, dtype=torch.float64, device="cuda")
        with pytest.raises(g.Ilu0DDError) as e:
            ctx.apply_rowsync(r)
        assert e.value.code == 3
    finally:
        ctx.close()


@pytest.mark.parametrize("bs", [3, 1])
@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_global_vector_apply_equals_shared(grid, sub, model, bs):
    """The FP64 apply with the subdomain vector in global memory (the shared-
    memory ablation) gives the shared-memory apply's bits."""
    s = synth.system(*grid, 22, model=model, bs=bs)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub)
    try:
        r = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, ctx.size)).cuda()
        assert torch.equal(ctx.apply_global_vector(r), ctx.apply(r))
    finally:
        ctx.close()


def test_global_vector_apply_needs_fp64():
    s = synth.system(8, 8, 8, 3)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, (8, 8, 8), (4, 4, 4), factor_prec="f32")
    try:
        with pytest.raises(g.Ilu0DDError) as e:
            ctx.apply_global_vector(torch.zeros(ctx.size, dtype=torch.float64, device="cuda"))
        assert e.value.code == 1
    finally:
        ctx.close()
