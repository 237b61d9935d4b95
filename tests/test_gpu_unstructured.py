"""The graph-partition path on the GPU: unstructured systems (irregular
27-point pattern, cells renumbered at random), subdomains from the
breadth-first partition, against the oracle with the same labels.

Also: Algorithm 2's labels passed as an explicit partition give exactly the
grid path's plan and results (the two entry points share everything after
the labels).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402

CASES = [((10, 9, 8), 64), ((16, 12, 10), 256), ((24, 20, 16), 2048), ((7, 7, 7), 1)]
IDS = [f"{a[0]}x{a[1]}x{a[2]}-part{k}" for a, k in CASES]


def nrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("grid,k", CASES, ids=IDS)
def test_partitioned_decomposition_apply_and_solve(grid, k):
    s = synth.unstructured(*grid, 23)
    part, nparts = g.partition_bfs(s.row_ptr, s.col, k)
    d = oracle.decompose_labeled(s.row_ptr, s.col, s.val, part, nparts)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts, keep_host=1)
    try:
        for what, ref in [(B.X_PART_ID, part), (B.X_PERM, d.perm), (B.X_IPERM, d.iperm),
                          (B.X_PART_PTR, d.part_ptr), (B.X_DD_ROW_PTR, d.Add.row_ptr), (B.X_DD_COL, d.Add.col),
                          (B.X_LEVEL_L, oracle.levels_lower(d.Add)[0]), (B.X_LEVEL_U, oracle.levels_upper(d.Add)[0])]:
            assert np.array_equal(ctx.export(what), ref), what
        r = np.random.default_rng(4).uniform(-1, 1, 3 * s.n)
        assert nrel(ctx.apply(torch.from_numpy(r).cuda()).cpu().numpy(), oracle.apply(d.LU, r)) <= 1e-12
        x, info = ctx.solve(torch.from_numpy(s.b).cuda())
        ref = oracle.bicgstab(d.Ap, d.LU, s.b.reshape(-1, 3)[d.perm].reshape(-1))
        assert info["status"] == 0 and info["iterations"] == ref.iterations
        xo = ref.x.reshape(-1, 3)[d.iperm].reshape(-1)
        assert nrel(x.cpu().numpy(), xo) <= 1e-12
    finally:
        ctx.close()


@pytest.mark.parametrize("grid,k", CASES, ids=IDS)
def test_partitioned_fp64_bitwise_vs_oracle_ildu0(grid, k):
    """Rows of up to 13 blocks a side: the library's ILDU0 factors (Algorithm 7,
    Section 4.3), its fused apply and its BiCGSTAB solve are the oracle's
    ILDU0-form results bit for bit (the slots beyond the descriptor's three are
    multiply-added in ascending column order, as the oracle's row sweep does)."""
    s = synth.unstructured(*grid, 23)
    part, nparts = g.partition_bfs(s.row_ptr, s.col, k)
    d = oracle.decompose_labeled(s.row_ptr, s.col, s.val, part, nparts)
    M = d.ildu()
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts, keep_host=1)
    try:
        kept = d.Add.nnzb
        rows = np.repeat(np.arange(s.n), np.diff(d.Add.row_ptr))
        lower, upper = d.Add.col < rows, d.Add.col > rows
        assert np.array_equal(ctx.export(B.X_L).reshape(kept, 3, 3)[lower], M.F.val[lower])
        assert np.array_equal(ctx.export(B.X_UT).reshape(kept, 3, 3)[upper], M.F.val[upper])
        assert np.array_equal(ctx.export(B.X_INVD).reshape(-1, 3, 3), M.inv_d)
        r = np.random.default_rng(4).uniform(-1, 1, 3 * s.n)
        assert np.array_equal(ctx.apply(torch.from_numpy(r).cuda()).cpu().numpy(), oracle.apply_ildu0(M, r))
        x, info = ctx.solve(torch.from_numpy(s.b).cuda())
        ref = oracle.bicgstab(d.Ap, M, s.b.reshape(-1, 3)[d.perm].reshape(-1))
        assert info["status"] == ref.status == 0
        assert info["iterations"] == ref.iterations and info["restarts"] == ref.restarts
        assert np.array_equal(ctx.history(info["iterations"] + 1), ref.history)
        assert np.array_equal(x.cpu().numpy(), ref.x.reshape(-1, 3)[d.iperm].reshape(-1))
    finally:
        ctx.close()


def test_row_thread_mapping_only_for_narrow_rows():
    """FP32/BF16 factors take one thread per row only when no row has more than
    three blocks on either side (7-point patterns); the 27-point pattern takes
    the three-thread mapping, as FP64 factors always do."""
    s = synth.unstructured(10, 9, 8, 23)
    part, nparts = g.partition_bfs(s.row_ptr, s.col, 64)
    seven = synth.system(12, 12, 12, 1)
    for prec in ("f32", "bf16"):
        wide = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts, factor_prec=prec)
        narrow = g.Ilu0DD(seven.row_ptr, seven.col, seven.val, (12, 12, 12), (4, 4, 4), factor_prec=prec)
        try:
            assert wide.query("row_thread") == 0 and narrow.query("row_thread") == 1
        finally:
            wide.close()
            narrow.close()
    f64 = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts)
    try:
        assert f64.query("row_thread") == 0
    finally:
        f64.close()


@pytest.mark.parametrize("prec,tol", [("df64", 1e-12), ("f32", 1e-5), ("bf16", 5e-2)])
def test_partitioned_precisions(prec, tol):
    s = synth.unstructured(16, 12, 10, 29)
    part, nparts = g.partition_bfs(s.row_ptr, s.col, 512)
    d = oracle.decompose_labeled(s.row_ptr, s.col, s.val, part, nparts)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts, factor_prec=prec)
    host = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts, factor_prec=prec, device_setup=False)
    try:
        r = np.random.default_rng(5).uniform(-1, 1, 3 * s.n)
        z = ctx.apply(torch.from_numpy(r).cuda())
        assert nrel(z.cpu().numpy(), oracle.apply(d.LU, r)) <= tol
        assert np.array_equal(ctx.export(B.X_STREAM), host.export(B.X_STREAM))
        assert torch.equal(z, host.apply(torch.from_numpy(r).cuda()))
    finally:
        ctx.close()
        host.close()


def test_explicit_geometric_labels_equal_grid_path():
    grid, sub = (33, 17, 9), (16, 16, 8)
    s = synth.system(*grid, 3, model=synth.MODEL_LAYERED)
    a = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, keep_host=1)
    b = g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=oracle.partition(grid, sub), nparts=oracle.nparts(grid, sub),
                 keep_host=1)
    try:
        for what in (B.X_PERM, B.X_PART_PTR, B.X_LEVEL_L, B.X_LEVEL_U, B.X_STREAM, B.X_SELL_VAL, B.X_INVD):
            assert np.array_equal(a.export(what), b.export(what)), what
        xa, ia = a.solve(torch.from_numpy(s.b).cuda())
        xb, ib = b.solve(torch.from_numpy(s.b).cuda())
        assert ia["iterations"] == ib["iterations"] and torch.equal(xa, xb)
    finally:
        a.close()
        b.close()
