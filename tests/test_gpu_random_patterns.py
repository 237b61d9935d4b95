"""Random block patterns with random partitions on the GPU against the
oracle: irregular rows (many blocks a side, unsymmetric patterns), empty and
one-row parts, parts of any shape. Every apply form of the library
(fused, unfused, row flags, edge-centric), the SpMV and BiCGSTAB, for 3x3
and scalar blocks, FP64 factors."""
import numpy as np
import pytest

import oracle
import paper_2508_04917_gb300 as g

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_plan_fuzz import random_pattern  # noqa: E402


def random_system(rng, n, bs, symmetric):
    rp, col = random_pattern(rng, n, float(rng.uniform(0.002, 0.04)), symmetric)
    nnz = len(col)
    val = rng.uniform(-0.1, 0.1, (nnz, bs, bs))
    for i in range(n):
        row = slice(rp[i], rp[i + 1])
        off = np.abs(val[row]).sum(axis=(0, 2)).max()
        d = rp[i] + int(np.where(col[row] == i)[0][0])
        val[d] += (off + 1.0) * np.eye(bs)  # block diagonally dominant
    if bs == 1:
        val = val.reshape(-1)
    return rp, col, val


def nrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("seed", range(12))
def test_random_pattern_applies_match_oracle(seed):
    rng = np.random.default_rng(700 + seed)
    bs = 3 if seed % 3 else 1
    n = int(rng.integers(2, 600))
    rp, col, val = random_system(rng, n, bs, bool(seed % 2))
    if seed % 4 == 0:
        nparts = int(rng.integers(1, 12))
        part = rng.integers(0, nparts, n).astype(np.int32)  # arbitrary labels, empty parts possible
    else:
        part, nparts = g.partition_bfs(rp, col, int(rng.integers(1, 200)))
    d = oracle.decompose_labeled(rp, col, val, part, nparts)
    assert d.status == 0
    ctx = g.Ilu0DD(rp, col, val, part_id=part, nparts=nparts)
    try:
        r = rng.uniform(-1, 1, ctx.size)
        zo = oracle.apply(d.LU, r)
        rd = torch.from_numpy(r).cuda()
        z = ctx.apply(rd)
        assert nrel(z.cpu().numpy(), zo) <= 1e-12
        assert torch.equal(ctx.apply_unfused(rd), z)
        assert torch.equal(ctx.apply_rowsync(rd), z)
        assert nrel(ctx.apply_edge(rd).cpu().numpy(), zo) <= 1e-12
        x = rng.uniform(-1, 1, ctx.size)
        assert np.array_equal(ctx.spmv(torch.from_numpy(x).cuda()).cpu().numpy(), oracle.spmv(d.Ap, x))
        # BiCGSTAB (natural numbering) against the oracle's (reordered numbering)
        b = oracle.spmv(oracle.BSR(rp, col, val), rng.uniform(-1, 1, ctx.size))
        xs, info = ctx.solve(torch.from_numpy(b).cuda())
        perm = np.asarray(d.perm)
        to_new = (lambda v: v.reshape(-1, bs)[perm].reshape(-1))
        ref = oracle.bicgstab(d.Ap, d.LU, to_new(b))
        assert info["status"] == 0 and info["iterations"] == ref.iterations
        assert nrel(to_new(xs.cpu().numpy()), ref.x) <= 1e-12
        assert ctx.device_error() == 0
    finally:
        ctx.close()
