"""Batched BiCGSTAB (one launch per step over many systems) against per-system solves.

The batched kernels run the same per-block device functions, in the same
per-system order, as the single-system kernels, so every system's iterates,
iteration count and solution must be bit-identical to its own bicgstab_solve.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402


def _systems(specs):
    out = []
    for grid, sub, seed, model in specs:
        s = synth.system(*grid, seed, model=model)
        out.append((grid, sub, s))
    return out


SPECS = [
    ((12, 9, 7), (4, 4, 4), 5001, synth.MODEL_LAPLACE),    # ragged edges
    ((16, 16, 8), (16, 16, 8), 5002, synth.MODEL_LAYERED),  # one subdomain
    ((1, 1, 1), (1, 1, 1), 5003, synth.MODEL_LAPLACE),      # a single cell
    ((24, 10, 13), (8, 8, 4), 5004, synth.MODEL_LAPLACE),
    ((7, 19, 5), (8, 8, 8), 5005, synth.MODEL_LAYERED),
]


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_batched_equals_per_system_solves(prec):
    systems = _systems(SPECS)
    ctxs = [g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec) for grid, sub, s in systems]
    bs = [torch.from_numpy(s.b).cuda() for _, _, s in systems]
    singles = [c.solve(b) for c, b in zip(ctxs, bs)]
    batch = g.Batch(ctxs)
    xs, infos = batch.solve(bs)
    for (x1, i1), x2, i2 in zip(singles, xs, infos):
        assert i2["status"] == 0 and i1["status"] == 0
        assert i2["iterations"] == i1["iterations"]
        assert torch.equal(x1, x2)
        assert i2["rel_res_true"] == i1["rel_res_true"] and i2["rel_res_true"] < 1e-8
    # a second batched solve reuses the captured graph and gives the same bits
    xs2, infos2 = batch.solve(bs)
    assert all(torch.equal(a, b) for a, b in zip(xs, xs2))
    batch.close()
    for c in ctxs:
        c.close()


def test_batched_matches_oracle_iterations():
    """Laplace systems of the batch reach the oracle's iteration counts."""
    specs = [s for s in SPECS if s[3] == synth.MODEL_LAPLACE]
    systems = _systems(specs)
    ctxs = [g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub) for grid, sub, s in systems]
    batch = g.Batch(ctxs, use_graphs=0, check_every=3)
    xs, infos = batch.solve([torch.from_numpy(s.b).cuda() for _, _, s in systems])
    for (grid, sub, s), x, info in zip(systems, xs, infos):
        d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
        ref = oracle.bicgstab(d.Ap, d.LU, s.b.reshape(-1, 3)[d.perm].reshape(-1))
        assert info["iterations"] == ref.iterations
        xo = ref.x.reshape(-1, 3)[d.iperm].reshape(-1)
        assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * np.abs(xo).max()
    batch.close()


def test_batched_zero_rhs_and_mixed_convergence():
    """A zero right-hand side finishes at once while the others keep iterating."""
    systems = _systems(SPECS[:2])
    ctxs = [g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub) for grid, sub, s in systems]
    bs = [torch.zeros(3 * systems[0][2].n, dtype=torch.float64, device="cuda"),
          torch.from_numpy(systems[1][2].b).cuda()]
    batch = g.Batch(ctxs)
    xs, infos = batch.solve(bs)
    assert infos[0]["iterations"] == 0 and not xs[0].any()
    assert infos[1]["iterations"] > 5 and infos[1]["rel_res_true"] < 1e-8
    batch.close()


def test_batch_rejects_mixed_precision():
    systems = _systems(SPECS[:2])
    c0 = g.Ilu0DD(systems[0][2].row_ptr, systems[0][2].col, systems[0][2].val, systems[0][0], systems[0][1])
    c1 = g.Ilu0DD(systems[1][2].row_ptr, systems[1][2].col, systems[1][2].val, systems[1][0], systems[1][1],
                  factor_prec="f32")
    with pytest.raises(g.Ilu0DDError):
        g.Batch([c0, c1])


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_batched_three_thread_mapping(prec):
    """FP32/BF16 systems with rows of more than three blocks a side (27-point
    unstructured patterns, graph partitions) take the three-thread mapping;
    their batch gives each system's single-solve bits. A batch that mixes them
    with row-thread systems is refused (one mapping per batched launch)."""
    ctxs = []
    for grid, k, seed in [((10, 9, 8), 64, 31), ((16, 12, 10), 256, 32), ((12, 8, 6), 128, 33)]:
        s = synth.unstructured(*grid, seed)
        part, nparts = g.partition_bfs(s.row_ptr, s.col, k)
        ctxs.append((g.Ilu0DD(s.row_ptr, s.col, s.val, part_id=part, nparts=nparts, factor_prec=prec), s))
    assert all(c.query("row_thread") == 0 for c, _ in ctxs)
    bs = [torch.from_numpy(s.b).cuda() for _, s in ctxs]
    singles = [c.solve(b) for (c, _), b in zip(ctxs, bs)]
    batch = g.Batch([c for c, _ in ctxs])
    xs, infos = batch.solve(bs)
    for (x1, i1), x2, i2 in zip(singles, xs, infos):
        assert i1["status"] == i2["status"] == 0 and i1["iterations"] == i2["iterations"]
        assert torch.equal(x1, x2)
    batch.close()
    grid, sub, s7 = _systems(SPECS[:1])[0]
    narrow = g.Ilu0DD(s7.row_ptr, s7.col, s7.val, grid, sub, factor_prec=prec)
    assert narrow.query("row_thread") == 1
    with pytest.raises(g.Ilu0DDError):
        g.Batch([narrow, ctxs[0][0]])
    narrow.close()
    for c, _ in ctxs:
        c.close()


def test_benchmark_batch_workload():
    """The benchmark's batched workload in full: 64 laplace systems with sides
    drawn from 24..96 (synth.ragged_batch), FP32 factors, 8x8x8 boxes at 160
    threads per block (the configuration the autotuner picks on GB300). Every
    system's batched solution has its single solve's bits and iteration count
    and a true residual below 1e-8; with FP64 factors the two smallest systems
    reach the oracle's iteration counts and solutions (1e-12)."""
    sides = synth.ragged_batch(64)
    systems = [synth.system(*sd, 5000 + i) for i, sd in enumerate(sides)]
    ctxs = [g.Ilu0DD(s.row_ptr, s.col, s.val, (s.nx, s.ny, s.nz), (8, 8, 8), factor_prec="f32",
                     threads_per_cta=160) for s in systems]
    bs = [torch.from_numpy(s.b).cuda() for s in systems]
    try:
        batch = g.Batch(ctxs)
        xs, infos = batch.solve(bs)
        batch.close()
        for c, b, x2, i2 in zip(ctxs, bs, xs, infos):
            x1, i1 = c.solve(b)
            assert i2["status"] == 0 and i2["rel_res_true"] < 1e-8
            assert i2["iterations"] == i1["iterations"] and torch.equal(x1, x2)
    finally:
        for c in ctxs:
            c.close()
    small = sorted(range(len(systems)), key=lambda i: systems[i].n)[:2]
    sel = [systems[i] for i in small]
    ctxs = [g.Ilu0DD(s.row_ptr, s.col, s.val, (s.nx, s.ny, s.nz), (8, 8, 8)) for s in sel]
    try:
        batch = g.Batch(ctxs)
        xs, infos = batch.solve([torch.from_numpy(s.b).cuda() for s in sel])
        batch.close()
        for s, x, info in zip(sel, xs, infos):
            grid = (s.nx, s.ny, s.nz)
            d = oracle.decompose(s.row_ptr, s.col, s.val, grid, (8, 8, 8))
            ref = oracle.bicgstab(d.Ap, d.LU, s.b.reshape(-1, 3)[d.perm].reshape(-1))
            assert info["iterations"] == ref.iterations
            xo = ref.x.reshape(-1, 3)[d.iperm].reshape(-1)
            assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * np.abs(xo).max()
    finally:
        for c in ctxs:
            c.close()
