"""Scalar (1x1-block) CSR systems on the GPU against the oracle.

The same bars as the 3x3 path: labels, permutation, patterns and levels
bit-exact; SpMV and dot products bit-exact (same per-row order, same fixed
reduction order); FP64 and DF64 applies within 1e-12 of the oracle's
sequential ILU0 substitution, FP32/BF16 within their storage precision; the
FP64 apply bit for bit the oracle's ILDU0-form substitution, and BiCGSTAB with
the oracle's (ILDU0-form) iteration count, history and solution bit for bit,
the ILU0-form counts identical on the laplace systems; the device setup, the unfused apply
and the host-buffer apply giving the same bits as their counterparts; a
batch of scalar systems giving each single solve's bits.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402

GEOMS = [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED),
    ((12, 12, 12), (4, 4, 4), synth.MODEL_LAPLACE),
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE),
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE),
    ((1, 1, 1), (1, 1, 1), synth.MODEL_LAPLACE),
    ((64, 64, 64), (32, 16, 16), synth.MODEL_LAPLACE),  # 8,192-row subdomains, the paper's CSR part size
]
IDS = [f"{a[0]}x{a[1]}x{a[2]}-sub{b[0]}x{b[1]}x{b[2]}-m{m}" for a, b, m in GEOMS]

_cache = {}


def case(grid, sub, model, prec="f64"):
    key = (grid, sub, model, prec)
    if key not in _cache:
        s = synth.system(*grid, 3, model=model, bs=1)
        d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
        ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec, keep_host=1)
        _cache[key] = (s, d, ctx)
    return _cache[key]


def nrel(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_scalar_decomposition_spmv_dot_exact(grid, sub, model):
    s, d, ctx = case(grid, sub, model)
    assert ctx.bs == 1 and ctx.size == s.n
    for what, ref in [(B.X_PERM, d.perm), (B.X_PART_PTR, d.part_ptr), (B.X_DD_ROW_PTR, d.Add.row_ptr),
                      (B.X_DD_COL, d.Add.col), (B.X_LEVEL_L, oracle.levels_lower(d.Add)[0]),
                      (B.X_LEVEL_U, oracle.levels_upper(d.Add)[0])]:
        assert np.array_equal(ctx.export(what), ref), what
    x = np.random.default_rng(1).uniform(-1, 1, s.n)
    assert np.array_equal(ctx.spmv(cu(x)).cpu().numpy(), oracle.spmv(d.Ap, x))
    w = np.random.default_rng(2).normal(size=s.n) * 1e3
    assert ctx.dot(cu(x), cu(w)).item() == oracle.dot(x, w, bs=1)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("df64", 1e-12), ("f32", 1e-5), ("bf16", 5e-2)])
@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_scalar_apply_matches_oracle(grid, sub, model, prec, tol):
    s, d, ctx = case(grid, sub, model, prec)
    r = np.random.default_rng(5).uniform(-1, 1, s.n)
    z = ctx.apply(cu(r)).cpu().numpy()
    assert nrel(z, oracle.apply(d.LU, r)) <= tol


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_scalar_apply_bitwise_vs_oracle_ildu0(grid, sub, model):
    """Scalar factors: inv_D_i = 1 / U_ii and U~_ik = inv_D_i U_ik (Algorithm 7's
    post-processing) and the fused apply are the oracle's ILDU0 form bit for bit."""
    s, d, ctx = case(grid, sub, model)
    M = d.ildu()
    rows = np.repeat(np.arange(s.n), np.diff(d.Add.row_ptr))
    lower, upper = d.Add.col < rows, d.Add.col > rows
    assert np.array_equal(ctx.export(B.X_L)[lower], M.F.val.reshape(-1)[lower])
    assert np.array_equal(ctx.export(B.X_UT)[upper], M.F.val.reshape(-1)[upper])
    assert np.array_equal(ctx.export(B.X_INVD), M.inv_d.reshape(-1))
    r = np.random.default_rng(5).uniform(-1, 1, s.n)
    assert np.array_equal(ctx.apply(cu(r)).cpu().numpy(), oracle.apply_ildu0(M, r))


@pytest.mark.parametrize("grid,sub,model", [GEOMS[0], GEOMS[1], GEOMS[2], GEOMS[6]],
                         ids=[IDS[0], IDS[1], IDS[2], IDS[6]])
def test_scalar_bicgstab_matches_oracle(grid, sub, model):
    s, d, ctx = case(grid, sub, model)
    x, info = ctx.solve(cu(s.b))
    ref = oracle.bicgstab(d.Ap, d.ildu(), s.b[d.perm])
    assert info["status"] == ref.status == 0 and info["rel_res_true"] < 1e-8
    assert info["iterations"] == ref.iterations and info["restarts"] == ref.restarts
    assert np.array_equal(ctx.history(info["iterations"] + 1), ref.history)
    assert np.array_equal(x.cpu().numpy(), ref.x[d.iperm])
    ilu = oracle.bicgstab(d.Ap, d.LU, s.b[d.perm])
    assert ilu.status == 0
    if model == synth.MODEL_LAPLACE:
        assert info["iterations"] == ilu.iterations
        assert nrel(x.cpu().numpy(), ilu.x[d.iperm]) <= 1e-12
    else:
        print("ILU0-form count comparison:", info["iterations"], ilu.iterations)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "bf16"])
def test_scalar_device_setup_unfused_and_host_apply(prec):
    grid, sub, model = GEOMS[1]
    s = synth.system(*grid, 4, model=model, bs=1)
    dev = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec, keep_host=1)
    host = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec, keep_host=1, device_setup=False)
    try:
        for what in (B.X_STREAM, B.X_SELL_COL, B.X_SELL_VAL, B.X_L, B.X_UT, B.X_INVD):
            assert np.array_equal(dev.export(what).view(np.uint8), host.export(what).view(np.uint8)), what
        r = np.random.default_rng(6).uniform(-1, 1, s.n)
        z = dev.apply(cu(r))
        zu = dev.apply_unfused(cu(r))
        if prec == "df64":
            assert float((z - zu).abs().max() / z.abs().max()) <= 1e-13
        else:
            assert torch.equal(z, zu)
        assert np.array_equal(dev.apply_host(r), z.cpu().numpy())
    finally:
        dev.close()
        host.close()


def test_scalar_batched_equals_single():
    """A batch of scalar systems (different grids and subdomain boxes) gives
    each system's single-solve bits and iteration count."""
    specs = [GEOMS[0], GEOMS[1], GEOMS[2]]
    ctxs, bvecs = [], []
    for k, (grid, sub, model) in enumerate(specs):
        s = synth.system(*grid, 21 + k, model=model, bs=1)
        ctxs.append(g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub))
        bvecs.append(cu(s.b))
    try:
        singles = [c.solve(b) for c, b in zip(ctxs, bvecs)]
        batch = g.Batch(ctxs)
        xs, infos = batch.solve(bvecs)
        for (x1, i1), x2, i2 in zip(singles, xs, infos):
            assert i2["status"] == 0 and i1["iterations"] == i2["iterations"] and torch.equal(x1, x2)
        batch.close()
    finally:
        for c in ctxs:
            c.close()


def test_batch_refuses_mixed_block_dims():
    s1 = synth.system(8, 8, 8, 5, bs=1)
    s3 = synth.system(8, 8, 8, 5)
    c1 = g.Ilu0DD(s1.row_ptr, s1.col, s1.val, (8, 8, 8), (4, 4, 4))
    c3 = g.Ilu0DD(s3.row_ptr, s3.col, s3.val, (8, 8, 8), (4, 4, 4))
    try:
        with pytest.raises(g.Ilu0DDError):
            g.Batch([c1, c3])
    finally:
        c1.close()
        c3.close()
