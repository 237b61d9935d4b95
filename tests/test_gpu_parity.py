"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars: integer arrays (labels, permutation, levels, patterns) bit-exact;
SpMV and dot products bit-exact (same per-row order, same fixed reduction
order on both sides); FP64 apply outputs within a normwise relative error of
1e-12 (max_i |g_i - o_i| / max_i |o_i|); BiCGSTAB iteration counts and
restarts identical; solutions within 1e-12 on the well-conditioned laplace
systems and, at any conditioning, differing by less than what the stopping
test allows (||A (x_gpu - x_oracle)|| < 2 rtol ||b||).
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402

FP64_TOL = 1e-12


def nrel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def pvec(v, perm):
    return np.ascontiguousarray(np.asarray(v).reshape(-1, 3)[perm].reshape(-1))


_cache = {}


def case(grid, sub, seed=1, model=synth.MODEL_LAPLACE, **opts):
    key = (grid, sub, seed, model, tuple(sorted(opts.items())))
    if key not in _cache:
        s = synth.system(*grid, seed, model=model)
        d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
        ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, keep_host=1, **opts)
        _cache[key] = (s, d, ctx)
    return _cache[key]


GEOMS = [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),     # the 16^3 correctness workload
    ((16, 16, 16), (16, 16, 8), synth.MODEL_LAYERED),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED),     # ragged: edge subdomains smaller
    ((12, 12, 12), (4, 4, 4), synth.MODEL_LAPLACE),
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE),         # one-cell subdomains (block Jacobi)
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE),       # 1D chain, one subdomain (exact LU)
    ((1, 1, 1), (1, 1, 1), synth.MODEL_LAPLACE),         # a single cell
    ((6, 6, 6), (6, 6, 6), synth.MODEL_LAYERED),         # one subdomain = global ILU0
]
IDS = [f"{g_[0]}x{g_[1]}x{g_[2]}-sub{s_[0]}x{s_[1]}x{s_[2]}-m{m}" for g_, s_, m in GEOMS]


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_decomposition_and_levels_exact(grid, sub, model):
    """Algorithm 2 labels, Algorithm 3 permutation, Section 3.2 pattern and the
    level sets of every subdomain DAG: identical integers."""
    s, d, ctx = case(grid, sub, model=model)
    assert np.array_equal(ctx.export(B.X_PART_ID), d.part_id)
    assert np.array_equal(ctx.export(B.X_PERM), d.perm)
    assert np.array_equal(ctx.export(B.X_IPERM), d.iperm)
    assert np.array_equal(ctx.export(B.X_PART_PTR), d.part_ptr)
    assert np.array_equal(ctx.export(B.X_AP_ROW_PTR), d.Ap.row_ptr)
    assert np.array_equal(ctx.export(B.X_AP_COL), d.Ap.col)
    assert np.array_equal(ctx.export(B.X_DD_ROW_PTR), d.Add.row_ptr)
    assert np.array_equal(ctx.export(B.X_DD_COL), d.Add.col)
    assert np.array_equal(ctx.export(B.X_LEVEL_L), oracle.levels_lower(d.Add)[0])
    assert np.array_equal(ctx.export(B.X_LEVEL_U), oracle.levels_upper(d.Add)[0])


@pytest.mark.parametrize("grid,sub,model", GEOMS[:4], ids=IDS[:4])
def test_ildu0_factors_match_oracle_ilu0(grid, sub, model):
    """Algorithm 7: the library's L, D^-1 and U~ = D^-1 U against the oracle's ILU0
    factors (L, U): L equal, D^-1 = U_ii^-1, U~_ik = U_ii^-1 U_ik."""
    s, d, ctx = case(grid, sub, model=model)
    kept = d.Add.nnzb
    L = ctx.export(B.X_L).reshape(kept, 3, 3)
    Ut = ctx.export(B.X_UT).reshape(kept, 3, 3)
    invD = ctx.export(B.X_INVD).reshape(-1, 3, 3)
    rp, col, lu = d.LU.row_ptr, d.LU.col, d.LU.val
    rows = np.repeat(np.arange(s.n), np.diff(rp))
    lower, upper, diag = col < rows, col > rows, col == rows
    assert nrel(L[lower], lu[lower]) <= FP64_TOL
    Uii = lu[diag]
    assert nrel(invD, np.linalg.inv(Uii)) <= FP64_TOL
    ref_ut = np.einsum("nab,nbc->nac", np.linalg.inv(Uii)[rows[upper]], lu[upper])
    if upper.any():
        assert nrel(Ut[upper], ref_ut) <= FP64_TOL
    assert not L[~lower].any() and not Ut[~upper].any()


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_apply_fp64_matches_oracle(grid, sub, model):
    """Fused L -> D^-1 -> U~ apply (Sections 4.3-4.4) against sequential ILU0
    substitution: normwise relative error <= 1e-12; repeat calls are bitwise equal."""
    s, d, ctx = case(grid, sub, model=model)
    r = np.random.default_rng(5).uniform(-1, 1, 3 * s.n)
    z = host(ctx.apply(cu(r)))
    zo = oracle.apply(d.LU, r)
    assert nrel(z, zo) <= FP64_TOL
    assert np.array_equal(host(ctx.apply(cu(r))), z)


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_spmv_and_dot_bitwise(grid, sub, model):
    """SpMV (full reordered matrix) and the fixed-order dot product are bit-identical
    to the oracle's, which follow the same per-row and reduction order."""
    s, d, ctx = case(grid, sub, model=model)
    x = np.random.default_rng(6).uniform(-1, 1, 3 * s.n)
    y = host(ctx.spmv(cu(x)))
    assert np.array_equal(y, oracle.spmv(d.Ap, x))
    w = np.random.default_rng(7).uniform(-1, 1, 3 * s.n)
    assert host(ctx.dot(cu(x), cu(w)))[0] == oracle.dot(x, w)


def test_dot_sizes_and_order():
    """Dot products over many tile counts (1 .. > 256 tiles, ragged last tile) match the
    oracle bit for bit, including the crafted order-sensitive case."""
    for grid in [(1, 1, 1), (7, 1, 1), (16, 16, 1), (17, 16, 1), (64, 32, 16), (64, 64, 33)]:
        s = synth.system(*grid, 2)
        ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, grid if grid[0] * grid[1] * grid[2] <= 2048 else (16, 16, 8))
        rng = np.random.default_rng(grid[0] * 1000 + grid[2])
        x, w = rng.normal(size=3 * s.n), rng.normal(size=3 * s.n) * 1e3
        assert host(ctx.dot(cu(x), cu(w)))[0] == oracle.dot(x, w)
        ctx.close()
    s = synth.system(32, 16, 1, 2)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, (32, 16, 1), (16, 16, 1))
    x = np.zeros(3 * 512)
    x[0], x[3], x[3 * 129] = 2.0 ** 53, 1.0, 1.0
    assert host(ctx.dot(cu(x), cu(np.ones_like(x))))[0] == 2.0 ** 53 + 2.0


def test_permute_round_trip():
    s, d, ctx = case((33, 17, 9), (16, 16, 8), model=synth.MODEL_LAYERED)
    x = np.random.default_rng(8).uniform(-1, 1, 3 * s.n)
    xp = host(ctx.permute(cu(x), 0))
    assert np.array_equal(xp, pvec(x, d.perm))
    assert np.array_equal(host(ctx.permute(cu(xp), 1)), x)


def check_solution(s, d, x, ref, rtol=1e-8, well_conditioned=True):
    """The GPU solution against the oracle's. Both stop on ||r|| < rtol ||b||, so their
    difference e satisfies ||A e|| < 2 rtol ||b|| at any conditioning; on the
    well-conditioned laplace systems the two also agree to 1e-12 (normwise)."""
    xo = pvec(ref.x, d.iperm)
    e = pvec(x - xo, d.perm)
    assert np.linalg.norm(oracle.spmv(d.Ap, e)) <= 2 * rtol * np.linalg.norm(s.b)
    if well_conditioned:
        assert nrel(x, xo) <= FP64_TOL


def count_report(info, hist, ref, rtol=1e-8):
    """The ILU0-form comparison of a solve: the count difference and, at the
    decisive iteration (the earlier stop), each side's margin ||r|| / ||b|| - rtol
    (negative: that side stopped there)."""
    j = min(info["iterations"], ref.iterations)
    return {"gpu_iterations": info["iterations"], "oracle_ilu0_iterations": ref.iterations,
            "difference": info["iterations"] - ref.iterations, "decisive_iteration": j,
            "margin_gpu": float(hist[j]) - rtol, "margin_oracle_ilu0": float(ref.history[j]) - rtol}


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_ildu0_factors_bitwise_vs_oracle_ildu0(grid, sub, model):
    """Algorithm 7 with Section 4.3's post-processing: the library's L, D^-1 and
    U~ are the oracle's ILDU0-form factors bit for bit."""
    s, d, ctx = case(grid, sub, model=model)
    M = d.ildu()
    kept = d.Add.nnzb
    L = ctx.export(B.X_L).reshape(kept, 3, 3)
    Ut = ctx.export(B.X_UT).reshape(kept, 3, 3)
    rows = np.repeat(np.arange(s.n), np.diff(d.Add.row_ptr))
    lower, upper = d.Add.col < rows, d.Add.col > rows
    assert np.array_equal(L[lower], M.F.val[lower])
    assert np.array_equal(Ut[upper], M.F.val[upper])
    assert np.array_equal(ctx.export(B.X_INVD).reshape(-1, 3, 3), M.inv_d)


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_apply_fp64_bitwise_vs_oracle_ildu0(grid, sub, model):
    """The fused apply (Sections 4.3-4.4) computes, row by row in level order, what
    the oracle's ILDU0-form substitution computes in row order, with the same
    per-row operations: the same bits."""
    s, d, ctx = case(grid, sub, model=model)
    r = np.random.default_rng(5).uniform(-1, 1, 3 * s.n)
    assert np.array_equal(host(ctx.apply(cu(r))), oracle.apply_ildu0(d.ildu(), r))


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_bicgstab_matches_oracle(grid, sub, model, record_property):
    """Algorithm 1 on the device against the oracle with the same (ILDU0-form)
    preconditioner: identical iteration count and restarts, the same residual
    history and the same solution, bit for bit.  Against the oracle's ILU0 form
    (an independent check of the arithmetic): both converge, the solutions
    differ by less than the stopping test allows, the counts are identical on
    the laplace systems and reported (difference and decisive-iteration
    margins) on the ill-conditioned layered ones."""
    s, d, ctx = case(grid, sub, model=model)
    x, info = ctx.solve(cu(s.b))
    x = host(x)
    b = pvec(s.b, d.perm)
    ref = oracle.bicgstab(d.Ap, d.ildu(), b)
    assert ref.status == 0 and info["status"] == 0
    assert info["iterations"] == ref.iterations and info["restarts"] == ref.restarts
    hist = ctx.history(info["iterations"] + 1)
    assert np.array_equal(hist, ref.history)
    assert np.array_equal(x, pvec(ref.x, d.iperm))
    assert info["rel_res_true"] == ref.rel_res_true < 1e-8
    ilu = oracle.bicgstab(d.Ap, d.LU, b)
    assert ilu.status == 0
    check_solution(s, d, x, ilu, well_conditioned=model == synth.MODEL_LAPLACE)
    rep = count_report(info, hist, ilu)
    record_property("ilu0_form_counts", rep)
    print("ILU0-form count comparison:", rep)
    if model == synth.MODEL_LAPLACE:
        assert rep["difference"] == 0


@pytest.mark.parametrize("sub", [(4, 4, 4), (8, 8, 8), (16, 16, 8)])
def test_bicgstab_64cubed_layered_identical(sub, record_property):
    """The layered (ill-conditioned, 160^3 benchmark class) model at 64^3 for the
    three subdomain sizes: identical counts, histories and solutions against the
    oracle's ILDU0-form solve; the ILU0-form counts reported."""
    s, d, ctx = case((64, 64, 64), sub, seed=3, model=synth.MODEL_LAYERED)
    x, info = ctx.solve(cu(s.b))
    b = pvec(s.b, d.perm)
    oracle.set_threads(min(16, os.cpu_count() or 1))
    try:
        ref = oracle.bicgstab(d.Ap, d.ildu(), b)
        ilu = oracle.bicgstab(d.Ap, d.LU, b)
    finally:
        oracle.set_threads(1)
    assert info["status"] == ref.status == 0
    assert info["iterations"] == ref.iterations and info["restarts"] == ref.restarts
    hist = ctx.history(info["iterations"] + 1)
    assert np.array_equal(hist, ref.history)
    assert np.array_equal(host(x), pvec(ref.x, d.iperm))
    assert ilu.status == 0
    check_solution(s, d, host(x), ilu, well_conditioned=False)
    rep = count_report(info, hist, ilu)
    record_property("ilu0_form_counts", rep)
    print("ILU0-form count comparison:", rep)


@pytest.mark.parametrize("grid,sub,model", [GEOMS[2], GEOMS[1]], ids=[IDS[2], IDS[1]])
def test_solve_is_deterministic(grid, sub, model):
    """Vertex-centric kernels and fixed-order reductions: repeated solves, on the same
    context and on a fresh one, give bit-identical iterates and iteration counts."""
    s, d, ctx = case(grid, sub, model=model)
    runs = [ctx.solve(cu(s.b)) for _ in range(3)]
    fresh = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub)
    runs.append(fresh.solve(cu(s.b)))
    x0, i0 = runs[0]
    for x, info in runs[1:]:
        assert info["iterations"] == i0["iterations"]
        assert torch.equal(x, x0)
    r = cu(np.random.default_rng(11).uniform(-1, 1, 3 * s.n))
    z0 = ctx.apply(r)
    for _ in range(20):
        assert torch.equal(ctx.apply(r), z0)
    fresh.close()


@pytest.mark.parametrize("sub", [(4, 4, 4), (8, 8, 8), (16, 16, 8)])
def test_bicgstab_64cubed_sweep(sub):
    """64^3 laplace system (262,144 block rows) for the three subdomain sizes: the
    oracle's iteration count, its solution within 1e-12, converged true residual."""
    s, d, ctx = case((64, 64, 64), sub, seed=2)
    x, info = ctx.solve(cu(s.b))
    ref = oracle.bicgstab(d.Ap, d.LU, pvec(s.b, d.perm))
    assert info["iterations"] == ref.iterations and info["status"] == 0
    check_solution(s, d, host(x), ref)


def test_solve_repeatable_and_graph_free_path_agree():
    """Two solves give identical bits; the CUDA-graph path equals plain launches."""
    s, d, ctx = case((16, 16, 16), (8, 8, 4))
    x1, i1 = ctx.solve(cu(s.b))
    x2, i2 = ctx.solve(cu(s.b))
    assert torch.equal(x1, x2) and i1["iterations"] == i2["iterations"]
    ctx2 = g.Ilu0DD(s.row_ptr, s.col, s.val, (16, 16, 16), (8, 8, 4), use_graphs=0, check_every=3)
    x3, i3 = ctx2.solve(cu(s.b))
    assert torch.equal(x1, x3) and i3["iterations"] == i1["iterations"]
    ctx2.close()


def test_zero_and_nonfinite_rhs():
    s, d, ctx = case((12, 12, 12), (4, 4, 4))
    x, info = ctx.solve(cu(np.zeros(3 * s.n)))
    assert info["status"] == 0 and info["iterations"] == 0 and not host(x).any()
    b = s.b.copy()
    b[5] = np.nan
    _, info = ctx.solve(cu(b), check=False)
    assert info["status"] == B.ERR_NONFINITE


def test_maxit_reports_not_converged():
    s = synth.system(16, 16, 16, 1, model=synth.MODEL_LAYERED)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, (16, 16, 16), (4, 4, 4), maxit=3)
    _, info = ctx.solve(cu(s.b), check=False)
    assert info["status"] == B.ERR_NOT_CONVERGED and info["iterations"] == 3
    ctx.close()


def test_largest_subdomain_fits_shared_memory():
    """8192-row subdomains (16x16x32 cells, 192 KiB FP64 vector) run and match."""
    grid = sub = (16, 16, 32)
    s, d, ctx = case(grid, sub, seed=4)
    r = np.random.default_rng(9).uniform(-1, 1, 3 * s.n)
    assert nrel(host(ctx.apply(cu(r))), oracle.apply(d.LU, r)) <= FP64_TOL
    assert ctx.query("smem") <= 232448


@pytest.mark.parametrize("prec,z,tol", [("f64", 37, 0.0), ("df64", 37, 1e-12), ("f32", 55, 1e-5), ("bf16", 55, 5e-2)])
def test_maximum_subdomain_per_precision(prec, z, tol):
    """The largest box subdomain whose vector fits the 227 KiB of shared memory
    per block: 16x16x37 cells (9,472 block rows, 24 bytes a row) with FP64 or
    float-pair factors, 16x16x55 (14,080 rows, 16 bytes a row in the row-thread
    layout) with FP32 or BF16 factors; one z-layer more is refused (CPU test).
    The apply against the oracle's ILDU0 form (FP64: bit for bit) and a solve to
    1e-8."""
    grid = sub = (16, 16, z)
    s, d, ctx = case(grid, sub, seed=12, model=synth.MODEL_LAYERED, factor_prec=prec)
    assert ctx.query("n") == 256 * z and ctx.query("nsub") == 1
    r = np.random.default_rng(13).uniform(-1, 1, 3 * s.n)
    z_gpu = host(ctx.apply(cu(r)))
    ref = oracle.apply_ildu0(d.ildu(), r)
    if tol == 0.0:
        assert np.array_equal(z_gpu, ref)
    else:
        assert nrel(z_gpu, ref) <= tol
    _, info = ctx.solve(cu(s.b))
    assert info["status"] == 0 and info["rel_res_true"] < 1e-8
    assert ctx.query("smem") <= 232448


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_row_thread_and_three_thread_mappings_same_bits(prec):
    """FP32 / BF16 factors on 7-point rows: the row-thread apply (one thread per
    row, the default here) and the three-thread apply (apply_mapping = 1) form
    each output component with the same operations in the same order, so the
    fused, unfused and row-flag applies and whole solves agree bit for bit."""
    grid, sub = (33, 17, 9), (16, 16, 8)
    s = synth.system(*grid, 3, model=synth.MODEL_LAYERED)
    rt = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec)
    tt = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec, apply_mapping=1)
    try:
        assert rt.query("row_thread") == 1 and tt.query("row_thread") == 0
        r = cu(np.random.default_rng(14).uniform(-1, 1, 3 * s.n))
        for name in ("apply", "apply_unfused", "apply_rowsync"):
            assert torch.equal(getattr(rt, name)(r), getattr(tt, name)(r)), name
        xa, ia = rt.solve(cu(s.b))
        xb, ib = tt.solve(cu(s.b))
        assert ia["status"] == ib["status"] == 0 and ia["iterations"] == ib["iterations"]
        assert torch.equal(xa, xb)
    finally:
        rt.close()
        tt.close()


def test_zero_pivot_reported():
    """A zero diagonal block on the first row of a subdomain is a zero pivot of ILU0."""
    s = synth.system(4, 4, 4, 1)
    val = s.val.copy()
    q = [q for q in range(s.row_ptr[0], s.row_ptr[1]) if s.col[q] == 0][0]
    val[q] = 0.0
    with pytest.raises(g.Ilu0DDError) as e:
        g.Ilu0DD(s.row_ptr, s.col, val, (4, 4, 4), (2, 2, 2))
    assert e.value.code == B.ERR_ZERO_PIVOT


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("bf16", 5e-2)])
def test_reduced_precision_factors(prec, tol):
    """FP32 / BF16-stored factors (FP32 arithmetic): apply error against the FP64
    oracle within the storage precision times a modest growth factor, and BiCGSTAB
    (FP64 vectors, dots and recurrences) still reaches 1e-8."""
    s, d, ctx = case((64, 64, 64), (16, 16, 8), seed=4, factor_prec=prec)
    r = np.random.default_rng(10).uniform(-1, 1, 3 * s.n)
    err = nrel(host(ctx.apply(cu(r))), oracle.apply(d.LU, r))
    assert err <= tol
    x, info = ctx.solve(cu(s.b))
    assert info["status"] == 0 and info["rel_res_true"] < 1e-8
    assert nrel(host(x), s.xstar) < 1e-6


def test_no_device_wait_expired():
    s, d, ctx = case((16, 16, 16), (8, 8, 4))
    ctx.apply(cu(np.ones(3 * s.n)))
    assert ctx.device_error() == 0
