"""The DF64 factor mode against the FP64 oracle.

DF64 stores each factor entry as a float pair hi + lo and runs the fused apply
in double-float arithmetic on the FP32 pipe (not in the paper). It is held to
the FP64 bars: apply within 1e-12 normwise of the oracle's sequential ILU0
substitution, BiCGSTAB with the oracle's iteration count on the laplace
systems and within 5 % on the ill-conditioned layered ones. The per-block
power-of-two scaling must make the result independent of the magnitude of r.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402

FP64_TOL = 1e-12

GEOMS = [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),
    ((16, 16, 16), (16, 16, 8), synth.MODEL_LAYERED),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED),
    ((12, 12, 12), (4, 4, 4), synth.MODEL_LAPLACE),
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE),
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE),
    ((1, 1, 1), (1, 1, 1), synth.MODEL_LAPLACE),
    ((64, 64, 64), (16, 16, 8), synth.MODEL_LAPLACE),
]
IDS = [f"{g_[0]}x{g_[1]}x{g_[2]}-sub{s_[0]}x{s_[1]}x{s_[2]}-m{m}" for g_, s_, m in GEOMS]

_cache = {}


def case(grid, sub, model, seed=1):
    key = (grid, sub, model, seed)
    if key not in _cache:
        s = synth.system(*grid, seed, model=model)
        d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
        ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec="df64")
        _cache[key] = (s, d, ctx)
    return _cache[key]


def nrel(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def pvec(v, perm):
    return np.ascontiguousarray(np.asarray(v).reshape(-1, 3)[perm].reshape(-1))


@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_df64_apply_matches_oracle(grid, sub, model):
    s, d, ctx = case(grid, sub, model)
    r = np.random.default_rng(5).uniform(-1, 1, 3 * s.n)
    z = ctx.apply(cu(r)).cpu().numpy()
    assert nrel(z, oracle.apply(d.LU, r)) <= FP64_TOL
    assert np.array_equal(ctx.apply(cu(r)).cpu().numpy(), z)


@pytest.mark.parametrize("factor", [2.0 ** -600, 2.0 ** 600, 1e-300, 3e250])
def test_df64_apply_is_scale_free(factor):
    """Per-block power-of-two scaling: tiny and huge vectors (far outside FP32's
    range) give the oracle's result for the scaled input."""
    grid, sub, model = GEOMS[1]
    s, d, ctx = case(grid, sub, model)
    r = np.random.default_rng(6).uniform(-1, 1, 3 * s.n) * factor
    z = ctx.apply(cu(r)).cpu().numpy()
    assert np.all(np.isfinite(z))
    assert nrel(z, oracle.apply(d.LU, r)) <= FP64_TOL


@pytest.mark.parametrize("kind", ["wide", "tiny_and_zero", "pow2"])
def test_df64_apply_wide_dynamic_range(kind):
    """Entries spread over many binades inside each subdomain: the float-pair
    split and its inverse (done by integer operations where every step stays
    normal, by FP64 operations elsewhere: zeros, values too small for a
    normal float after the block's scaling) give the oracle's result."""
    grid, sub, model = GEOMS[2]
    s, d, ctx = case(grid, sub, model)
    rng = np.random.default_rng(11)
    n3 = 3 * s.n
    if kind == "wide":
        r = rng.uniform(-1, 1, n3) * np.exp2(rng.uniform(-90, 10, n3))
    elif kind == "tiny_and_zero":
        r = np.where(rng.uniform(0, 1, n3) < 0.3, 0.0,
                     rng.uniform(-1, 1, n3) * np.exp2(rng.integers(-140, 5, n3).astype(float)))
    else:
        r = np.exp2(rng.integers(-40, 40, n3).astype(float)) * rng.choice([-1.0, 1.0], n3)
    z = ctx.apply(cu(r)).cpu().numpy()
    assert np.all(np.isfinite(z))
    assert nrel(z, oracle.apply(d.LU, r)) <= FP64_TOL


def test_df64_apply_of_zero_and_mixed_blocks():
    """An all-zero subdomain next to ordinary ones: zeros stay exact zeros."""
    grid, sub, model = GEOMS[3]
    s, d, ctx = case(grid, sub, model)
    r = np.random.default_rng(7).uniform(-1, 1, 3 * s.n)
    r[: 3 * 64] = 0.0  # the first 4x4x4 subdomain (reordered rows 0..63)
    z = ctx.apply(cu(r)).cpu().numpy()
    assert not z[: 3 * 64].any()
    assert nrel(z, oracle.apply(d.LU, r)) <= FP64_TOL


@pytest.mark.parametrize("grid,sub,model", [GEOMS[0], GEOMS[1], GEOMS[2], GEOMS[7]],
                         ids=[IDS[0], IDS[1], IDS[2], IDS[7]])
def test_df64_bicgstab_matches_oracle(grid, sub, model):
    s, d, ctx = case(grid, sub, model)
    x, info = ctx.solve(cu(s.b))
    ref = oracle.bicgstab(d.Ap, d.LU, pvec(s.b, d.perm))
    assert info["status"] == 0 and info["rel_res_true"] < 1e-8
    if model == synth.MODEL_LAPLACE:
        assert info["iterations"] == ref.iterations
        xo = ref.x.reshape(-1, 3)[d.iperm].reshape(-1)
        assert nrel(x.cpu().numpy(), xo) <= FP64_TOL
    else:
        assert abs(info["iterations"] - ref.iterations) <= max(2, ref.iterations // 20)


def test_df64_rejects_factors_outside_its_range():
    """L and U~ = D^-1 U do not change when A is scaled, D^-1 scales inversely:
    with A scaled by 1e-40, D^-1 (about 1e39) exceeds 2^100 and cannot be held
    as a float pair: DF64 setup refuses with ILU0DD_ERR_INVALID; FP64 accepts."""
    grid, sub = (8, 8, 8), (4, 4, 4)
    s = synth.system(*grid, 3)
    val = s.val * 1e-40
    with pytest.raises(g.Ilu0DDError) as e:
        g.Ilu0DD(s.row_ptr, s.col, val, grid, sub, factor_prec="df64")
    assert e.value.code == 1
    ok = g.Ilu0DD(s.row_ptr, s.col, val, grid, sub)
    ok.close()
