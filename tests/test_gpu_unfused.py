"""The unfused apply (two launches: L sweep, then D^-1 and U~ sweep) against
the fused one (Section 4.4) and the oracle.

Both run the same per-row arithmetic on the same packed stream; only the
intermediate vector makes a round trip through global memory (as FP64, which
holds the FP32 and BF16 modes' FP32 values exactly). So FP64, FP32 and BF16
results are bit-identical; DF64 rescales its vector between the launches and
agrees to rounding.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402

GEOMS = [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED),
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE),     # no L pieces at all
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE),
    ((64, 64, 64), (16, 16, 8), synth.MODEL_LAYERED),
]
IDS = [f"{a[0]}x{a[1]}x{a[2]}-sub{b[0]}x{b[1]}x{b[2]}-m{m}" for a, b, m in GEOMS]


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16", "df64"])
@pytest.mark.parametrize("grid,sub,model", GEOMS, ids=IDS)
def test_unfused_equals_fused(grid, sub, model, prec):
    s = synth.system(*grid, 21, model=model)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec)
    try:
        r = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, 3 * s.n)).cuda()
        zf = ctx.apply(r)
        zu = ctx.apply_unfused(r)
        if prec == "df64":
            assert float((zf - zu).abs().max() / zf.abs().max()) <= 1e-13
        else:
            assert torch.equal(zf, zu)
        if prec == "f64":
            d = oracle.decompose(s.row_ptr, s.col, s.val, grid, sub)
            zo = oracle.apply(d.LU, r.cpu().numpy())
            assert np.abs(zu.cpu().numpy() - zo).max() <= 1e-12 * np.abs(zo).max()
    finally:
        ctx.close()
