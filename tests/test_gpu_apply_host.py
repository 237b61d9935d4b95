"""ilu0_dd_apply_host: the apply from and to host buffers, pipelined over
chunks of subdomains, must give the device apply's bits."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402


@pytest.mark.parametrize("grid,sub,prec", [((16, 16, 16), (8, 8, 4), "f64"),      # 16 subdomains
                                           ((33, 17, 9), (16, 16, 8), "f32"),     # 6 (< 8 chunks)
                                           ((64, 64, 64), (16, 16, 8), "df64"),   # 128
                                           ((1, 1, 1), (1, 1, 1), "f64")])        # 1
def test_apply_host_equals_device_apply(grid, sub, prec):
    s = synth.system(*grid, 31, model=synth.MODEL_LAYERED)
    ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub, factor_prec=prec)
    try:
        rng = np.random.default_rng(8)
        for call in range(3):  # repeated calls reuse the context's streams and staging
            r = rng.uniform(-1, 1, 3 * s.n)
            ref = ctx.apply(torch.from_numpy(r).cuda()).cpu().numpy()
            pinned = torch.from_numpy(r).pin_memory()
            z = torch.empty_like(pinned).pin_memory()
            ctx.apply_host(pinned, z)
            assert np.array_equal(z.numpy(), ref)
            zp = ctx.apply_host(r)  # pageable numpy buffers
            assert np.array_equal(zp, ref)
    finally:
        ctx.close()
