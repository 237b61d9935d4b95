"""Device-side numeric setup against the host setup.

The device path (ilu0_dd_setup_planned with scratch: block ILU0 of Algorithm 7
level-scheduled per subdomain, packing of the factor stream and of the SpMV
matrix on the GPU) repeats the host's arithmetic operation by operation
without contraction, so every byte it writes must equal the host path's:
the packed stream in every precision, the sliced-ELL arrays, and the exported
L, U~ = D^-1 U and D^-1. Its error paths (zero pivot, DF64 range) report the
host's codes. Every other GPU test builds its contexts through the device
path (the binding's default), so they also hold it to the oracle.
"""
import numpy as np
import pytest

import synth
from test_gpu_general_pattern import stencil27

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from paper_2508_04917_gb300 import binding as B  # noqa: E402

CASES = [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED),  # ragged edge subdomains
    ((12, 12, 12), (4, 4, 4), synth.MODEL_LAPLACE),
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE),      # one-cell subdomains
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE),    # 1D chain
    ((1, 1, 1), (1, 1, 1), synth.MODEL_LAPLACE),
    ((64, 64, 64), (16, 16, 8), synth.MODEL_LAYERED),
]
IDS = [f"{a[0]}x{a[1]}x{a[2]}-sub{b[0]}x{b[1]}x{b[2]}-m{m}" for a, b, m in CASES]


def _pair(rp, col, val, grid, sub, prec):
    h = g.Ilu0DD(rp, col, val, grid, sub, factor_prec=prec, keep_host=1, device_setup=False)
    d = g.Ilu0DD(rp, col, val, grid, sub, factor_prec=prec, keep_host=1, device_setup=True)
    return h, d


def _same(h, d):
    for what in (B.X_STREAM, B.X_SELL_COL, B.X_SELL_VAL, B.X_L, B.X_UT, B.X_INVD):
        a, b = h.export(what), d.export(what)
        assert a.dtype == b.dtype and a.shape == b.shape
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), what


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "bf16"])
@pytest.mark.parametrize("grid,sub,model", CASES, ids=IDS)
def test_device_setup_is_bit_identical(grid, sub, model, prec):
    s = synth.system(*grid, 7, model=model)
    h, d = _pair(s.row_ptr, s.col, s.val, grid, sub, prec)
    try:
        _same(h, d)
        r = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, 3 * s.n)).cuda()
        assert torch.equal(h.apply(r), d.apply(r))
    finally:
        h.close()
        d.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_device_setup_wide_rows(prec):
    """27-point pattern: rows with more blocks than the descriptor's slot counts."""
    rp, col, val, b, n = stencil27(8, 8, 8, seed=13)
    h, d = _pair(rp, col, val, (8, 8, 8), (4, 4, 4), prec)
    try:
        _same(h, d)
    finally:
        h.close()
        d.close()


def test_device_setup_zero_pivot():
    s = synth.system(4, 4, 4, 1)
    val = s.val.copy()
    q = [q for q in range(s.row_ptr[0], s.row_ptr[1]) if s.col[q] == 0][0]
    val[q] = 0.0
    with pytest.raises(g.Ilu0DDError) as e:
        g.Ilu0DD(s.row_ptr, s.col, val, (4, 4, 4), (2, 2, 2), device_setup=True)
    assert e.value.code == B.ERR_ZERO_PIVOT


def test_device_setup_df64_range():
    s = synth.system(8, 8, 8, 3)
    with pytest.raises(g.Ilu0DDError) as e:
        g.Ilu0DD(s.row_ptr, s.col, s.val * 1e-40, (8, 8, 8), (4, 4, 4), factor_prec="df64", device_setup=True)
    assert e.value.code == B.ERR_INVALID


def test_plan_is_single_use_and_sizes_match():
    """ilu0dd_plan_create reports the same workspace as ilu0_dd_workspace_size; a
    consumed plan is refused."""
    import ctypes
    s = synth.system(12, 10, 9, 2)
    lib = B.load()
    b, keep = B._bsr(s.row_ptr, s.col, s.val)
    geom = B.Geom(12, 10, 9, 4, 4, 4)
    opts = B.default_opts()
    plan = ctypes.c_void_p()
    nw, ns, nref = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.ilu0dd_plan_create(ctypes.byref(b), ctypes.byref(geom), ctypes.byref(opts), ctypes.byref(plan),
                                  ctypes.byref(nw), ctypes.byref(ns)) == 0
    assert lib.ilu0_dd_workspace_size(ctypes.byref(b), ctypes.byref(geom), ctypes.byref(opts), ctypes.byref(nref)) == 0
    assert nw.value == nref.value and ns.value > 0
    ws = torch.empty(nw.value, dtype=torch.uint8, device="cuda")
    sc = torch.empty(ns.value, dtype=torch.uint8, device="cuda")
    ctx = ctypes.c_void_p()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (plan, ctypes.byref(b), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(nw.value),
            ctypes.c_void_p(sc.data_ptr()), ctypes.c_size_t(ns.value), stream, ctypes.byref(ctx))
    assert lib.ilu0_dd_setup_planned(*args) == 0
    ctx2 = ctypes.c_void_p()
    args2 = args[:-1] + (ctypes.byref(ctx2),)
    assert lib.ilu0_dd_setup_planned(*args2) == B.ERR_INVALID
    lib.ilu0_dd_destroy(ctx)
    lib.ilu0dd_plan_destroy(plan)
    del keep
