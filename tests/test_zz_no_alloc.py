"""The allocation-free dot product, ilu0dd_dot_noalloc, against ilu0_dd_dot.

Who needs it: a caller that cannot allocate device memory where it calls the
library -- for example code running while a CUDA graph is being captured
(cudaMalloc is not allowed there), or code that lives inside another
framework's fixed device-memory budget. The entry point therefore keeps its
reduction scratch in a static device array that ships with the library instead
of in a caller-allocated workspace.

The result must equal the context-based dot product bit for bit (both follow
the same fixed summation order), on calls in a row of shrinking size: the
second call's 300 tile partials are padded with zeros to 512, inside the range
the first call (1,104 tiles) left its partials in, so it checks that the zero
padding is written and leftovers in the shared array do not leak into a later
call; a one-tile call follows.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
import synth  # noqa: E402


def _noalloc(lib, x, y, out):
    return lib.ilu0dd_dot_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_int64(x.numel() // 3), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_dot_matches_context_dot_on_two_calls():
    lib = g.load()
    # 1,104 tiles, then 300 tiles (padded to 512: within the first call's
    # leftovers), then 1 tile
    cases = [((64, 64, 69), (16, 16, 8)), ((80, 60, 16), (16, 16, 8)), ((16, 16, 1), (16, 16, 1))]
    for i, (grid, sub) in enumerate(cases):
        s = synth.system(*grid, 3)
        ctx = g.Ilu0DD(s.row_ptr, s.col, s.val, grid, sub)
        rng = np.random.default_rng(100 + i)
        x = torch.from_numpy(rng.normal(size=3 * s.n)).cuda()
        y = torch.from_numpy(rng.normal(size=3 * s.n) * 1e2).cuda()
        ref = ctx.dot(x, y)
        assert (s.n + 255) // 256 == [1104, 300, 1][i]
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, x, y, out) == 0
        torch.cuda.synchronize()
        assert out.item() == ref.item()
        ctx.close()


def test_noalloc_dot_repeated_calls_agree():
    lib = g.load()
    n = 4096 * 3
    x = torch.linspace(-1, 1, n, dtype=torch.float64, device="cuda")
    y = torch.cos(x * 7.0)
    a = torch.empty(1, dtype=torch.float64, device="cuda")
    b = torch.empty(1, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, x, y, a) == 0
    assert _noalloc(lib, x, y, b) == 0
    torch.cuda.synchronize()
    assert a.item() == b.item()
    assert abs(a.item() - float(torch.dot(x, y))) <= 1e-12 * float(torch.dot(x.abs(), y.abs()))


def test_noalloc_dot_rejects_sizes_beyond_its_array():
    lib = g.load()
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.ilu0dd_dot_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_int64(16384 * 256 + 1), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(0))
    assert rc == 8  # ILU0DD_ERR_WORKSPACE
