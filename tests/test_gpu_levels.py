"""Level sets on the device (Algorithm 5, one thread block per subdomain)
against the oracle's level sets of the same dropped pattern: bit-exact, for
box subdomains (3x3 and scalar blocks), the 27-point block stencil, the
graph-partitioned unstructured system, and the degenerate cases (one-row
subdomains, one subdomain holding a whole 1D chain)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2508_04917_gb300 as g  # noqa: E402
from test_gpu_general_pattern import stencil27  # noqa: E402


def check(d):
    lev_l, lev_u, nl, nu = g.levels_device(d.Add.row_ptr, d.Add.col, d.part_ptr)
    ref_l, ref_u = oracle.levels_lower(d.Add)[0], oracle.levels_upper(d.Add)[0]
    assert np.array_equal(lev_l.cpu().numpy(), ref_l)
    assert np.array_equal(lev_u.cpu().numpy(), ref_u)
    pp = np.asarray(d.part_ptr)
    for s in range(len(pp) - 1):
        a, b = pp[s], pp[s + 1]
        assert nl[s].item() == (ref_l[a:b].max() + 1 if b > a else 0)
        assert nu[s].item() == (ref_u[a:b].max() + 1 if b > a else 0)


@pytest.mark.parametrize("grid,sub,model,bs", [
    ((16, 16, 16), (8, 8, 4), synth.MODEL_LAPLACE, 3),
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED, 3),
    ((64, 64, 64), (16, 16, 8), synth.MODEL_LAYERED, 3),
    ((40, 1, 1), (40, 1, 1), synth.MODEL_LAPLACE, 3),   # a chain: 40 levels
    ((4, 3, 2), (1, 1, 1), synth.MODEL_LAPLACE, 3),     # one row per subdomain
    ((33, 17, 9), (16, 16, 8), synth.MODEL_LAYERED, 1),
    ((64, 32, 32), (32, 16, 16), synth.MODEL_LAYERED, 1),  # 8,192-row subdomains
])
def test_device_levels_boxes(grid, sub, model, bs):
    s = synth.system(*grid, 9, model=model, bs=bs)
    check(oracle.decompose(s.row_ptr, s.col, s.val, grid, sub, factor=False))


def test_device_levels_27_point():
    rp, col, val, b, n = stencil27(12, 10, 8, seed=4)
    check(oracle.decompose(rp, col, val, (12, 10, 8), (6, 5, 4), factor=False))


def test_device_levels_partitioned_unstructured():
    s = synth.unstructured(24, 20, 16, 8)
    part, nparts = g.partition_bfs(s.row_ptr, s.col, 512)
    check(oracle.decompose_labeled(s.row_ptr, s.col, s.val, part, nparts, factor=False))
